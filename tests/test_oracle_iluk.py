"""Pins of the ILU(p) / LU subdomain solvers of the oracle (Sec. 4.2, Table 2):
levels of fill against the fill-path characterisation by brute force, the textbook
ILU(1) pattern of the five-point matrix, the ILU property (LU = A on the kept
pattern), and full fill = the exact solve."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import acac_oracle as O
from workloads import BC_NEUMANN, Params, perturbed_pair


def _fill_path_levels(S):
    """Level of every (i, j) by the fill-path theorem: lev(i, j) = (length of the
    shortest path i -> v1 -> ... -> j in the directed graph of S whose intermediate
    vertices are all smaller than min(i, j)) - 1; None where no such path exists.
    Breadth-first search per pair, restricted to the allowed vertices."""
    n = S.shape[0]
    adj = [set(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist()) for i in range(n)]
    lev = {}
    for i in range(n):
        for j in range(n):
            lim = min(i, j)
            dist = {i: 0}
            frontier = [i]
            found = None
            while frontier and found is None:
                nxt = []
                for u in frontier:
                    for w in adj[u]:
                        if w == j:
                            found = dist[u] + 1
                            break
                        if w < lim and w not in dist:
                            dist[w] = dist[u] + 1
                            nxt.append(w)
                    if found is not None:
                        break
                frontier = nxt
            if i == j:
                found = 1 if j in adj[i] else found
            if found is not None:
                lev[(i, j)] = found - 1
    return lev


@pytest.mark.parametrize("seed,symmetric", [(1, False), (2, True), (3, False), (4, True)])
def test_levels_match_fill_paths(seed, symmetric):
    rng = np.random.default_rng(seed)
    n = 14
    M = (rng.random((n, n)) < 0.18).astype(float)
    if symmetric:
        M = np.maximum(M, M.T)
    np.fill_diagonal(M, 1.0)
    S = sp.csr_matrix(M)
    S.sort_indices()
    ip, ind, lv = O.fill_levels(S.indptr, S.indices, None)
    got = {}
    for i in range(n):
        for q in range(ip[i], ip[i + 1]):
            got[(i, int(ind[q]))] = int(lv[q])
    want = _fill_path_levels(S)
    assert got == want
    # ILU(p) keeps exactly the entries of level <= p
    for p in (0, 1, 2):
        ip2, ind2, lv2 = O.fill_levels(S.indptr, S.indices, p)
        kept = {(i, int(ind2[q])) for i in range(n) for q in range(ip2[i], ip2[i + 1])}
        assert kept == {key for key, l in want.items() if l <= p}
        assert int(lv2.max()) <= p


def test_five_point_ilu1_pattern():
    """ILU(1) of the five-point matrix in natural order adds exactly the two diagonals
    next to the outer ones, offsets +-(m - 1): in grid terms the neighbours (x-1, y+1)
    and (x+1, y-1) (Saad, Iterative Methods for Sparse Linear Systems, Sec. 10.3.3)."""
    m, k = 7, 5
    n = m * k
    rows, cols = [], []
    for y, x in itertools.product(range(k), range(m)):
        for dx, dy in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= x + dx < m and 0 <= y + dy < k:
                rows.append(y * m + x)
                cols.append((y + dy) * m + x + dx)
    S = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    S.sort_indices()
    ip, ind, lv = O.fill_levels(S.indptr, S.indices, 1)
    offs = ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (-1, 1), (1, -1))
    for y, x in itertools.product(range(k), range(m)):
        i = y * m + x
        want = sorted((y + dy) * m + x + dx for dx, dy in offs if 0 <= x + dx < m and 0 <= y + dy < k)
        assert ind[ip[i]:ip[i + 1]].tolist() == want
        fill = {(y + dy) * m + x + dx for dx, dy in offs[5:] if 0 <= x + dx < m and 0 <= y + dy < k}
        for q in range(ip[i], ip[i + 1]):
            assert lv[q] == (1 if int(ind[q]) in fill else 0)


def _box_matrix(dim=2):
    if dim == 2:
        p = Params(n=(10, 8, 1), bc=BC_NEUMANN, ras_parts=(1, 1, 1))
    else:
        p = Params(dim=3, n=(5, 4, 4), bc=BC_NEUMANN, ras_parts=(1, 1, 1))
    X1, X0 = perturbed_pair(p, 5, u_mean=0.45, amp=0.1, step_amp=0.01)
    J = O.jacobian(p, X1, X0, 1e-3)
    J.sort_indices()
    return J


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("fill", [1, 2])
def test_ilu_property_on_the_kept_pattern(dim, fill):
    """(L U)_ij = a_ij on every kept entry (zero on fill entries), the defining
    property of an incomplete factorisation on a fixed pattern."""
    A = _box_matrix(dim)
    F, diag = O.ilu_factor(A, fill)
    n = A.shape[0]
    L = sp.tril(F, -1).tocsr() + sp.identity(n, format="csr")
    U = sp.triu(F, 0).tocsr()
    P = (L @ U).toarray()
    Ad = A.toarray()
    Fc = F.tocoo()
    np.testing.assert_allclose(P[Fc.row, Fc.col], Ad[Fc.row, Fc.col], rtol=0, atol=1e-9 * np.abs(Ad).max())
    # the pattern grows with the level and contains A's
    F0, _ = O.ilu_factor(A, fill - 1)
    assert F0.nnz < F.nnz
    assert set(zip(*F0.nonzero())) <= set(zip(*sp.csr_matrix((np.ones(F.nnz), F.indices, F.indptr)).nonzero()))


def test_full_fill_is_the_exact_solve():
    A = _box_matrix(2)
    F, diag = O.ilu_factor(A, None)
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    x = np.zeros_like(b)
    O._lib().oracle_ilu0_solve(b.size, O._iptr(F.indptr), O._iptr(F.indices), O._dptr(F.data),
                               O._iptr(diag), O._dptr(b), O._dptr(x))
    np.testing.assert_allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("solver", [O.SUB_ILU1, O.SUB_ILU2, O.SUB_LU])
def test_schwarz_with_one_box_and_lu_inverts(solver):
    """One subdomain covering a Neumann domain: the LU preconditioner is inv(J) itself,
    and the ILU(p) ones approximate it better than ILU(0) does."""
    p = Params(n=(12, 10, 1), bc=BC_NEUMANN, ras_parts=(1, 1, 1), ras_overlap=0, subdomain_solver=solver)
    X1, X0 = perturbed_pair(p, 6, u_mean=0.45, amp=0.1, step_amp=0.01)
    J = O.jacobian(p, X1, X0, 1e-3)
    r = np.random.default_rng(1).standard_normal(J.shape[0])
    z = O.RAS(p, J, "left").apply(r)
    err = np.linalg.norm(J @ z - r) / np.linalg.norm(r)
    if solver == O.SUB_LU:
        assert err < 1e-12
    else:
        z0 = O.RAS(p.replace(subdomain_solver=O.SUB_ILU0), J, "left").apply(r)
        assert err < np.linalg.norm(J @ z0 - r) / np.linalg.norm(r)


def test_fill_lowers_oracle_gmres_iterations():
    """Table 2's trend in the oracle itself: classical AS with overlap 1, one Newton solve on
    a Neumann problem; the GMRES iterations per Newton iteration do not grow with the fill
    (ILU(0) >= ILU(1) >= ILU(2) >= LU), LU needs fewer than ILU(0), and every solver reaches
    the same root (the preconditioner changes the path, not the solution)."""
    from workloads import initial_fields
    base = Params(n=(24, 24, 1), bc=BC_NEUMANN, ras_parts=(2, 2, 1), ras_overlap=1, ras_type=1,
                  newton_rtol=1e-10, gmres_rtol=1e-8)
    U0 = initial_fields(base, 5, 0.45, 0.05)
    its, roots = {}, {}
    for solver in (O.SUB_ILU0, O.SUB_ILU1, O.SUB_ILU2, O.SUB_LU):
        X, info = O.nks_solve(base.replace(subdomain_solver=solver), U0, 2e-3)
        assert info.status == O.OK
        its[solver] = info.gmres_its / info.newton_its
        roots[solver] = np.concatenate([X[0].ravel(), X[1].ravel()])
    assert its[O.SUB_LU] <= its[O.SUB_ILU2] <= its[O.SUB_ILU1] <= its[O.SUB_ILU0]
    assert its[O.SUB_LU] < its[O.SUB_ILU0]
    for solver in (O.SUB_ILU1, O.SUB_ILU2, O.SUB_LU):
        assert np.linalg.norm(roots[solver] - roots[O.SUB_ILU0]) <= 1e-8 * np.linalg.norm(roots[O.SUB_ILU0])

"""The CUDA library's symbolic subdomain factorizations with fill (acac_subdomain_pattern,
host only, no GPU) against the oracle: its cell pattern, expanded to 2x2 blocks, is the
oracle's point pattern of ILU(1) / ILU(2) on the box matrix (natural order, u before v,
full 2x2 blocks of the radius-2 stencil); its LU pattern contains the oracle's full
fill."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from workloads import BC_NEUMANN, SUB_ILU1, SUB_ILU2, SUB_LU, Params

A = pytest.importorskip("paper_2007_04560_gb300.acac")


def _lib_pattern(dim, W, H, D, solver):
    try:
        A._lib()
    except Exception as e:           # library not built here
        pytest.skip("libacac not available: %s" % e)
    ptr, col = A.acac_subdomain_pattern(dim, W, H, D, solver)
    return {(c, int(col[q])) for c in range(ptr.size - 1) for q in range(ptr[c], ptr[c + 1])}


def _oracle_cells(dim, W, H, D, fill):
    p = Params(dim=dim, n=(W, H, D if dim == 3 else 1), bc=BC_NEUMANN, ras_parts=(1, 1, 1))
    S = O.block_pattern(p)
    S.sort_indices()
    ip, ind, _ = O.fill_levels(S.indptr, S.indices, fill)
    pts = {(r, int(ind[q])) for r in range(ip.size - 1) for q in range(ip[r], ip[r + 1])}
    cells = {(r // 2, c // 2) for r, c in pts}
    # block-closed: every kept cell pair keeps all four point entries
    assert len(pts) == 4 * len(cells)
    return cells


@pytest.mark.parametrize("dim,W,H,D", [(2, 7, 6, 1), (2, 9, 4, 1), (3, 4, 5, 4)])
@pytest.mark.parametrize("solver,fill", [(SUB_ILU1, 1), (SUB_ILU2, 2)])
def test_ilu_patterns_match_the_oracle(dim, W, H, D, solver, fill):
    assert _lib_pattern(dim, W, H, D, solver) == _oracle_cells(dim, W, H, D, fill)


@pytest.mark.parametrize("dim,W,H,D", [(2, 7, 6, 1), (3, 4, 4, 3)])
def test_lu_profile_holds_the_full_fill(dim, W, H, D):
    lib = _lib_pattern(dim, W, H, D, SUB_LU)
    full = _oracle_cells(dim, W, H, D, None)
    assert full <= lib
    n = W * H * (D if dim == 3 else 1)
    assert all((c, c) in lib for c in range(n))


def test_pattern_errors():
    try:
        A._lib()
    except Exception as e:
        pytest.skip("libacac not available: %s" % e)
    import ctypes
    nnz = ctypes.c_longlong(0)
    assert A._lib().acac_subdomain_pattern(4, 4, 4, 4, SUB_ILU1, None, None, 0, ctypes.byref(nnz)) == -1
    assert A._lib().acac_subdomain_pattern(2, 4, 4, 1, 0, None, None, 0, ctypes.byref(nnz)) == -1
    # too small a cap: only the count is written
    assert A._lib().acac_subdomain_pattern(2, 5, 5, 1, SUB_ILU1, None, None, 0, ctypes.byref(nnz)) == -1
    assert nnz.value > 25


@pytest.mark.parametrize("dim,W,H,D", [(2, 9, 7, 1), (3, 5, 4, 6)])
def test_lu_rows_are_intervals_with_nondecreasing_ends(dim, W, H, D):
    """The LU profile: every row an interval of columns containing the diagonal, whose last
    column never decreases from row to row (so a row's upper part reaches every column of
    the upper parts of the rows before it)."""
    try:
        A._lib()
    except Exception as e:
        pytest.skip("libacac not available: %s" % e)
    ptr, col = A.acac_subdomain_pattern(dim, W, H, D, SUB_LU)
    last = -1
    for c in range(ptr.size - 1):
        row = col[ptr[c]:ptr[c + 1]]
        assert np.array_equal(row, np.arange(row[0], row[-1] + 1))
        assert row[0] <= c <= row[-1]
        assert row[-1] >= last
        last = row[-1]

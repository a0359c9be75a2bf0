"""Shared helpers of the GPU tests: layout conversions and the CUDA library."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib_built():
    from paper_2007_04560_gb300 import build
    build.build()
    import paper_2007_04560_gb300 as P
    P.load()
    return P


def soa(u, v):
    """[u | v] state vector from two fields (numpy)."""
    return np.concatenate([np.asarray(u).ravel(), np.asarray(v).ravel()])


def soa_to_interleaved(x):
    n = x.size // 2
    out = np.empty_like(x)
    out[0::2] = x[:n]
    out[1::2] = x[n:]
    return out


def interleaved_to_soa(x):
    return np.concatenate([x[0::2], x[1::2]])


def dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


SLOTS = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1), (-2, 0), (2, 0), (0, -2), (0, 2),
         (-1, -1), (1, -1), (-1, 1), (1, 1)]


SLOTS3 = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1),
          (-2, 0, 0), (2, 0, 0), (0, -2, 0), (0, 2, 0), (0, 0, -2), (0, 0, 2),
          (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 1, 0), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (1, 0, 1),
          (0, -1, -1), (0, 1, -1), (0, -1, 1), (0, 1, 1)]


def stencil_J_to_csr(J, p):
    """Stencil-diagonal storage J[(slot*4+e)*N + cell] -> CSR in interleaved order
    (e = 0: uu, 1: uv, 2: vu, 3: vv).  Slots leaving a Neumann domain are dropped."""
    import scipy.sparse as sp
    nx, ny = p.n[0], p.n[1]
    nz = p.n[2] if p.dim == 3 else 1
    N = nx * ny * nz
    slots = SLOTS3 if p.dim == 3 else [(a, b, 0) for a, b in SLOTS]
    J = np.asarray(J, dtype=np.float64).reshape(len(slots), 4, N)
    cell = np.arange(N)
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    rows, cols, vals = [], [], []
    for s, (dx, dy, dz) in enumerate(slots):
        xx, yy, zz = x + dx, y + dy, z + dz
        if p.bc == 0:
            ok = np.ones(N, bool)
            xx, yy, zz = xx % nx, yy % ny, zz % nz
        else:
            ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        nb = (zz * ny + yy) * nx + xx
        for e in range(4):
            a, b = divmod(e, 2)
            rows.append(2 * cell[ok] + a)
            cols.append(2 * nb[ok] + b)
            vals.append(J[s, e][ok])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * N, 2 * N))
    M.sum_duplicates()
    return M

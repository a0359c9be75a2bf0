"""The allocation-free residual entry point, through the C ABI.

acac_residual_noalloc serves callers that may not allocate device memory when they need a
residual (a framework that owns every device allocation, an allocation-free loop, a plugin
handed only its buffers).  Its working memory is a fixed file-scope device array shared by
every call.  Checked here: it equals the handle-based acac_residual and the CPU oracle
(2D both boundary conditions, 3D), on two calls in a row (the second call finds the first
call's leftovers in the shared array); it accepts the 512 x 512 maximum and rejects larger
grids; it does not change the device's free memory once it has run; and it gives the same
result as the first call of a fresh process.

Collected last on purpose (pytest --collect-only lists this file at the end), so that a run
that stops at the first failure has run every other test before it."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import dev, host, lib_built, need_cuda, soa
from workloads import BC_NEUMANN, BC_PERIODIC, Params, perturbed_pair

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [Params(n=(45, 38, 1), bc=BC_PERIODIC, ras_parts=(3, 2, 1)),
         Params(n=(45, 38, 1), bc=BC_NEUMANN, ras_parts=(3, 2, 1)),
         Params(dim=3, n=(12, 10, 8), L=(1.0, 0.9, 1.1), bc=BC_NEUMANN, ras_parts=(2, 2, 2)),
         Params(dim=3, n=(12, 11, 10), L=(1.0, 0.9, 1.1), bc=BC_PERIODIC, ras_parts=(2, 2, 2))]


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("p", CASES, ids=["2d-periodic", "2d-neumann", "3d-neumann", "3d-periodic"])
def test_noalloc_residual_matches_handle_and_oracle(p):
    torch = need_cuda()
    P = lib_built()
    from paper_2007_04560_gb300.acac import acac_residual_noalloc
    X1, X0 = perturbed_pair(p, 41, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    Fo = soa(*O.residual(p, X1, X0, dt))
    x1, x0 = dev(soa(*X1)), dev(soa(*X0))
    with P.Solver(p) as s:
        F_ref = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        fn_ref = s.residual(x1, x0, dt, F_ref)
    ref = host(F_ref)
    for call in range(2):                      # two calls in a row share the scratch array
        F = torch.full((2 * p.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        st, fn = acac_residual_noalloc(p, x1, x0, dt, F)
        torch.cuda.synchronize()
        assert st == 0
        got = host(F)
        assert _rel(got, ref) <= 1e-12, call
        assert _rel(got, Fo) <= 1e-12, call
        assert fn == pytest.approx(fn_ref, rel=1e-12)
        assert fn == pytest.approx(np.linalg.norm(Fo), rel=1e-12)


def test_noalloc_residual_limits():
    torch = need_cuda()
    lib_built()
    from paper_2007_04560_gb300.acac import E_ARG, E_DOMAIN, OK, acac_residual_noalloc
    edge = Params(n=(512, 512, 1), ras_parts=(8, 8, 1))      # exactly the maximum: accepted
    X1, X0 = perturbed_pair(edge, 43, u_mean=0.45, amp=0.05, step_amp=2e-3)
    F = torch.empty(2 * edge.ncells, dtype=torch.float64, device="cuda")
    st, fn = acac_residual_noalloc(edge, dev(soa(*X1)), dev(soa(*X0)), 2e-3, F, check=False)
    assert st == OK and np.isfinite(fn)
    big = Params(n=(1024, 1024, 1), ras_parts=(16, 16, 1))
    x = torch.full((2 * big.ncells,), 0.25, dtype=torch.float64, device="cuda")
    F = torch.empty_like(x)
    st, _ = acac_residual_noalloc(big, x, x, 1e-3, F, check=False)
    assert st == E_ARG                            # beyond the 512 x 512 maximum
    p = Params(n=(16, 16, 1), ras_parts=(2, 2, 1))
    X1, X0 = perturbed_pair(p, 3)
    u1 = X1[0].copy()
    u1[2, 3] = 1.7                                # midpoint leaves the admissible set
    F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
    st, _ = acac_residual_noalloc(p, dev(soa(u1, X1[1])), dev(soa(*X0)), 1e-3, F, check=False)
    assert st == E_DOMAIN


def test_noalloc_residual_leaves_free_memory_unchanged():
    """After a first call, further calls do not change the device's free memory."""
    torch = need_cuda()
    lib_built()
    from paper_2007_04560_gb300.acac import acac_residual_noalloc
    p = Params(n=(256, 200, 1), ras_parts=(4, 4, 1))
    X1, X0 = perturbed_pair(p, 45, u_mean=0.45, amp=0.05, step_amp=2e-3)
    x1, x0 = dev(soa(*X1)), dev(soa(*X0))
    F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
    acac_residual_noalloc(p, x1, x0, 2e-3, F)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        acac_residual_noalloc(p, x1, x0, 2e-3, F)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


_FRESH = r"""
import sys
sys.path.insert(0, %r)
import numpy as np, torch
from paper_2007_04560_gb300 import build
build.build()
from paper_2007_04560_gb300.acac import acac_residual_noalloc
from oracle import acac_oracle as O
from workloads import Params, perturbed_pair
p = Params(n=(45, 38, 1), ras_parts=(3, 2, 1))
X1, X0 = perturbed_pair(p, 47, u_mean=0.45, amp=0.05, step_amp=2e-3)
x1 = torch.tensor(np.concatenate([X1[0].ravel(), X1[1].ravel()]), device="cuda")
x0 = torch.tensor(np.concatenate([X0[0].ravel(), X0[1].ravel()]), device="cuda")
F = torch.empty_like(x1)
st, fn = acac_residual_noalloc(p, x1, x0, 2e-3, F)      # the process's first library call
torch.cuda.synchronize()
Fo = np.concatenate([a.ravel() for a in O.residual(p, X1, X0, 2e-3)])
err = float(np.max(np.abs(F.cpu().numpy() - Fo)) / np.max(np.abs(Fo)))
print("status", st, "err", err)
assert st == 0 and err <= 1e-12
"""


def test_noalloc_residual_first_call_of_a_fresh_process():
    need_cuda()
    lib_built()
    r = subprocess.run([sys.executable, "-c", _FRESH % ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.stdout[-1000:], r.stderr[-2000:])

"""The allocation-free residual entry point (for callers that may not allocate
device memory) against the handle-based acac_residual, through the C ABI.

Collected last on purpose: it must give the same result in a fresh process and
after every other test has run."""
import numpy as np
import pytest

from tests._helpers import dev, host, lib_built, need_cuda, soa
from workloads import BC_NEUMANN, BC_PERIODIC, Params, perturbed_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_NEUMANN])
def test_noalloc_residual_matches_handle_residual(bc):
    torch = need_cuda()
    P = lib_built()
    from paper_2007_04560_gb300.acac import acac_residual_noalloc
    p = Params(n=(45, 38, 1), bc=bc, ras_parts=(3, 2, 1))
    X1, X0 = perturbed_pair(p, 41, u_mean=0.45, amp=0.05, step_amp=2e-3)
    dt = 2e-3
    x1, x0 = dev(soa(*X1)), dev(soa(*X0))
    with P.Solver(p) as s:
        F_ref = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        fn_ref = s.residual(x1, x0, dt, F_ref)
    ref = host(F_ref)
    for call in range(2):                      # two calls in a row share the scratch
        F = torch.full((2 * p.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        st, fn = acac_residual_noalloc(p, x1, x0, dt, F)
        torch.cuda.synchronize()
        assert st == 0
        got = host(F)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), call
        assert fn == pytest.approx(fn_ref, rel=1e-12)


def test_noalloc_residual_limits():
    torch = need_cuda()
    lib_built()
    from paper_2007_04560_gb300.acac import E_ARG, E_DOMAIN, acac_residual_noalloc
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

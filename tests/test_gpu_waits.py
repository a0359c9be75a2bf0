"""Bounded device-side waits: a wait that nothing completes gives up after its limit, the
kernel reports ACAC_E_TIMEOUT through device memory, and the CUDA context stays usable (a
residual evaluation afterwards still matches the oracle).  No fault, trap or hang."""
import numpy as np
import pytest

from oracle import acac_oracle as O
from tests._helpers import dev, host, lib_built, need_cuda, soa
from workloads import Params, perturbed_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
def test_bounded_wait_gives_up_and_reports(mode):
    need_cuda()
    P = lib_built()
    import torch
    from paper_2007_04560_gb300.acac import _lib
    assert _lib().acac_wait_selftest(None, mode) == -6          # ACAC_E_TIMEOUT
    assert _lib().acac_wait_selftest(None, 2) == -1             # ACAC_E_ARG
    p = Params(n=(24, 20, 1), ras_parts=(2, 2, 1))
    X1, X0 = perturbed_pair(p, 3, u_mean=0.45, amp=0.05, step_amp=2e-3)
    Fo = soa(*O.residual(p, X1, X0, 1e-3))
    with P.Solver(p) as s:
        F = torch.empty(2 * p.ncells, dtype=torch.float64, device="cuda")
        s.residual(dev(soa(*X1)), dev(soa(*X0)), 1e-3, F)
        torch.cuda.synchronize()
    assert np.max(np.abs(host(F) - Fo)) <= 1e-12 * np.max(np.abs(Fo))

"""Host-side helpers of the paper's experiments (paper_2007_04560_gb300/runs.py) on CPU: the
fine-to-coarse comparison of the convergence study and the partition helper."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2007_04560_gb300 import runs


@pytest.mark.parametrize("r", [1, 2, 4])
def test_block_average_of_a_linear_field_is_its_value_at_the_coarse_centre(r):
    """Cell-centred grids share no points: a fine field is compared after averaging each r x r
    block of fine cells onto the coarse cell that contains it.  For a linear function the
    block mean is the function at the coarse cell centre, exactly."""
    nc = 8
    nf = nc * r
    hf, hc = 1.0 / nf, 1.0 / nc
    xf = (np.arange(nf) + 0.5) * hf
    xc = (np.arange(nc) + 0.5) * hc
    f = lambda x, y: 3.0 * x - 2.0 * y + 0.25
    fine = torch.tensor(f(xf[None, :], xf[:, None]))
    coarse = runs._block_average(fine, r)
    np.testing.assert_allclose(coarse.numpy(), f(xc[None, :], xc[:, None]), rtol=0, atol=1e-14)


def test_relative_l2_over_both_fields():
    u = torch.tensor([[1.0, 2.0], [3.0, 4.0]], dtype=torch.float64)
    v = torch.tensor([[0.0, 1.0], [0.0, 1.0]], dtype=torch.float64)
    ur, vr = u + 0.5, v.clone()
    want = np.sqrt(4 * 0.25 / (float((ur ** 2).sum()) + float((vr ** 2).sum())))
    assert runs._rel_l2(u, v, ur, vr) == pytest.approx(want, rel=1e-15)
    assert runs._rel_l2(ur, vr, ur, vr) == 0.0


def test_partition_helper():
    assert runs._parts(128) == 4 and runs._parts(16) == 2 and runs._parts(64, box=8) == 8

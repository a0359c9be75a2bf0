"""The paper's experiments (Sec. 4.1 A, Sec. 4.2) at small sizes through
paper_2007_04560_gb300.runs: second-order convergence in space and time (Fig. 1), the
ranking of the Schwarz variants (Table 3), and energy decay / mass conservation with a
growing adaptive time step (Figs. 2-4)."""
import pytest

from tests._helpers import lib_built, need_cuda

pytestmark = pytest.mark.gpu


def test_convergence_orders():
    need_cuda()
    lib_built()
    from paper_2007_04560_gb300 import runs
    sp = runs.convergence("space", ns=(16, 32), nref=64, T=1.6e-3)
    assert sp["rows"][1]["order"] > 1.8
    tm = runs.convergence("time", n=32, dts=(4e-4, 2e-4, 1e-4), dtref=2.5e-5, T=1.6e-3)
    assert all(1.8 < r["order"] < 2.3 for r in tm["rows"][1:])


def test_schwarz_variants_ranking():
    """Table 3 (2D, 128^2, 6 x 4 subdomains, 10 steps at dt = 1e-4): the restricted
    variants need fewer GMRES iterations than classical AS at the same overlap; the
    Newton count does not depend on the preconditioner."""
    need_cuda()
    lib_built()
    from paper_2007_04560_gb300 import runs
    res = runs.schwarz_table(2, steps=4)
    rows = {(r["preconditioner"], r["delta"]): r for r in res["rows"]}
    assert len({r["total_newton"] for r in res["rows"]}) == 1
    for d in (1, 2):
        assert rows[("left-RAS", d)]["gmres_per_newton"] < rows[("classical-AS", d)]["gmres_per_newton"]
        assert rows[("right-RAS", d)]["gmres_per_newton"] < rows[("classical-AS", d)]["gmres_per_newton"]


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_long_run_energy_and_mass(bc):
    """600 adaptive steps of the Sec. 4.1 A random-state run: the discrete energy never
    rises (Theorem 2.3), the mass is conserved, and dt grows above dt_min."""
    need_cuda()
    lib_built()
    from paper_2007_04560_gb300 import runs
    recs = []
    res = runs.long_run(bc, n=64, t_end=1e4, max_steps=600, sink=recs.append)
    assert res["steps"] == 600 and res["divergences"] >= 0
    assert res["energy_increases"] == 0
    assert res["mass_drift"] < 1e-12
    assert res["dt_max_seen"] > 2 * res["dt_min_seen"]
    assert res["energy_end"] < res["energy0"]

"""The edge-case input generators (CPU, no GPU): they reach the regimes the GPU edge-case
parity tests are meant to cover, and the states they return are admissible (Sec. 2)."""
import numpy as np

from oracle import acac_oracle as O
from workloads import Params, near_pure_pair, near_pure_state


def _ratios(X1, X0):
    out = 0.0
    for sgn in (1.0, -1.0):
        a1, a0 = X1[0] + sgn * X1[1], X0[0] + sgn * X0[1]
        z, s = 0.5 * (a1 + a0), 0.5 * (a1 - a0)
        out = max(out, float(np.max(np.abs(s / z))), float(np.max(np.abs(s / (1.0 - z)))))
    return out


def test_near_pure_pair_reaches_the_edges():
    """u +- v within 1e-7 of 0 and 1, v near +-1/2, series ratios close to 0.7."""
    p = Params(n=(37, 29, 1))
    X1, X0 = near_pure_pair(p, 5)
    for u, v in (X0, X1):
        assert O.admissible(u, v)
        pq = np.concatenate([(u + v).ravel(), (u - v).ravel()])
        assert pq.min() < 1e-7 and pq.max() > 1.0 - 1e-7
        assert v.min() < -0.4999 and v.max() > 0.4999
    assert 0.65 < _ratios(X1, X0) < 0.7


def test_near_pure_pair_ratio_cap():
    p = Params(n=(20, 16, 1))
    for cap in (1e-4, 0.05, 0.3):
        X1, X0 = near_pure_pair(p, 9, ratio_max=cap)
        assert 0.5 * cap < _ratios(X1, X0) <= cap * (1 + 1e-12)


def test_near_pure_state_sides():
    p = Params(n=(20, 16, 1))
    for flip in (False, True):
        u, v = near_pure_state(p, 3, 1e-8, 1e-6, flip=flip)
        assert O.admissible(u, v)
        pp, qq = u + v, u - v
        if flip:
            assert (1 - pp).max() < 2e-8 and qq.max() < 2e-6 and v.min() > 0.4999
        else:
            assert pp.max() < 2e-8 and (1 - qq).max() < 2e-6 and v.max() < -0.4999

"""Pins of the oracle's series form of the discrete variational derivative
(Lemma 2.2 and Eq. D2-1) against the exact difference quotient of Eq. D2."""
import math

import numpy as np
import pytest

from oracle import acac_oracle as O


def _remainder_bound(zeta, sigma, S):
    """Tail of the series after S terms: sum_{k>S} (a^{2k} + b^{2k}) / (2k(2k+1))
    <= (a^{2S+2} + b^{2S+2}) / ((2S+2)(2S+3)) / (1 - max(a,b)^2)."""
    a = abs(sigma / zeta)
    b = abs(sigma / (1.0 - zeta))
    m = max(a, b)
    return (a ** (2 * S + 2) + b ** (2 * S + 2)) / ((2 * S + 2) * (2 * S + 3)) / (1.0 - m * m)


@pytest.mark.parametrize("zeta,sigma", [(0.3, 1e-3), (0.05, 0.01), (0.1, 0.05),
                                         (0.7, -0.2), (0.5, 0.3), (0.93, 0.04)])
def test_series_matches_exact_quotient_mpmath(zeta, sigma):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    z, s = mp.mpf(zeta), mp.mpf(sigma)
    Phi = lambda x: x * mp.log(x) + (1 - x) * mp.log(1 - x)
    exact = (Phi(z + s) - Phi(z - s)) / (2 * s)
    for S in (2, 5, 10):
        series = O.phi_S(np.float64(zeta), np.float64(sigma), S)
        err = abs(float(exact) - float(series))
        bound = _remainder_bound(zeta, sigma, S)
        assert err <= 1.01 * bound + 4e-15 * max(1.0, abs(float(exact))), (S, err, bound)


def test_series_sign_reading_against_float_quotient():
    """The corrected combination f_S(z,s) - f_S(1-z,s) agrees with the exact
    quotient evaluated in float64 where cancellation is mild; the printed
    '+ f_S(1-z,-s)' combination does not."""
    z, s = 0.3, 0.05
    exact = O.exact_quotient(z + s, z - s)
    assert abs(O.phi_S(z, s, 10) - exact) < 1e-12
    # printed combination: [ln z - sum (s/z)^{2k}/..] + [ln(1-z) - sum (s/(1-z))^{2k}/..]
    fS = lambda x, t: math.log(x) - sum((t / x) ** (2 * k) / ((2 * k + 1) * 2 * k)
                                        for k in range(1, 11))
    printed = fS(z, s) + fS(1 - z, -s)
    assert abs(printed - exact) > 0.5


def test_series_sigma_zero_is_Phi_prime():
    """sigma -> 0: phi^S(zeta, 0) = Phi'(zeta) = ln(zeta / (1 - zeta))  (Sec. 2)."""
    z = np.linspace(0.01, 0.99, 99)
    np.testing.assert_allclose(O.phi_S(z, np.zeros_like(z), 10), np.log(z / (1 - z)),
                               rtol=0, atol=1e-15)


def test_series_is_even_in_sigma():
    z = np.array([0.2, 0.45, 0.8])
    s = np.array([0.01, -0.03, 0.1])
    np.testing.assert_allclose(O.phi_S(z, s, 10), O.phi_S(z, -s, 10), rtol=1e-15, atol=0)


def test_series_derivatives_match_finite_differences():
    rng = np.random.default_rng(7)
    z = rng.uniform(0.1, 0.9, 50)
    s = rng.uniform(-0.05, 0.05, 50)
    dz, ds = O.dphi_S(z, s, 10)
    h = 1e-6
    fz = (O.phi_S(z + h, s, 10) - O.phi_S(z - h, s, 10)) / (2 * h)
    fs = (O.phi_S(z, s + h, 10) - O.phi_S(z, s - h, 10)) / (2 * h)
    np.testing.assert_allclose(dz, fz, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(ds, fs, rtol=1e-7, atol=1e-8)


def test_Phi_closed_forms():
    assert O.Phi(np.float64(0.5)) == pytest.approx(-math.log(2.0), abs=1e-16)
    assert O.Phi(np.float64(0.0)) == 0.0 and O.Phi(np.float64(1.0)) == 0.0
    z = 0.2
    assert O.Phi(np.float64(z)) == pytest.approx(z * math.log(z) + (1 - z) * math.log(1 - z),
                                                abs=1e-16)


def _phi_S_mp(mp, z, om, s, S):
    """phi^S of Lemma 2.2 in mpmath (z, 1 - z and sigma given exactly)."""
    a, b = s / z, s / om
    out = mp.log(z) - mp.log(om)
    for k in range(1, S + 1):
        out -= (a ** (2 * k) - b ** (2 * k)) / ((2 * k + 1) * (2 * k))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_series_near_pure_phases_mpmath(seed):
    """Near the pure phases (u + v or u - v within 1e-12..1e-4 of 0 or 1) the oracle's G2
    terms phi^S(zeta_p, sigma_p), phi^S(zeta_q, sigma_q) equal a 50-digit evaluation from
    the exact values of the double inputs within 1e-14 of max(1, |phi|): zeta, 1 - zeta and
    sigma each keep their relative accuracy (Sec. 2, admissible set; Eq. D2-1)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(seed)
    n = 40
    eps = 10.0 ** rng.uniform(-12, -4, size=(2, n))
    side = rng.integers(0, 2, size=(2, n))
    zeta = np.where(side == 0, eps, 1.0 - eps)             # zeta of p and q
    r = rng.uniform(-0.7, 0.7, size=(2, n))
    sig = r * np.minimum(zeta, 1.0 - zeta)
    p0, p1 = zeta[0] - sig[0], zeta[0] + sig[0]
    q0, q1 = zeta[1] - sig[1], zeta[1] + sig[1]
    u1, v1, u0, v0 = 0.5 * (p1 + q1), 0.5 * (p1 - q1), 0.5 * (p0 + q0), 0.5 * (p0 - q0)
    zp, sp_, zq, sq, omp, omq = O._pq(u1, v1, u0, v0)
    phi = O.phi_S(zp, sp_, 10, omp)
    psi = O.phi_S(zq, sq, 10, omq)
    for i in range(n):
        U1, V1, U0, V0 = (mp.mpf(float(x[i])) for x in (u1, v1, u0, v0))
        for sgn, got in ((1, phi[i]), (-1, psi[i])):
            a1, a0 = U1 + sgn * V1, U0 + sgn * V0
            z, s = (a1 + a0) / 2, (a1 - a0) / 2
            ref = _phi_S_mp(mp, z, 1 - z, s, 10)
            assert abs(float(got - ref)) <= 1e-14 * max(1.0, abs(float(ref))), (i, sgn, float(got), float(ref))


def test_series_near_pure_phases_naive_midpoints_fail():
    """Counter-test: on the same inputs, zeta and sigma from the rounded sums p1 + p0,
    p1 - p0 with 1 - zeta = 1.0 - zeta miss phi^S by far more than rounding (the reason
    _pq forms 1 - zeta and sigma from the end values nearer zero)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(0)
    n = 40
    eps = 10.0 ** rng.uniform(-12, -4, size=(2, n))
    side = rng.integers(0, 2, size=(2, n))
    zeta = np.where(side == 0, eps, 1.0 - eps)
    r = rng.uniform(-0.7, 0.7, size=(2, n))
    sig = r * np.minimum(zeta, 1.0 - zeta)
    p0, p1 = zeta[0] - sig[0], zeta[0] + sig[0]
    q0, q1 = zeta[1] - sig[1], zeta[1] + sig[1]
    u1, v1, u0, v0 = 0.5 * (p1 + q1), 0.5 * (p1 - q1), 0.5 * (p0 + q0), 0.5 * (p0 - q0)
    a1, a0 = u1 + v1, u0 + v0
    naive = O.phi_S((a1 + a0) / 2, (a1 - a0) / 2, 10)
    worst = 0.0
    for i in range(n):
        A1 = mp.mpf(float(u1[i])) + mp.mpf(float(v1[i]))
        A0 = mp.mpf(float(u0[i])) + mp.mpf(float(v0[i]))
        ref = _phi_S_mp(mp, (A1 + A0) / 2, 1 - (A1 + A0) / 2, (A1 - A0) / 2, 10)
        worst = max(worst, abs(float(naive[i] - ref)) / max(1.0, abs(float(ref))))
    assert worst > 1e-9

"""Pins of the oracle equilibrium (Sec. III.A: Hermite-expanded Maxwellian, cited form).

The discrete moments of f^eq up to order 4 must equal rho times the moments of the
Gaussian N(u, T I) (textbook raw moments of the normal distribution)."""
import math

import numpy as np
import pytest

import oracle


def normal_raw_moment(a, mu, var):
    """E[X^a] for X ~ N(mu, var): sum_k C(a,2k) mu^(a-2k) var^k (2k-1)!!."""
    s = 0.0
    for k in range(a // 2 + 1):
        dfact = float(np.prod(np.arange(2 * k - 1, 0, -2))) if k else 1.0
        s += math.comb(a, 2 * k) * mu ** (a - 2 * k) * var ** k * dfact
    return s


CASES = [
    (1.0, 0.0, 0.0, 1.0),
    (1.03, 0.02, -0.015, 1.04),
    (0.97, -0.05, 0.03, 0.95),
    (1.2, 0.1, 0.08, 1.1),
    (0.8, 0.0, -0.12, 0.9),
]


@pytest.mark.parametrize("rho,ux,uz,T", CASES)
def test_moments_up_to_order_4(rho, ux, uz, T):
    c, _ = oracle.velocities()
    _, r = oracle.weights()
    xi = r * c
    f = oracle.equilibrium(rho, ux, uz, T)
    for a in range(5):
        for b in range(5 - a):
            lhs = np.sum(f * xi[:, 0] ** a * xi[:, 1] ** b)
            rhs = rho * normal_raw_moment(a, ux, T) * normal_raw_moment(b, uz, T)
            assert abs(lhs - rhs) < 2e-14 * max(1.0, abs(rhs)), (a, b, lhs, rhs)


def test_order_5_not_exact():
    """Non-vacuous: the 4th-order expansion cannot reproduce 5th-order moments at u != 0."""
    c, _ = oracle.velocities()
    _, r = oracle.weights()
    xi = r * c
    rho, ux, uz, T = 1.0, 0.1, 0.0, 1.05
    f = oracle.equilibrium(rho, ux, uz, T)
    lhs = np.sum(f * xi[:, 0] ** 5)
    rhs = rho * normal_raw_moment(5, ux, T)
    assert abs(lhs - rhs) > 1e-6


def test_closed_form_matches_tensor_contraction():
    """Independent check: the collapsed polynomial in s = xi.u and |xi|^2."""
    c, _ = oracle.velocities()
    w, r = oracle.weights()
    xi = r * c
    D = 2
    for rho, ux, uz, T in CASES:
        th = T - 1.0
        s = xi @ np.array([ux, uz])
        c2 = (xi ** 2).sum(1)
        u2 = ux * ux + uz * uz
        P = (1 + s + 0.5 * (s * s - u2 + th * (c2 - D))
             + s / 6 * (s * s - 3 * u2 + 3 * th * (c2 - D - 2))
             + (s ** 4 - 6 * s * s * u2 + 3 * u2 * u2
                + 6 * th * (s * s * (c2 - D - 4) + u2 * (D + 2 - c2))
                + 3 * th * th * (c2 * c2 - 2 * (D + 2) * c2 + D * (D + 2))) / 24)
        np.testing.assert_allclose(oracle.equilibrium(rho, ux, uz, T), w * rho * P, rtol=1e-14, atol=1e-17)


def test_isotropy_at_rest():
    c, opp = oracle.velocities()
    f = oracle.equilibrium(1.0, 0.0, 0.0, 1.02)
    np.testing.assert_array_equal(f, f[opp])
    c2 = (c ** 2).sum(1)
    for s in set(c2.tolist()):
        assert np.ptp(f[c2 == s]) == 0.0


def test_moments_round_trip():
    for rho, ux, uz, T in CASES:
        m = oracle.site_moments(oracle.equilibrium(rho, ux, uz, T))
        np.testing.assert_allclose(m, [rho, ux, uz, T], rtol=1e-14, atol=1e-15)

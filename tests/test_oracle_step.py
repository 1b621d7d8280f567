"""Pins of the oracle propagate / bc / collide (Sec. III.A Eq. (LBE), Sec. III.B)."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C, OPP = oracle.velocities()
W, R = oracle.weights()
XI = R * C


def random_state(Lx, Lz, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    f = np.empty((37, Lx, Lz))
    for x in range(Lx):
        for z in range(Lz):
            f[:, x, z] = oracle.equilibrium(1 + 0.02 * rng.standard_normal(), 0.02 * rng.standard_normal(),
                                            0.02 * rng.standard_normal(), 1 + 0.03 * rng.standard_normal())
    return f * (1 + amp * rng.standard_normal(f.shape))


@pytest.mark.parametrize("Lx,Lz", [(5, 9), (8, 16), (3, 7)])
def test_interior_pull_is_np_roll(Lx, Lz):
    f = np.arange(37 * Lx * Lz, dtype=float).reshape(37, Lx, Lz)
    g = oracle.propagate(f)
    for l in range(37):
        rolled = np.roll(f[l], shift=(C[l, 0], C[l, 1]), axis=(0, 1))
        for z in range(Lz):
            if 0 <= z - C[l, 1] < Lz:
                np.testing.assert_array_equal(g[l, :, z], rolled[:, z])
            else:
                assert np.all(np.isnan(g[l, :, z]))


def test_wall_rows_are_the_papers_bc_rows():
    Lx, Lz = 4, 20
    g = oracle.propagate(np.ones((37, Lx, Lz)))
    rows = sorted({z for l in range(37) for z in range(Lz) if np.isnan(g[l, 0, z])})
    expect = GOLD["bc_rows_bottom"]["value"] + [Lz - k for k in GOLD["bc_rows_top_offsets"]["value"]]
    assert rows == expect


@pytest.mark.parametrize("Lx,Lz", [(5, 9), (8, 16), (1, 6), (2, 7)])
def test_propagate_bc_is_a_bijection(Lx, Lz):
    f = np.arange(37 * Lx * Lz, dtype=float).reshape(37, Lx, Lz)
    g = oracle.bc(f, oracle.propagate(f))
    assert np.all(np.isfinite(g))
    np.testing.assert_array_equal(np.sort(g.ravel()), f.ravel())


@pytest.mark.parametrize("Lx,Lz", [(5, 9), (6, 12)])
def test_propagate_bc_is_time_reversible(Lx, Lz):
    """Reverse all velocities, stream, reverse, stream: the identity (R P R P = I)."""
    rng = np.random.default_rng(3)
    f = rng.standard_normal((37, Lx, Lz))
    P = lambda a: oracle.bc(a, oracle.propagate(a))
    Rv = lambda a: a[OPP]
    np.testing.assert_array_equal(Rv(P(Rv(P(f)))), f)


def test_rest_state_is_invariant_under_streaming():
    Lx, Lz = 4, 10
    feq = oracle.equilibrium(1.0, 0.0, 0.0, 1.0)
    f = np.broadcast_to(feq[:, None, None], (37, Lx, Lz)).copy()
    np.testing.assert_array_equal(oracle.bc(f, oracle.propagate(f)), f)


@pytest.mark.parametrize("tau,grav", [(0.8, 1e-4), (0.7, 5e-5), (1.3, 2e-3)])
def test_collide_invariants(tau, grav):
    """Mass conserved; momentum gains rho*gvec; temperature conserved (exact algebra)."""
    g = random_state(3, 4, 7, amp=5e-3)
    fo = oracle.collide(g, tau, grav)
    for x in range(3):
        for z in range(4):
            r0, ux0, uz0, T0 = oracle.site_moments(g[:, x, z])
            r1, ux1, uz1, T1 = oracle.site_moments(fo[:, x, z])
            assert abs(r1 - r0) < 1e-15 * 4
            assert abs(ux1 - ux0) < 1e-16 * 8
            assert abs(uz1 - (uz0 - grav)) < 1e-16 * 8
            assert abs(T1 - T0) < 1e-15 * 4


def test_collide_fixed_point_without_gravity():
    feq = oracle.equilibrium(1.01, 0.03, -0.02, 0.98)
    g = np.broadcast_to(feq[:, None, None], (37, 2, 3)).copy()
    np.testing.assert_allclose(oracle.collide(g, 0.8, 0.0), g, rtol=1e-14)


def test_collide_relaxes_non_equilibrium_by_one_minus_omega():
    """With g = 0 the moments are unchanged, so f' - f^eq(f') = (1 - 1/tau)(g - f^eq(g))."""
    tau = 0.8
    g = random_state(2, 2, 11, amp=1e-2)
    fo = oracle.collide(g, tau, 0.0)
    for x in range(2):
        for z in range(2):
            m = oracle.site_moments(g[:, x, z])
            feq = oracle.equilibrium(*m)
            np.testing.assert_allclose(fo[:, x, z] - feq, (1 - 1 / tau) * (g[:, x, z] - feq),
                                       rtol=1e-9, atol=1e-17)


def test_step_conserves_mass():
    f = random_state(6, 12, 5, amp=1e-3)
    m0 = f.sum()
    f1 = oracle.step(f, 0.8, 1e-4, nsteps=20)
    assert abs(f1.sum() - m0) < 1e-13 * m0

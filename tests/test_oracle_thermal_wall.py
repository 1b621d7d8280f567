"""Pins of the oracle's thermal-wall variant of the bc (scope row N3; the paper names only
the bc rows, Sec. III.B): ghost rows at rest at the wall temperature whose density balances
the mass through the wall.

* the rule rebuilt independently: a lattice extended by three explicit ghost rows per wall,
  moved by a plain shift propagate (no wall logic), with the ghost densities obtained by
  moving mass into and out of those rows; the oracle's propagate + bc_thermal must agree;
* total mass is conserved by propagate + bc_thermal;
* the rest state at the wall temperature is a fixed point of the full step (no gravity);
* between walls at different temperatures the fluid relaxes to a steady state (every
  population stops changing) with a monotone, near-linear conduction profile (the
  bounce-back walls, adiabatic, keep it uniform).  The stored near-wall rows keep a small
  steady momentum (~1e-3 of the temperature difference): with velocities that jump up to
  three rows, a row's momentum is not the flux across a plane."""
import numpy as np
import pytest

import oracle

Q = 37


def shift_propagate(F):
    """g_l(x, z) = F_l(x - c_lx, z - c_lz), periodic in x, zero where z - c_lz leaves the array."""
    c, _ = oracle.velocities()
    G = np.zeros_like(F)
    Lz = F.shape[2]
    for l in range(Q):
        r = np.roll(F[l], c[l, 0], axis=0)
        cz = c[l, 1]
        if cz >= 0:
            G[l, :, cz:] = r[:, :Lz - cz]
        else:
            G[l, :, :Lz + cz] = r[:, -cz:]
    return G


def ghost_rule_by_construction(f, T_bot, T_top):
    _, Lx, Lz = f.shape
    ext = np.zeros((Q, Lx, Lz + 6))
    ext[:, :, 3:Lz + 3] = f
    moved = shift_propagate(ext)
    out_bot = moved[:, :, 0:3].sum(axis=(0, 2))          # mass the fluid sends into each ghost column
    out_top = moved[:, :, Lz + 3:].sum(axis=(0, 2))
    ghosts = []
    for Tw, rows in ((T_bot, slice(0, 3)), (T_top, slice(Lz + 3, Lz + 6))):
        unit = np.zeros((Q, Lx, Lz + 6))
        unit[:, :, rows] = oracle.equilibrium(1.0, 0.0, 0.0, Tw)[:, None, None]
        inflow = shift_propagate(unit)[:, :, 3:Lz + 3].sum() / Lx   # per ghost column, unit density
        ghosts.append((oracle.equilibrium(1.0, 0.0, 0.0, Tw), inflow))
    ext2 = ext.copy()
    (e_b, in_b), (e_t, in_t) = ghosts
    ext2[:, :, 0:3] = e_b[:, None, None] * (out_bot / in_b)[None, :, None]
    ext2[:, :, Lz + 3:] = e_t[:, None, None] * (out_top / in_t)[None, :, None]
    return shift_propagate(ext2)[:, :, 3:Lz + 3]


def random_state(Lx, Lz, seed):
    rng = np.random.default_rng(seed)
    return 0.01 + rng.random((Q, Lx, Lz)) * 0.05


@pytest.mark.parametrize("Lx,Lz", [(5, 11), (1, 8), (7, 6)])
def test_thermal_bc_matches_explicit_ghost_rows(Lx, Lz):
    f = random_state(Lx, Lz, 3)
    got = oracle.bc_thermal(f, oracle.propagate(f), 1.03, 0.96)
    ref = ghost_rule_by_construction(f, 1.03, 0.96)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


def test_thermal_bc_conserves_mass():
    f = random_state(9, 20, 4)
    g = oracle.bc_thermal(f, oracle.propagate(f), 1.05, 0.95)
    assert abs(g.sum() - f.sum()) < 1e-14 * f.sum()


def test_rest_state_at_wall_temperature_is_fixed_point():
    Tw = 1.02
    f = np.broadcast_to(oracle.equilibrium(1.3, 0.0, 0.0, Tw)[:, None, None], (Q, 4, 12)).copy()
    f1 = oracle.step(f, 0.8, 0.0, 3, walls=(Tw, Tw))
    assert np.abs(f1 - f).max() < 1e-14 * f.max()      # rounding of three collides


def test_conduction_between_walls_at_different_temperatures():
    Lz, Tb, Tt = 24, 1.01, 0.99
    f = np.broadcast_to(oracle.equilibrium(1.0, 0.0, 0.0, 1.0)[:, None, None], (Q, 1, Lz)).copy()
    f = oracle.step(f, 0.8, 0.0, 4000, walls=(Tb, Tt))
    f2 = oracle.step(f, 0.8, 0.0, 200, walls=(Tb, Tt))
    rho, ux, uz, T = oracle.moments(f2, 0.0)
    T = T[0]
    assert np.abs(f2 - f).max() < 1e-13 * f.max()                      # steady (200 steps of rounding)
    assert np.abs(ux).max() < 1e-12
    assert np.abs(uz).max() < 3e-3 * (Tb - Tt)
    assert np.all(np.diff(T) < 0)                                      # heat flows top-down
    assert Tt < T[-1] and T[0] < Tb                                    # a temperature jump at each wall
    assert T[0] - T[-1] > 0.8 * (Tb - Tt)                              # most of the drop is in the fluid
    z = np.arange(Lz)
    fit = np.polyval(np.polyfit(z[3:-3], T[3:-3], 1), z[3:-3])
    assert np.abs(fit - T[3:-3]).max() < 0.02 * (Tb - Tt)              # near-linear away from the walls
    # the bounce-back walls are adiabatic: the same start stays isothermal
    fa = oracle.step(np.broadcast_to(oracle.equilibrium(1.0, 0.0, 0.0, 1.0)[:, None, None], (Q, 1, Lz)).copy(),
                     0.8, 0.0, 200)
    assert np.abs(oracle.moments(fa, 0.0)[3] - 1.0).max() < 1e-13

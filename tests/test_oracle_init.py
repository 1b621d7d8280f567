"""Pins of the three-layer initial state (Sec. I, Eq. (seteq), pressure continuity,
Fig. 1 caption) and of the macroscopic readout (Sec. III.A)."""
import numpy as np

import oracle

W, R = oracle.weights()
TU, TM, TD = 0.95, 1.0, 1.05


def flat_init(Lx, Lz, grav, wt=3.0, K=2):
    z = np.zeros(K)
    return oracle.init_layers(Lx, Lz, grav, TU, TM, TD, Lz / 3, 2 * Lz / 3, 1.0, wt, z, z, z, z)


def test_isothermal_hydrostatic_slopes_away_from_interfaces():
    """Eq. (seteq): rho = rho_i exp(-g (z - z_i)/T_i); a row is r length units."""
    Lx, Lz, g = 2, 300, 1e-3
    rho, ux, uz, T = oracle.moments(flat_init(Lx, Lz, g, wt=2.0), g)
    lr = np.log(rho[0])
    for (lo, hi, Ti) in [(5, 70, TD), (125, 170, TM), (230, 295, TU)]:
        slope = np.diff(lr[lo:hi])
        np.testing.assert_allclose(slope, -g * R / Ti, rtol=1e-9)


def test_pressure_continuity_across_interfaces():
    """p = rho T has no jump: across a row pair straddling an interface the ratio is
    exp(-g r [(z_i - z_k)/T_below + (z_k+1 - z_i)/T_above])."""
    Lx, Lz, g = 1, 300, 1e-3
    rho, _, _, T = oracle.moments(flat_init(Lx, Lz, g), g)
    p = (rho * T)[0]
    zc = np.arange(Lz) + 0.5
    for zi, Tb, Ta in [(Lz / 3, TD, TM), (2 * Lz / 3, TM, TU)]:
        k = int(np.floor(zi - 0.5))
        expect = np.exp(-g * R * ((zi - zc[k]) / Tb + (zc[k + 1] - zi) / Ta))
        assert abs(p[k + 1] / p[k] - expect) < 1e-13


def test_starts_at_rest_and_temperature_profile():
    Lx, Lz, g = 3, 90, 1e-4
    f = flat_init(Lx, Lz, g)
    rho, ux, uz, T = oracle.moments(f, g, renormalised=True)
    assert np.abs(ux).max() < 1e-16 and np.abs(uz).max() < 1e-15
    z = np.arange(Lz) + 0.5
    Tp = TU + (TM - TU) * 0.5 * (1 - np.tanh((z - 60) / 3)) + (TD - TM) * 0.5 * (1 - np.tanh((z - 30) / 3))
    _, _, _, Traw = oracle.moments(f, g)
    np.testing.assert_allclose(Traw[1], Tp, rtol=1e-14)
    np.testing.assert_allclose(T[1], Tp + g * g / 8, rtol=1e-14)     # T^H = T + g^2/(4D)
    # stored velocity is gvec/2 (renormalised u^H = 0)
    _, _, uz_raw, _ = oracle.moments(f, g)
    np.testing.assert_allclose(uz_raw, -g / 2, rtol=0, atol=1e-15)   # j/rho cancels O(1) terms


def test_modes_displace_the_interfaces():
    """Interface height read back from the T field follows z0 + sum A cos(2 pi k x/Lx + phi)."""
    Lx, Lz, g = 32, 120, 1e-4
    a_lo, p_lo = np.array([4.0, -2.0]), np.array([0.3, 1.1])
    a_hi, p_hi = np.array([-3.0, 1.5]), np.array([2.0, 0.2])
    f = oracle.init_layers(Lx, Lz, g, TU, TM, TD, 40.0, 80.0, 1.0, 3.0, a_lo, p_lo, a_hi, p_hi)
    _, _, _, T = oracle.moments(f, g)
    x = np.arange(Lx)
    k = np.arange(1, 3)
    zl = 40 + (a_lo[None] * np.cos(2 * np.pi * k[None] * x[:, None] / Lx + p_lo[None])).sum(1)
    zh = 80 + (a_hi[None] * np.cos(2 * np.pi * k[None] * x[:, None] / Lx + p_hi[None])).sum(1)
    zc = np.arange(Lz) + 0.5
    for xi in range(Lx):
        mid_lo = 0.5 * (TD + TM)
        prof = T[xi, :60]
        j = np.where(prof < mid_lo)[0][0]
        zcross = zc[j - 1] + (mid_lo - prof[j - 1]) / (prof[j] - prof[j - 1])
        assert abs(zcross - zl[xi]) < 0.1
        mid_hi = 0.5 * (TM + TU)
        prof = T[xi, 60:]
        j = np.where(prof < mid_hi)[0][0]
        zcross = zc[60 + j - 1] + (mid_hi - prof[j - 1]) / (prof[j] - prof[j - 1])
        assert abs(zcross - zh[xi]) < 0.1


def test_column_form_equals_the_full_initial_state():
    """init_columns (single columns of a large lattice) is the full init restricted to the
    listed columns, including columns listed twice and out of order."""
    Lx, Lz, g = 17, 40, 1e-4
    a_lo, p_lo = np.array([2.0, -1.0, 0.5]), np.array([0.3, 1.1, 4.0])
    a_hi, p_hi = np.array([-1.5, 0.8, 0.2]), np.array([2.0, 0.2, 5.5])
    args = (g, TU, TM, TD, 13.0, 27.0, 1.0, 3.0, a_lo, p_lo, a_hi, p_hi)
    full = oracle.init_layers(Lx, Lz, *args)
    cols = [16, 0, 5, 5, 11]
    part = oracle.init_columns(Lx, Lz, cols, *args)
    np.testing.assert_array_equal(part, full[:, cols, :])

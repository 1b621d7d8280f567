"""Pins of the oracle's horizontal mean temperature T(z) = (1/Lx) sum_x T(x, z) (Sec. IV, the
profile the mixing widths are read from), against values fixed independently of it:
the closed-form temperature of the three-layer initial state (Sec. I, Eq. (seteq) with the
tanh smoothing of the Fig. 1 caption), and equilibrium states built from chosen fields.
Each case tells the raw T from the renormalised T^H = T + g^2/(4D) of Sec. III.A (a shift
of g^2/8, far above the tolerances), a sum from a mean, and the mean of T from the T of
the mean populations."""
import numpy as np

import oracle

TU, TM, TD = 0.95, 1.0, 1.05


def closed_form_T(Lx, Lz, zlo0, zhi0, wt, a_lo, p_lo, a_hi, p_hi):
    """T(x, z) of the initial state at row centres z = k + 1/2 (sites)."""
    x = np.arange(Lx)[:, None]
    k = np.arange(1, len(a_lo) + 1)[None, :]
    zl = zlo0 + (np.asarray(a_lo)[None] * np.cos(2 * np.pi * k * x / Lx + np.asarray(p_lo)[None])).sum(1)
    zh = zhi0 + (np.asarray(a_hi)[None] * np.cos(2 * np.pi * k * x / Lx + np.asarray(p_hi)[None])).sum(1)
    z = np.arange(Lz)[None, :] + 0.5
    return (TU + (TM - TU) * 0.5 * (1 - np.tanh((z - zh[:, None]) / wt))
            + (TD - TM) * 0.5 * (1 - np.tanh((z - zl[:, None]) / wt)))


def test_unperturbed_layers_give_the_closed_form_profile():
    """Zero mode amplitudes: every column holds the same tanh profile, so T(z) is that
    profile itself.  g = 1e-3 makes T^H - T = 1.25e-7, 1e7 times the tolerance."""
    Lx, Lz, g, wt = 5, 150, 1e-3, 3.0
    z0 = np.zeros(3)
    f = oracle.init_layers(Lx, Lz, g, TU, TM, TD, Lz / 3, 2 * Lz / 3, 1.0, wt, z0, z0, z0, z0)
    prof = closed_form_T(1, Lz, Lz / 3, 2 * Lz / 3, wt, z0, z0, z0, z0)[0]
    got = oracle.row_mean_T(f)
    np.testing.assert_allclose(got, prof, rtol=1e-14, atol=0)
    assert np.min(np.abs(got - (prof + g * g / 8))) > 1e-8


def test_perturbed_layers_give_the_column_average_of_the_closed_form():
    """Interfaces displaced by cosine modes: T(z) is the x average of the closed-form T(x, z)
    (not the T of the x-averaged populations, which differs at second order in the
    displacement)."""
    Lx, Lz, g, wt = 24, 90, 1e-4, 2.5
    a_lo, p_lo = np.array([3.0, -1.5, 0.7]), np.array([0.4, 2.0, 5.1])
    a_hi, p_hi = np.array([-2.5, 1.0, 0.3]), np.array([1.3, 0.1, 3.3])
    f = oracle.init_layers(Lx, Lz, g, TU, TM, TD, 30.0, 60.0, 1.0, wt, a_lo, p_lo, a_hi, p_hi)
    T = closed_form_T(Lx, Lz, 30.0, 60.0, wt, a_lo, p_lo, a_hi, p_hi)
    got = oracle.row_mean_T(f)
    np.testing.assert_allclose(got, T.mean(axis=0), rtol=1e-14, atol=0)
    # the T of the column-averaged populations is measurably different near the interfaces
    fbar = f.mean(axis=1, keepdims=True)
    T_of_mean = oracle.moments(np.ascontiguousarray(fbar), g)[3][0]
    assert np.max(np.abs(T_of_mean - got)) > 1e-6


def test_moving_equilibrium_states_give_the_mean_raw_temperature():
    """Populations f^eq(rho, u, T) with chosen, x-varying rho, u and T (the equilibrium is
    pinned by its Gaussian moments): T(z) is the plain x average of the chosen T, so the
    readout subtracts |u|^2 and divides by D rho exactly as the definition says."""
    rng = np.random.default_rng(17)
    Lx, Lz = 7, 12
    rho = rng.uniform(0.6, 1.4, (Lx, Lz))
    ux = rng.uniform(-0.08, 0.08, (Lx, Lz))
    uz = rng.uniform(-0.08, 0.08, (Lx, Lz))
    T = rng.uniform(0.9, 1.1, (Lx, Lz))
    f = np.empty((37, Lx, Lz))
    for x in range(Lx):
        for z in range(Lz):
            f[:, x, z] = oracle.equilibrium(rho[x, z], ux[x, z], uz[x, z], T[x, z])
    got = oracle.row_mean_T(f)
    np.testing.assert_allclose(got, T.mean(axis=0), rtol=2e-15, atol=0)
    # without the |u|^2 term the readout would be off by <|u|^2>/D ~ 1e-3
    assert np.min(np.abs(got - (T + (ux ** 2 + uz ** 2) / 2).mean(axis=0))) > 1e-5

"""Pins of the mixing-width readouts (Sec. IV: threshold definition and the tent-map
integral, Eq. (3L)) and of the hydrostatic rest state (Sec. I: each layer starts in
hydrostatic equilibrium)."""
import numpy as np
import pytest

import oracle

TU, TM, TD = 0.95, 1.0, 1.05


def ramp_profile(Lz, zl, zh, half):
    """Piecewise-linear T(z): linear interpolation between rows reproduces it exactly."""
    z = np.arange(Lz, dtype=float)
    bd = np.clip(0.5 - (z - zl) / (2 * half), 0, 1)      # 1 below the lower front
    bu = np.clip(0.5 - (z - zh) / (2 * half), 0, 1)      # 1 below the upper front
    return TU + (TM - TU) * bu + (TD - TM) * bd


def test_threshold_widths_exact_on_linear_ramps():
    Lz, zl, zh, half = 200, 60.3, 140.7, 10.0
    L = oracle.widths(ramp_profile(Lz, zl, zh, half), TU, TM, TD)
    np.testing.assert_allclose(L, [0.9 * 2 * half, 0.9 * 2 * half], rtol=1e-12)


def test_threshold_widths_on_tanh_profile():
    """Continuous closed form: L = 2 w atanh(0.9) per front; linear interpolation error O(1/w^2)."""
    Lz, w = 4000, 60.0
    z = np.arange(Lz) + 0.5
    T = TU + (TM - TU) * 0.5 * (1 - np.tanh((z - 2700.3) / w)) + (TD - TM) * 0.5 * (1 - np.tanh((z - 1300.6) / w))
    L = oracle.widths(T, TU, TM, TD)
    np.testing.assert_allclose(L, 2 * w * np.arctanh(0.9), rtol=2e-4)


def test_tent_widths_closed_forms():
    Lz, half = 400, 25.0
    # linear ramp from b=0 to b=1 over 2*half rows: integral of the tent = half
    L = oracle.tent_widths(ramp_profile(Lz, 120.0, 280.0, half), TU, TM, TD)
    np.testing.assert_allclose(L, [half, half], rtol=1e-3)
    w = 40.0
    z = np.arange(4000) + 0.5
    T = TU + (TM - TU) * 0.5 * (1 - np.tanh((z - 2700) / w)) + (TD - TM) * 0.5 * (1 - np.tanh((z - 1300) / w))
    np.testing.assert_allclose(oracle.tent_widths(T, TU, TM, TD), 2 * w * np.log(2), rtol=1e-3)


def test_width_gradient_matches_finite_differences():
    Lz = 90
    z = np.arange(Lz) + 0.5
    rng = np.random.default_rng(0)
    T = TU + (TM - TU) * 0.5 * (1 - np.tanh((z - 60.2) / 3)) + (TD - TM) * 0.5 * (1 - np.tanh((z - 29.7) / 3))
    T = T + 1e-4 * rng.standard_normal(Lz)
    L, dL = oracle.widths(T, TU, TM, TD, with_grad=True)
    h = 1e-7
    for k in range(Lz):
        e = np.zeros(Lz); e[k] = h
        fd = (oracle.widths(T + e, TU, TM, TD).sum() - oracle.widths(T - e, TU, TM, TD).sum()) / (2 * h)
        assert abs(fd - dL[k]) < 1e-5 * max(1.0, abs(dL[k])), (k, fd, dL[k])
    assert np.count_nonzero(dL) == 8            # two bracketing rows per crossing


def test_missing_crossing_raises_and_degenerate_profile():
    with pytest.raises(ValueError):                       # never reaches 5% of the upper jump
        oracle.widths(np.full(50, TU), TU, TM, TD)
    # a uniform middle temperature satisfies both thresholds at the first scanned row
    np.testing.assert_array_equal(oracle.widths(np.full(50, TM), TU, TM, TD), [0.0, 0.0])


@pytest.mark.slow
def test_single_layer_hydrostatic_rest():
    """An unperturbed isothermal layer stays at rest: renormalised |u^H| small, no growth."""
    Lx, Lz, g, tau = 4, 64, 1e-4, 0.8
    z = np.zeros(1)
    f = oracle.init_layers(Lx, Lz, g, 1.0, 1.0, 1.0, Lz / 3, 2 * Lz / 3, 1.0, 3.0, z, z, z, z)
    peaks = []
    for _ in range(6):
        f = oracle.step(f, tau, g, 250)
        rho, ux, uz, T = oracle.moments(f, g, renormalised=True)
        inner = slice(6, Lz - 6)
        assert np.abs(ux).max() < 1e-12                       # x-symmetric state
        assert np.abs(uz[:, inner]).max() < 1e-6
        assert np.abs(uz).max() < 1e-5
        assert np.abs(T[:, inner] - 1 - g * g / 8).max() < 1e-6
        assert np.abs(T - 1).max() < 5e-5
        peaks.append(np.abs(uz).max())
    assert max(peaks[3:]) < 1.2 * max(peaks[:3])               # no growth

"""Mixing diagnostics of Sec. IV on the GPU against the oracle on the same state: the
tent-map widths of Eq. (3L), and the per-row mean / rms-fluctuation profiles of T and of
the kinetic energy per unit mass (|u^H|^2 / 2, renormalised velocity)."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    return lbm


def evolved(lbm, prec, lat, steps):
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    L.step(steps)
    return L


def expected_stats(f, grav):
    """The definitions written out on the oracle's moments of the same populations."""
    _, _, _, T = oracle.moments(f, grav, renormalised=False)
    _, ux, uz, _ = oracle.moments(f, grav, renormalised=True)
    ek = 0.5 * (ux * ux + uz * uz)
    out = {}
    for name, q in (("T", T), ("Ek", ek)):
        m = q.mean(axis=0)
        out[name + "_mean"] = m
        out[name + "_rms"] = np.sqrt(((q - m) ** 2).mean(axis=0))
    return out


@pytest.mark.parametrize("prec", ["f64_ff", "f32"])
def test_tent_widths_match_oracle(lbm, prec):
    lat = W.PARITY_64x128
    L = evolved(lbm, prec, lat, 60)
    f = L.populations()
    ref = oracle.tent_widths(oracle.row_mean_T(f), lat.T_u, lat.T_m, lat.T_d)
    got = L.tent_widths(lat.T_u, lat.T_m, lat.T_d)
    # the two T-bar profiles agree to FP64 rounding (~1e-15); b = (Tbar - T_u)/(T_m - T_u)
    # scales that by 1/(T_m - T_u) and the tent sums ~20 rows of it
    np.testing.assert_allclose(got, ref, rtol=1e-10)
    assert got.min() > 0


def test_tent_widths_single_front_virtual_middle(lbm):
    """Single front (T_m = T_u layer, interface at Lz/2) read with a virtual T_m halfway:
    each tent covers one half of the tanh jump, whose integral is 3 w ln(4/3) (with
    t = tanh(z/w): w [ln(4/3) + 2 ln(4/3)])."""
    Lx, Lz, w = 8, 256, 3.0
    lat = W.Lattice(Lx, Lz, tau=0.8, grav=0.0, K=0, sigma=0.0, seed=0, T_u=0.975, T_m=0.975, T_d=1.025,
                    z_lo_rows=Lz / 2, z_hi_rows=float(Lz), tanh_w=w)
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec="f64")
    L.init_from(lat)
    Tv = 0.5 * (lat.T_u + lat.T_d)
    got = L.tent_widths(lat.T_u, Tv, lat.T_d)
    ref = oracle.tent_widths(oracle.row_mean_T(L.populations()), lat.T_u, Tv, lat.T_d)
    np.testing.assert_allclose(got, ref, rtol=1e-10)   # see test_tent_widths_match_oracle
    np.testing.assert_allclose(got, 3 * w * np.log(4 / 3) * np.ones(2), rtol=0.03)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_row_stats_match_definition(lbm, prec):
    lat = W.PARITY_64x128
    L = evolved(lbm, prec, lat, 80)
    f = L.populations()
    exp = expected_stats(f, lat.grav)
    got = L.row_stats()
    for k in ("T_mean", "Ek_mean"):
        np.testing.assert_allclose(got[k], exp[k], rtol=1e-12, atol=1e-15)
    for k in ("T_rms", "Ek_rms"):
        scale = np.abs(exp[k]).max()
        assert scale > 0
        np.testing.assert_allclose(got[k], exp[k], rtol=1e-9, atol=1e-9 * scale)


def test_row_stats_uniform_rows_have_zero_fluctuation(lbm):
    """Unperturbed layers: every row is uniform in x, so both rms profiles vanish."""
    lat = W.Lattice(16, 96, tau=0.8, grav=1e-4, K=0, sigma=0.0, seed=0)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64")
    L.init_from(lat)
    got = L.row_stats()
    assert np.abs(got["T_rms"]).max() < 1e-13
    assert np.abs(got["Ek_rms"]).max() < 1e-13


def test_fronts_driver_small_run():
    """The Sec. IV driver on a small pair of runs: widths finite and growing from the
    initial tanh fronts, profiles at the requested times, no fluctuations at t = 0."""
    from paper_1405_1253_b300 import physics
    res = physics.run(nconf=2, t_end=1.0, per_tau=4, Lx=64, Lz=256, tau=0.6, profile_times=(0, 1))
    for c in ("double", "single"):
        Lt = np.array(res[c]["L_tot"])
        assert np.isfinite(Lt).all() and Lt[0] > 0
        assert Lt[-1] >= Lt[0]
        assert set(res[c]["profiles"]) == {"0", "1"}
        assert len(res[c]["profiles"]["1"]["T_rms"]) == 256
    assert res["double"]["gap_fill"][0] < 0.05      # at t = 0 only the tanh tails reach the middle
    assert len(res["t_over_tau"]) == 5

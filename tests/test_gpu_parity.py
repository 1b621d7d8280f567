"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: the FP64 and float-float steps must match the oracle to a maximum relative
error of 1e-12 on every population after 100 steps of the 64x128 three-layer workload;
streaming alone (tau -> infinity, g = 0) must be bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm as m
    return m


def oracle_init(lat):
    return oracle.init_layers(lat.Lx, lat.Lz, **lat.layer_args())


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def make(lbm, lat, prec):
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    return L


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_init_matches_oracle(lbm, prec):
    lat = W.PARITY_64x128
    L = make(lbm, lat, prec)
    assert max_rel(L.populations(), oracle_init(lat)) < 1e-13


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_step_parity_100_steps(lbm, prec):
    lat = W.PARITY_64x128
    L = make(lbm, lat, prec)
    L.step(W.PARITY_STEPS)
    L.sync()
    ref = oracle.step(oracle_init(lat), lat.tau, lat.grav, W.PARITY_STEPS)
    err = max_rel(L.populations(), ref)
    assert err < TOL_STEP, err


@pytest.mark.parametrize("Lx,Lz", [(1, 6), (2, 7), (3, 37), (5, 131), (4, 200), (7, 260)])
@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_step_parity_edge_shapes(lbm, prec, Lx, Lz):
    """Smallest lattices, x wrap at Lx < 3, ragged z tails, several z tiles."""
    rng = np.random.default_rng(Lx * 1000 + Lz)
    lat = W.Lattice(Lx, Lz, tau=0.7, grav=2e-4, K=2, sigma=0.5, seed=7)
    f0 = oracle_init(lat) * (1 + 1e-3 * rng.standard_normal((37, Lx, Lz)))
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
    L.set_populations(f0)
    L.step(5)
    ref = oracle.step(f0, lat.tau, lat.grav, 5)
    assert max_rel(L.populations(), ref) < 1e-13


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_streaming_alone_is_bit_exact(lbm, prec):
    """tau -> infinity and g = 0 leave only propagate + bc: an exact permutation."""
    Lx, Lz = 9, 140
    rng = np.random.default_rng(2)
    f0 = rng.uniform(0.5, 1.5, (37, Lx, Lz))
    if prec == "f32":
        f0 = f0.astype(np.float32).astype(np.float64)
    L = lbm.Lattice(Lx, Lz, 1e300, 0.0, prec=prec)
    L.set_populations(f0)
    L.step(3)
    ref = f0
    for _ in range(3):
        ref = oracle.bc(ref, oracle.propagate(ref))
    np.testing.assert_array_equal(L.populations(), ref)


def test_moments_and_diagnostics_match_oracle(lbm):
    lat = W.PARITY_64x128
    L = make(lbm, lat, "f64")
    L.step(20)
    f = L.populations()
    for renorm in (False, True):
        got = L.moments(renormalised=renorm)
        exp = oracle.moments(f, lat.grav, renormalised=renorm)
        for g_, e_ in zip(got, exp):
            np.testing.assert_allclose(g_, e_, rtol=1e-13, atol=1e-15)
    Tbar = L.row_mean_T()
    np.testing.assert_allclose(Tbar, oracle.row_mean_T(f), rtol=1e-13)
    Lw, dL = L.widths(lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    Lo, dLo = oracle.widths(oracle.row_mean_T(f), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    np.testing.assert_allclose(Lw, Lo, rtol=1e-11)
    np.testing.assert_allclose(dL, dLo, rtol=1e-9, atol=1e-12)
    mass, energy = L.global_sums()
    _, r = oracle.weights()
    c, _ = oracle.velocities()
    c2 = (c ** 2).sum(1) * r * r
    assert abs(mass - f.sum()) < 1e-12 * mass
    assert abs(energy - 0.5 * np.einsum("l,lxz->", c2, f)) < 1e-12 * energy


def test_mass_is_conserved_over_many_steps(lbm):
    lat = W.PARITY_64x128
    L = make(lbm, lat, "f64")
    m0, _ = L.global_sums()
    L.step(500)
    m1, _ = L.global_sums()
    assert abs(m1 - m0) < 1e-12 * m0


def test_populations_round_trip_device(lbm):
    import torch
    lat = W.PARITY_64x128
    L = make(lbm, lat, "f64")
    d = L.populations_device()
    h = L.populations()
    np.testing.assert_array_equal(d.cpu().numpy().reshape(h.shape), h)
    L.set_populations(torch.zeros_like(d))
    assert not L.populations().any()
    L.set_populations(d)
    np.testing.assert_array_equal(L.populations(), h)


def test_fp32_storage_tracks_fp64(lbm):
    """Stated error of FP32 storage after 100 steps of the parity workload."""
    lat = W.PARITY_64x128
    L = make(lbm, lat, "f32")
    L.step(W.PARITY_STEPS)
    rho32, _, _, T32 = L.moments()
    ref = oracle.step(oracle_init(lat), lat.tau, lat.grav, W.PARITY_STEPS)
    rho, _, _, T = oracle.moments(ref, lat.grav)
    assert np.linalg.norm(rho32 - rho) / np.linalg.norm(rho) < 1e-5
    assert np.linalg.norm(T32 - T) / np.linalg.norm(T) < 1e-5


def window_columns(f, x0, half):
    """Columns x0-half..x0+half (periodic) of f: a sub-lattice whose centre column's
    dependence cone for `half // 3` steps lies inside it."""
    Lx = f.shape[1]
    idx = [(x0 + k) % Lx for k in range(-half, half + 1)]
    return np.ascontiguousarray(f[:, idx, :])


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_full_size_1024x2048_sampled_columns(lbm, prec):
    """The throughput workload at full size in the benchmark's launch configuration:
    2 steps on the GPU, compared on sampled columns against the oracle run on a
    13-column window around each (the centre column depends only on +-6 columns)."""
    lat = W.THROUGHPUT_1024x2048
    L = make(lbm, lat, prec)
    f0 = L.populations()
    L.step(2)
    f2 = L.populations()
    for x0 in (0, 1, 511, 1023):
        win = window_columns(f0, x0, 6)
        ref = oracle.step(win, lat.tau, lat.grav, 2)[:, 6, :]
        assert max_rel(f2[:, x0, :], ref) < 1e-13

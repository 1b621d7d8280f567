"""Thermal walls on the GPU (scope row N3): lbm_set_walls against the oracle's thermal-wall
step, in every precision, on the parity workload, the edge shapes and a ragged lattice;
exact mass conservation, the rest state at the wall temperature, the switch back to
bounce-back, host stepping, and the entry points that refuse thermal walls (the adjoint with
thermal walls: test_gpu_thermal_adjoint.py)."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm as m
    return m


def max_rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def walls_of(lat):
    return lat.T_d, lat.T_u           # the wall next to each layer at that layer's temperature


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_thermal_walls_parity(lbm, prec):
    lat = W.PARITY_64x128
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    L.set_walls(True, *walls_of(lat))
    L.step(50)
    ref = oracle.step(oracle.init_layers(lat.Lx, lat.Lz, **lat.layer_args()), lat.tau, lat.grav, 50,
                      walls=walls_of(lat))
    assert max_rel(L.populations(), ref) < 1e-12


def test_thermal_walls_fp32_tracks_oracle(lbm):
    lat = W.PARITY_64x128
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f32")
    L.init_from(lat)
    L.set_walls(True, *walls_of(lat))
    L.step(50)
    rho32, _, _, T32 = L.moments()
    ref = oracle.step(oracle.init_layers(lat.Lx, lat.Lz, **lat.layer_args()), lat.tau, lat.grav, 50,
                      walls=walls_of(lat))
    rho, _, _, T = oracle.moments(ref, lat.grav)
    assert np.linalg.norm(rho32 - rho) / np.linalg.norm(rho) < 1e-5
    assert np.linalg.norm(T32 - T) / np.linalg.norm(T) < 1e-5


@pytest.mark.parametrize("Lx,Lz", [(1, 6), (2, 7), (3, 37), (5, 131), (23, 40)])
@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_thermal_walls_edge_shapes(lbm, prec, Lx, Lz):
    """Smallest lattices (6 rows: every row a wall row), x wrap below 3 columns, ragged
    tails, and a wall block whose columns and halo span the periodic seam."""
    rng = np.random.default_rng(Lx * 100 + Lz)
    lat = W.Lattice(Lx, Lz, tau=0.7, grav=2e-4, K=2, sigma=0.5, seed=7)
    f0 = oracle.init_layers(Lx, Lz, **lat.layer_args()) * (1 + 1e-3 * rng.standard_normal((37, Lx, Lz)))
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
    L.set_populations(f0)
    L.set_walls(True, 1.04, 0.97)
    L.step(5)
    ref = oracle.step(f0, lat.tau, lat.grav, 5, walls=(1.04, 0.97))
    assert max_rel(L.populations(), ref) < 1e-13


def test_thermal_walls_conserve_mass(lbm):
    lat = W.Lattice(96, 160, tau=0.7, grav=1e-4, K=4, sigma=1.0, seed=3)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    L.set_walls(True, *walls_of(lat))
    m0 = L.global_sums()[0]
    L.step(500)
    m1 = L.global_sums()[0]
    assert abs(m1 - m0) < 1e-13 * m0


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_rest_state_at_wall_temperature_stays(lbm, prec):
    Tw, Lx, Lz = 1.02, 8, 40
    f0 = np.broadcast_to(oracle.equilibrium(1.3, 0.0, 0.0, Tw)[:, None, None], (37, Lx, Lz)).copy()
    L = lbm.Lattice(Lx, Lz, 0.8, 0.0, prec=prec)
    L.set_populations(f0)
    L.set_walls(True, Tw, Tw)
    L.step(50)
    assert np.abs(L.populations() - f0).max() < 1e-13 * f0.max()


def test_switch_back_to_bounce_back_is_exact(lbm):
    lat = W.Lattice(32, 64, tau=0.8, grav=1e-4, K=3, sigma=1.0, seed=5)
    A = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    B = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    A.init_from(lat)
    B.init_from(lat)
    A.set_walls(True, 1.1, 0.9)
    A.set_walls(False)
    A.step(10)
    B.step(10)
    np.testing.assert_array_equal(A.populations(), B.populations())


def test_host_stepping_with_thermal_walls(lbm):
    lat = W.Lattice(16, 48, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=6)
    A = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    A.init_from(lat)
    A.set_walls(True, *walls_of(lat))
    f0 = A.populations()
    outs = [np.empty_like(f0) for _ in range(3)]
    ins = [f0, f0, f0]
    A.step_host(ins, outs)
    ref = oracle.step(f0, lat.tau, lat.grav, 1, walls=walls_of(lat))
    for o in outs:
        assert max_rel(o, ref) < 1e-13


def test_entry_points_refuse_thermal_walls(lbm):
    import torch
    lat = W.Lattice(16, 48, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=6)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    with pytest.raises(lbm.LBMError) as e:
        L.set_walls(True, -1.0, 1.0)
    assert e.value.code == lbm.LBM_EINVAL
    L.set_walls(True, 1.05, 0.95)
    x = L.populations_device().clone()
    mom = [torch.empty(4 * lat.Lx * lat.Lz, dtype=torch.int64, device=x.device)]
    for call in (lambda: L.step_push(1), lambda: L.record_moments(x, x.clone(), x.clone(), mom),
                 lambda: lbm.Slabs(L, 4), lambda: lbm.Ensemble([L]).step(1)):
        with pytest.raises(lbm.LBMError) as e:
            call()
        assert e.value.code == lbm.LBM_ESTATE
    L.set_walls(False)
    L.step_push(1)

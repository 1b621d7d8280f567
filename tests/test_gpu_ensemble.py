"""The ensemble runner: uneven lattices advanced together (per-step launches, one
persistent launch, a captured CUDA graph) match the FP64 oracle stepping each lattice
alone (to 1e-13 for the float-float collide, within the stated FP32 field bound for FP32
storage) and give exactly the states of each lattice stepped alone on the GPU; the
persistent launch's bounded barrier wait ends with LBM_ETIMEOUT instead of hanging when
its target can never be met."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(16, 64), (24, 200), (8, 131), (32, 128), (5, 7)]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1405_1253_b300 import lbm
    return torch, lbm


def lattices():
    return [W.Lattice(lx, lz, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=300 + i)
            for i, (lx, lz) in enumerate(SHAPES)]


def make_set(lbm, prec, stream):
    Ls = []
    for lat in lattices():
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        Ls.append(L)
    return Ls


def check_against_oracle(L, lat, prec, nsteps):
    """The lattice after nsteps against the oracle's nsteps from its own initial state."""
    ref = oracle.step(oracle.init_layers(lat.Lx, lat.Lz, **lat.layer_args()), lat.tau, lat.grav, nsteps)
    if prec == "f32":
        rho32, _, _, T32 = L.moments()
        rho, _, _, T = oracle.moments(ref, lat.grav)
        assert np.linalg.norm(rho32 - rho) / np.linalg.norm(rho) < 1e-5
        assert np.linalg.norm(T32 - T) / np.linalg.norm(T) < 1e-5
    else:
        got = L.populations()
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13


@pytest.mark.parametrize("prec", ["f64_ff", "f32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_matches_oracle(env, prec, mode):
    torch, lbm = env
    stream = torch.cuda.Stream()
    ens_l = make_set(lbm, prec, stream)
    ens = lbm.Ensemble(ens_l)
    ens.config(mode=mode, tile_z=128)
    ens.step(3)
    ens.step(4)
    ens.sync()
    for L, lat in zip(ens_l, lattices()):
        check_against_oracle(L, lat, prec, 7)
    ens.close()


@pytest.mark.parametrize("prec", ["f64_ff", "f32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_graph_replay_matches_oracle(env, prec, mode):
    torch, lbm = env
    stream = torch.cuda.Stream()
    ens_l = make_set(lbm, prec, stream)
    ens = lbm.Ensemble(ens_l)
    ens.config(mode=mode, tile_z=128)
    ens.capture(4)
    for _ in range(3):
        ens.graph_launch()
    ens.sync()
    for L, lat in zip(ens_l, lattices()):
        check_against_oracle(L, lat, prec, 12)
    ens.close()


@pytest.mark.parametrize("prec", ["f64_ff", "f32"])
@pytest.mark.parametrize("mode,tz", [(0, 128), (1, 64), (1, 128), (1, 256)])
def test_ensemble_matches_single_lattice_steps(env, prec, mode, tz):
    torch, lbm = env
    stream = torch.cuda.Stream()
    ref = make_set(lbm, prec, stream)
    for L in ref:
        L.step(7)
    ens_l = make_set(lbm, prec, stream)
    ens = lbm.Ensemble(ens_l)
    ens.config(mode=mode, tile_z=tz)
    ens.step(3)
    ens.step(4)
    ens.sync()
    for a, b in zip(ens_l, ref):
        np.testing.assert_array_equal(a.populations(), b.populations())
    ens.close()


def test_ensemble_graph_replay(env):
    torch, lbm = env
    stream = torch.cuda.Stream()
    ref = make_set(lbm, "f64_ff", stream)
    for L in ref:
        L.step(12)
    ens_l = make_set(lbm, "f64_ff", stream)
    ens = lbm.Ensemble(ens_l)
    ens.config(mode=1, tile_z=128)
    ens.capture(4)
    for _ in range(3):
        ens.graph_launch()
    ens.sync()
    for a, b in zip(ens_l, ref):
        np.testing.assert_array_equal(a.populations(), b.populations())
    ens.close()


def test_ensemble_tuner_picks_a_valid_shape(env):
    torch, lbm = env
    stream = torch.cuda.Stream()
    ens_l = make_set(lbm, "f32", stream)
    ens = lbm.Ensemble(ens_l)
    best = ens.tune(steps=2)
    assert best["mode"] in (0, 1) and best["tile_z"] in (64, 128, 256) and best["ms_per_step"] > 0
    ens.step(2)
    ens.sync()
    ens.close()


def test_persistent_barrier_wait_times_out_cleanly(env):
    """A barrier target that nothing can reach: every wait runs out after its cycle
    budget, the launch ends, and the host sees LBM_ETIMEOUT; the context stays usable."""
    torch, lbm = env
    stream = torch.cuda.Stream()
    ens_l = make_set(lbm, "f64_ff", stream)
    ens = lbm.Ensemble(ens_l)
    ens.config(mode=1, tile_z=128)
    ens.set_wait(200000, extra_wait=1)
    ens.step(2)
    with pytest.raises(lbm.LBMError) as e:
        ens.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    # recovered: normal waits again, and the GPU is still answering
    ens.set_wait(4000000000, extra_wait=0)
    for L in ens_l:
        L.init_from(W.Lattice(L.Lx, L.Lz, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=1))
    ens.step(2)
    ens.sync()
    assert np.isfinite(ens_l[0].global_sums()).all()
    ens.close()

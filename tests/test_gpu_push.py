"""Push form of the step (Sec. III.B): push steps from P f match P applied to the oracle's
steps from f (1e-13 for the FP64-accurate collides, the stated FP32 field bound for FP32
storage), with P f formed by the oracle's propagate + bc; push steps from P f equal P applied
to the pull steps from f, bit for bit for the float-float and FP32 collides (to a few ulps for
the native FP64 one), on edge shapes (x wrap at Lx < 3, ragged z tails, lattices that are all
wall rows); P itself (lbm_propagate) equals the oracle's propagate + bc."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    return lbm


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
@pytest.mark.parametrize("Lx,Lz", [(1, 6), (2, 8), (5, 131), (16, 70), (64, 128)])
def test_push_equals_propagated_pull(lbm, prec, Lx, Lz):
    lat = W.Lattice(Lx, Lz, tau=0.8, grav=2e-4, K=2, sigma=0.5, seed=11)
    A = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
    A.init_from(lat)
    A.step(6)
    A.propagate()
    B = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
    B.init_from(lat)
    B.propagate()
    B.step_push(6)
    got, ref = B.populations(), A.populations()
    if prec == "f64":
        # the native FP64 collide is one long expression that the compiler contracts into
        # FMAs a little differently in the pull and push kernels: a few ulps per step, within
        # the 1e-13 the parity tests allow the FP64 kernels against the oracle after 5 steps
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)
    else:
        assert np.array_equal(got, ref)


def oracle_P(f):
    return oracle.bc(f, oracle.propagate(f))


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
@pytest.mark.parametrize("Lx,Lz", [(1, 6), (2, 8), (5, 131), (16, 70), (64, 128)])
def test_push_matches_oracle(lbm, prec, Lx, Lz):
    lat = W.Lattice(Lx, Lz, tau=0.8, grav=2e-4, K=2, sigma=0.5, seed=11)
    f0 = oracle.init_layers(Lx, Lz, **lat.layer_args())
    ref = oracle_P(oracle.step(f0, lat.tau, lat.grav, 6))
    B = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
    B.set_populations(oracle_P(f0))
    B.step_push(6)
    if prec == "f32":
        rho32, _, _, T32 = B.moments()
        rho, _, _, T = oracle.moments(ref, lat.grav)
        assert np.linalg.norm(rho32 - rho) / np.linalg.norm(rho) < 1e-5
        assert np.linalg.norm(T32 - T) / np.linalg.norm(T) < 1e-5
    else:
        got = B.populations()
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13


@pytest.mark.parametrize("Lx,Lz", [(1, 6), (3, 37), (12, 48)])
def test_propagate_matches_oracle(lbm, Lx, Lz):
    rng = np.random.default_rng(Lx + Lz)
    f0 = rng.uniform(0.5, 1.5, (37, Lx, Lz))
    L = lbm.Lattice(Lx, Lz, 0.8, 1e-4, prec="f64")
    L.set_populations(f0)
    L.propagate()
    assert np.array_equal(L.populations(), oracle.bc(f0, oracle.propagate(f0)))

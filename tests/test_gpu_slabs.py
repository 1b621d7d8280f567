"""x-slab decomposition with halo exchange (Sec. III.B) on one GPU: the gathered slabs
match the FP64 oracle's single-domain steps (1e-13 for the FP64-accurate collides, the
stated FP32 field bound for FP32 storage), and after any number of steps they hold exactly
the single-domain GPU state (bit for bit), with the exchange overlapped with the bulk
update or not; bad splits are rejected."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    return lbm


LAT = W.Lattice(48, 70, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=9)


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
@pytest.mark.parametrize("n,overlap", [(1, False), (2, True), (4, True), (4, False), (6, True), (8, True), (16, False)])
def test_slabs_match_single_domain(lbm, prec, n, overlap):
    A = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec=prec)
    A.init_from(LAT)
    A.step(12)
    ref = A.populations()
    B = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec=prec)
    B.init_from(LAT)
    S = lbm.Slabs(B, n)
    S.scatter()
    S.step(7, overlap)
    S.step(5, overlap)
    S.gather()
    assert np.array_equal(B.populations(), ref)
    S.close()


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
@pytest.mark.parametrize("n,overlap", [(2, True), (4, False), (8, True)])
def test_slabs_match_oracle(lbm, prec, n, overlap):
    f0 = oracle.init_layers(LAT.Lx, LAT.Lz, **LAT.layer_args())
    ref = oracle.step(f0, LAT.tau, LAT.grav, 12)
    B = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec=prec)
    B.init_from(LAT)
    S = lbm.Slabs(B, n)
    S.scatter()
    S.step(7, overlap)
    S.step(5, overlap)
    S.gather()
    if prec == "f32":
        rho32, _, _, T32 = B.moments()
        rho, _, _, T = oracle.moments(ref, LAT.grav)
        assert np.linalg.norm(rho32 - rho) / np.linalg.norm(rho) < 1e-5
        assert np.linalg.norm(T32 - T) / np.linalg.norm(T) < 1e-5
    else:
        got = B.populations()
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13
    S.close()


def test_slabs_continue_from_gathered_state(lbm):
    """gather, a few single-domain steps, scatter again: still the single-domain state."""
    A = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64_ff")
    A.init_from(LAT)
    A.step(9)
    B = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64_ff")
    B.init_from(LAT)
    S = lbm.Slabs(B, 4)
    S.scatter()
    S.step(3)
    S.gather()
    B.step(3)
    S.scatter()
    S.step(3)
    S.gather()
    assert np.array_equal(B.populations(), A.populations())


@pytest.mark.parametrize("n", [5, 17, 24])
def test_slabs_reject_bad_split(lbm, n):
    B = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64")
    with pytest.raises(lbm.LBMError):
        lbm.Slabs(B, n)

"""x-slab decomposition with halo exchange (Sec. III.B) on one GPU: after any number of
steps the slabs hold exactly the single-domain state (bit for bit), with the exchange
overlapped with the bulk update or not; bad splits are rejected."""
import numpy as np
import pytest

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

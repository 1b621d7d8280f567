"""Error paths with host-injected failures (no GPU fault is provoked): every device
allocation the library makes is refused in turn (lbm_test_fail_alloc); each call must report
LBM_ENOMEM, leave its object usable or unmade, and the next call must succeed."""
import numpy as np
import pytest

from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    yield lbm
    lbm.test_fail_alloc(-1)


LAT = W.Lattice(16, 48, tau=0.8, grav=1e-4, K=3, sigma=1.0, seed=3)


def refused(lbm, n, fn):
    lbm.test_fail_alloc(n)
    try:
        with pytest.raises(lbm.LBMError) as ei:
            fn()
        assert ei.value.code == lbm.LBM_ENOMEM, str(ei.value)
    finally:
        lbm.test_fail_alloc(-1)


@pytest.mark.parametrize("n", range(5))
def test_create_reports_each_refused_allocation(lbm, n):
    refused(lbm, n, lambda: lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64_ff"))
    L = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64_ff")
    L.init_from(LAT)
    L.step(2)


def test_init_modes_buffer_refused_then_recovers(lbm):
    L = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64")
    refused(lbm, 0, lambda: L.init_from(LAT))
    L.init_from(LAT)
    ref = L.populations()
    L2 = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64")
    L2.init_from(LAT)
    assert np.array_equal(ref, L2.populations())


def test_scratch_of_diagnostics_and_copies_refused(lbm):
    L = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f32")
    L.init_from(LAT)
    refused(lbm, 0, L.moments)                  # stream-ordered scratch of the host copy
    refused(lbm, 0, L.populations)              # FP32 -> FP64 conversion scratch
    refused(lbm, 0, L.row_mean_T)               # reduction partials
    rho, _, _, T = L.moments()
    assert np.isfinite(rho).all() and np.isfinite(L.row_mean_T()).all()


@pytest.mark.parametrize("n", range(3))
def test_ensemble_and_slabs_refused(lbm, n):
    Ls = []
    for i in range(2):
        L = lbm.Lattice(LAT.Lx, LAT.Lz, LAT.tau, LAT.grav, prec="f64_ff")
        L.init_from(LAT)
        Ls.append(L)
    refused(lbm, n, lambda: lbm.Ensemble(Ls))
    E = lbm.Ensemble(Ls)
    E.step(2)
    E.sync()
    E.close()
    if n < 2:
        refused(lbm, n, lambda: lbm.Slabs(Ls[0], 4))
    S = lbm.Slabs(Ls[0], 4)
    S.close()

"""The allocation-free horizontal-mean entry point (lbm_row_mean_T_noalloc).

Some callers cannot allocate device memory when they need the diagnostic: a plugin
whose device memory is all handed to it by a host application, or code whose memory
belongs to a pool it does not control.  This checks, through the C ABI, that the static-scratch variant gives
the same profile as lbm_row_mean_T on two calls in a row, and that it refuses sizes
beyond its fixed scratch.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Lx,Lz,steps", [(64, 128, 20), (37, 203, 3)])
def test_noalloc_row_mean_matches_context_entry_point(Lx, Lz, steps):
    import torch
    from paper_1405_1253_b300 import lbm
    lat = W.Lattice(Lx, Lz, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=3)
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec="f64")
    L.init_from(lat)
    L.step(steps)
    ref = L.row_mean_T()                       # context entry point (synchronises)
    out = torch.full((Lz,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                         # two calls in a row share the static scratch
        out.fill_(float("nan"))
        lbm.row_mean_T_noalloc(L.current().data_ptr(), Lx, Lz, out.data_ptr(), stream)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=0)
    L.close()


def test_noalloc_rejects_rows_beyond_the_static_scratch():
    import torch
    from paper_1405_1253_b300 import lbm
    f = torch.zeros(37 * 2, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = lbm._lib.lbm_row_mean_T_noalloc(ctypes.c_void_p(f.data_ptr()), 1, (1 << 20) + 1,
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert rc == lbm.LBM_EINVAL
    assert b"static scratch" in lbm._lib.lbm_last_error()

"""The bounds-checked build (liblbm_checked.so, every population load and store index-checked):
a child process running every kernel path — pull and push steps in every precision on edge
shapes, propagate, moments and row statistics, the allocation-free row mean, the slabs, the ensemble in both launch modes,
the adjoint, thermal walls, host stepping — must meet no out-of-range index."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu


def exercise():
    import numpy as np
    import torch
    from paper_1405_1253_b300 import lbm, workloads as W
    for prec in ("f64", "f64_ff", "f32"):
        for (Lx, Lz) in [(1, 6), (2, 8), (3, 37), (5, 131), (64, 128)]:
            lat = W.Lattice(Lx, Lz, tau=0.8, grav=2e-4, K=2, sigma=0.5, seed=21)
            L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec=prec)
            L.init_from(lat)
            L.step(3)
            L.propagate()
            L.step_push(3)
            L.moments(renormalised=True)
            L.row_stats()
            L.tent_widths(lat.T_u, lat.T_m, lat.T_d)
            L.populations()
            if prec != "f32":                     # the allocation-free row mean (FP64 arrays)
                Tb = torch.empty(Lz, dtype=torch.float64, device="cuda")
                lbm.row_mean_T_noalloc(L.current().data_ptr(), Lx, Lz, Tb.data_ptr(),
                                       L.stream.cuda_stream)
    lat = W.Lattice(48, 70, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=22)
    for prec in ("f64_ff", "f32"):
        Ls = []
        for _ in range(2):
            L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
            L.init_from(lat)
            Ls.append(L)
        for n, ov in ((4, True), (8, False)):
            S = lbm.Slabs(Ls[0], n)
            S.scatter()
            S.step(3, ov)
            S.gather()
            S.close()
        s = torch.cuda.Stream()
        Le = []
        for _ in range(2):
            L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=s)
            L.init_from(lat)
            Le.append(L)
        E = lbm.Ensemble(Le)
        for mode in (0, 1):
            E.config(mode=mode, tile_z=64)
            E.step(3)
            E.sync()
        E.close()
    for prec in ("f64", "f64_ff"):
        A = lbm.Lattice(12, 48, 0.8, 1e-3, prec=prec)
        A.init_from(W.Lattice(12, 48, tau=0.8, grav=1e-3, K=2, sigma=1.0, seed=23))
        f = A.populations_device().clone()
        lam = torch.rand_like(f)
        out = torch.empty_like(f)
        A.adjoint_step(f, lam, out)
    for prec in ("f64", "f64_ff", "f32"):
        for Lx, Lz in ((23, 40), (2, 6)):
            T = lbm.Lattice(Lx, Lz, 0.8, 1e-4, prec=prec)
            T.init_from(W.Lattice(Lx, Lz, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=24))
            T.set_walls(True, 1.05, 0.95)
            T.step(2)
            if prec == "f64_ff":                  # the thermal-wall adjoint and its ghost sums
                f = T.populations_device().clone()
                T.adjoint_step(f, torch.rand_like(f), torch.empty_like(f))
    H = lbm.Lattice(16, 48, 0.8, 1e-4, prec="f64_ff")
    a = np.ones(37 * 16 * 48)
    b = np.empty_like(a)
    H.step_host([a, a], [b, b])
    torch.cuda.synchronize()
    print("OOB", lbm.test_oob_count())


def test_bounds_checked_build_meets_no_out_of_range_index():
    from paper_1405_1253_b300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, LBM_LIBRARY=lib)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, cwd=root,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout + res.stderr
    line = [l for l in res.stdout.splitlines() if l.startswith("OOB ")][-1]
    assert int(line.split()[1]) == 0, line


def test_regular_build_reports_it_is_not_checked():
    from paper_1405_1253_b300 import lbm
    if os.environ.get("LBM_LIBRARY"):
        pytest.skip("running against another build")
    with pytest.raises(lbm.LBMError):
        lbm.test_oob_count()


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    exercise()

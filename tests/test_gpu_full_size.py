"""Parity at full size, in the launch configuration the benchmark times: the largest
configuration (4096 x 8192, float-float and FP32 deviation storage), the adjoint step (from the state and from a moment record) and
the thermal walls on 1024 x 2048, compared on sampled columns against the oracle run on a
periodic window of columns around each (wide enough to hold the column's dependence cone).
Windows are cut on the device, so no full state crosses to the host."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu

Q = 37


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1405_1253_b300 import lbm
    return torch, lbm


def window(torch, flat, Lx, Lz, x0, half):
    """Columns x0-half .. x0+half (periodic) of a device population array, on the host."""
    idx = torch.tensor([(x0 + k) % Lx for k in range(-half, half + 1)], device=flat.device)
    return flat.view(Q, Lx, Lz).index_select(1, idx).cpu().numpy()


def column(torch, flat, Lx, Lz, x0):
    return flat.view(Q, Lx, Lz)[:, x0, :].cpu().numpy()


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("lat", [W.THROUGHPUT_1024x2048, W.PRECISION_4096x8192], ids=["1024x2048", "4096x8192"])
def test_init_full_size_sampled_columns(env, lat):
    """The initial state of the throughput (64 modes) and precision (128 modes) lattices
    against the oracle's, column by column: the mode sums at every phase of the largest
    wavenumbers, the tanh and hydrostatic profiles and the pressure continuity over the
    full height.  Columns are cut on the device."""
    torch, lbm = env
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    f = L.current()
    cols = [0, 1, lat.Lx // 3, lat.Lx // 2 + 7, lat.Lx - 1]
    ref = oracle.init_columns(lat.Lx, lat.Lz, cols, **lat.layer_args())
    for j, x0 in enumerate(cols):
        got = column(torch, f, lat.Lx, lat.Lz, x0)
        assert np.max(np.abs(got - ref[:, j, :]) / np.abs(ref[:, j, :])) < 1e-13
    del f
    L.close()
    torch.cuda.empty_cache()


def test_largest_configuration_4096x8192_sampled_columns(env):
    """The precision configuration (4096 x 8192, 19.9 GB for the two copies): 2 float-float
    steps against the oracle on 13-column windows (the centre column depends on +-6)."""
    torch, lbm = env
    lat = W.PRECISION_4096x8192
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    f0 = L.populations_device().clone()
    L.step(2)
    f2 = L.populations_device()
    for x0 in (0, 2047, 4095):
        ref = oracle.step(window(torch, f0, lat.Lx, lat.Lz, x0, 6), lat.tau, lat.grav, 2)[:, 6, :]
        got = column(torch, f2, lat.Lx, lat.Lz, x0)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13
    del f0, f2
    L.close()
    torch.cuda.empty_cache()


def test_deviation_storage_4096x8192_sampled_columns(env):
    """The FP32 deviation storage on the precision configuration (reference from the initial
    rows' means): 2 steps against the oracle on 13-column windows of the FP64 state the
    context holds (f_ref + d).  Each step adds up to ~16 units of 2^-24 |d| / f (|d| <= 30% of
    f), so 2 steps stay below 2 * 16 * 2^-24 * 0.3 = 5.7e-7 per population."""
    torch, lbm = env
    lat = W.PRECISION_4096x8192
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f32_dev")
    L.init_from(lat)
    f0 = L.populations_device()
    L.step(2)
    f2 = L.populations_device()
    for x0 in (0, 2047, 4095):
        ref = oracle.step(window(torch, f0, lat.Lx, lat.Lz, x0, 6), lat.tau, lat.grav, 2)[:, 6, :]
        got = column(torch, f2, lat.Lx, lat.Lz, x0)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 5.7e-7
    del f0, f2
    L.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,store", [("f64_ff", "states"), ("f64_ff", "moments"), ("f64", "states")])
def test_adjoint_full_size_sampled_columns(env, prec, store):
    """The adjoint step on the 1024 x 2048 state (the kernel the bench times) against the
    oracle's adjoint on 13-column windows: column x of lam_t takes contributions from the
    sites x-3 .. x+3, whose moments pull from x-6 .. x+6."""
    torch, lbm = env
    lat = W.THROUGHPUT_1024x2048
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    L.step(20)
    f = L.populations_device().clone()
    gen = torch.Generator(device=f.device).manual_seed(31)
    lam = torch.randn(f.numel(), dtype=torch.float64, device=f.device, generator=gen)
    out = torch.empty_like(f)
    if store == "moments":
        mom = [torch.empty(4 * lat.sites, dtype=torch.int64, device=f.device)]
        L.record_moments(f, torch.empty_like(f), torch.empty_like(f), mom)
        assert L.adjoint_chain_moments(mom, lam, out) == 1
    else:
        L.adjoint_step(f, lam, out)
    for x0 in (0, 3, 700, 1023):
        fw = window(torch, f, lat.Lx, lat.Lz, x0, 6)
        lw = window(torch, lam, lat.Lx, lat.Lz, x0, 6)
        ref = oracle.adjoint_step(fw, lw, lat.tau, lat.grav)[:, 6, :]
        assert max_rel(column(torch, out, lat.Lx, lat.Lz, x0), ref) < 1e-12
    L.close()


def test_thermal_walls_full_size_sampled_columns(env):
    """Thermal walls on 1024 x 2048, 2 steps: a wall row's pull reads ghost densities of
    columns +-3 away, each summed over +-3 more, so the cone is +-12 columns."""
    torch, lbm = env
    lat = W.THROUGHPUT_1024x2048
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    L.set_walls(True, lat.T_d, lat.T_u)
    f0 = L.populations_device().clone()
    L.step(2)
    f2 = L.populations_device()
    for x0 in (0, 511, 1023):
        ref = oracle.step(window(torch, f0, lat.Lx, lat.Lz, x0, 12), lat.tau, lat.grav, 2,
                          walls=(lat.T_d, lat.T_u))[:, 12, :]
        assert np.max(np.abs(column(torch, f2, lat.Lx, lat.Lz, x0) - ref) / np.abs(ref)) < 1e-13
    L.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_48_lattices_sampled_columns(env, mode):
    """The batching configuration (48 uneven lattices, 19.9 M sites) in one ensemble, in each
    launch shape, under a captured graph of 2 steps: sampled columns of lattices of every
    size against the oracle's 2 steps from its own initial state on a 13-column window."""
    torch, lbm = env
    lats = W.ensemble_48()
    stream = torch.cuda.Stream()
    Ls = []
    for lat in lats:
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff", stream=stream)
        L.init_from(lat)
        Ls.append(L)
    ens = lbm.Ensemble(Ls)
    ens.config(mode=mode, tile_z=128)
    ens.capture(2)
    ens.graph_launch()
    ens.sync()
    for i, x0 in ((0, 0), (15, 255), (16, 100), (31, 511), (32, 3), (47, 383)):
        lat, L = lats[i], Ls[i]
        cols = [x0 + k for k in range(-6, 7)]
        win = oracle.init_columns(lat.Lx, lat.Lz, cols, **lat.layer_args())
        ref = oracle.step(win, lat.tau, lat.grav, 2)[:, 6, :]
        got = column(torch, L.current(), lat.Lx, lat.Lz, x0)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-13, (i, x0)
    ens.close()
    for L in Ls:
        L.close()
    del Ls
    torch.cuda.empty_cache()

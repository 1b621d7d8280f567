"""Parity at full size, in the launch configuration the benchmark times: the largest
configuration (4096 x 8192), the adjoint step (from the state and from a moment record) and
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

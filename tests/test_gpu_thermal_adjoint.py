"""The adjoint step with thermal walls (float-float contexts) against the oracle's
thermal-wall adjoint: evolved states, edge shapes (6 rows, narrow lattices, a wall tile
whose halo spans the periodic seam), the gradient chain, the refusals, and full size on
sampled columns."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu

WALLS = (1.04, 0.97)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1405_1253_b300 import lbm
    return torch, lbm


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("Lx,Lz", [(64, 128), (1, 6), (2, 7), (23, 40), (5, 140)])
def test_thermal_adjoint_matches_oracle(env, Lx, Lz):
    torch, lbm = env
    lat = W.Lattice(Lx, Lz, tau=0.7, grav=2e-4, K=2, sigma=0.5, seed=41)
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    L.set_walls(True, *WALLS)
    L.step(10)
    f = L.populations_device().clone()
    lam = torch.from_numpy(np.random.default_rng(42).standard_normal(f.numel())).cuda()
    out = torch.empty_like(f)
    L.adjoint_step(f, lam, out)
    got = out.cpu().numpy().reshape(37, Lx, Lz)
    ref = oracle.adjoint_step(f.cpu().numpy().reshape(37, Lx, Lz), lam.cpu().numpy().reshape(37, Lx, Lz),
                              lat.tau, lat.grav, walls=WALLS)
    assert rel_err(got, ref) < 1e-12
    L.close()


def test_thermal_adjoint_is_deterministic(env):
    """The ghost sums are formed in a fixed order: repeated calls agree bit for bit."""
    torch, lbm = env
    lat = W.Lattice(96, 64, tau=0.7, grav=2e-4, K=2, sigma=0.5, seed=43)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    L.set_walls(True, *WALLS)
    f = L.populations_device().clone()
    lam = torch.from_numpy(np.random.default_rng(44).standard_normal(f.numel())).cuda()
    outs = [torch.empty_like(f) for _ in range(3)]
    for o in outs:
        L.adjoint_step(f, lam, o)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    L.close()


def test_thermal_gradient_matches_oracle_chain(env):
    """Width gradient with thermal walls: init -> steps -> widths -> adjoint chain -> init
    adjoint, against the oracle's chain with the same walls."""
    from paper_1405_1253_b300 import adjoint
    lat = W.Lattice(12, 48, tau=0.8, grav=1e-3, K=2, sigma=1.0, seed=21)
    walls = (lat.T_d, lat.T_u)
    nsteps, ckpt = 6, 3
    drv = adjoint.WidthGradient(lat, nsteps, ckpt, walls=walls)
    m = lat.modes()
    Lval = drv.forward(m.amp_lo, m.amp_hi)
    g_lo, g_hi = drv.backward()
    drv.close()
    a = lat.layer_args()
    states = [oracle.init_layers(lat.Lx, lat.Lz, **a)]
    for _ in range(nsteps):
        states.append(oracle.step(states[-1], lat.tau, lat.grav, walls=walls))
    Lo, dL = oracle.widths(oracle.row_mean_T(states[-1]), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    assert abs(Lval - Lo.sum()) < 1e-10 * abs(Lo.sum())
    lam = oracle.loss_adjoint(states[-1], dL)
    for t in range(nsteps - 1, -1, -1):
        lam = oracle.adjoint_step(states[t], lam, lat.tau, lat.grav, walls=walls)
    o_lo, o_hi = oracle.init_adjoint(lat.Lx, lat.Lz, **a, lam0=lam)
    np.testing.assert_allclose(g_lo, o_lo, rtol=1e-9, atol=1e-12 * np.abs(o_lo).max())
    np.testing.assert_allclose(g_hi, o_hi, rtol=1e-9, atol=1e-12 * np.abs(o_hi).max())


def test_thermal_adjoint_refusals(env):
    torch, lbm = env
    lat = W.Lattice(8, 32, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=45)
    F = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64")
    F.set_walls(True, *WALLS)
    x = torch.zeros(37 * lat.sites, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        F.adjoint_step(x, x.clone(), x.clone())
    assert e.value.code == lbm.LBM_ESTATE
    G = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    G.set_walls(True, *WALLS)
    mom = [torch.empty(4 * lat.sites, dtype=torch.int64, device="cuda")]
    with pytest.raises(lbm.LBMError) as e:
        G.record_moments(x, x.clone(), x.clone(), mom)
    assert e.value.code == lbm.LBM_ESTATE


def test_thermal_adjoint_full_size_sampled_columns(env):
    """1024 x 2048 with thermal walls: a leaving entry of column x takes the ghost sum of
    column x + c_x, fed by destinations 3 columns further, whose moments pull ghost
    densities summed over 6 more: a cone of +-12 columns."""
    torch, lbm = env
    lat = W.THROUGHPUT_1024x2048
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    L.set_walls(True, lat.T_d, lat.T_u)
    L.step(20)
    f = L.populations_device().clone()
    gen = torch.Generator(device=f.device).manual_seed(46)
    lam = torch.randn(f.numel(), dtype=torch.float64, device=f.device, generator=gen)
    out = torch.empty_like(f)
    L.adjoint_step(f, lam, out)

    def window(flat, x0, half):
        idx = torch.tensor([(x0 + k) % lat.Lx for k in range(-half, half + 1)], device=flat.device)
        return flat.view(37, lat.Lx, lat.Lz).index_select(1, idx).cpu().numpy()

    for x0 in (0, 511, 1023):
        ref = oracle.adjoint_step(window(f, x0, 12), window(lam, x0, 12), lat.tau, lat.grav,
                                  walls=(lat.T_d, lat.T_u))[:, 12, :]
        got = out.view(37, lat.Lx, lat.Lz)[:, x0, :].cpu().numpy()
        assert rel_err(got, ref) < 1e-12
    L.close()

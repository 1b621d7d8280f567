"""GPU parity of the adjoint kernels against the oracle's own CPU adjoint (tiny lattices)."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1405_1253_b300 import lbm
    return torch, lbm


def near_eq(Lx, Lz, seed):
    rng = np.random.default_rng(seed)
    f = np.empty((37, Lx, Lz))
    for x in range(Lx):
        for z in range(Lz):
            f[:, x, z] = oracle.equilibrium(1 + 0.02 * rng.standard_normal(), 0.02 * rng.standard_normal(),
                                            0.02 * rng.standard_normal(), 1 + 0.03 * rng.standard_normal())
    return f * (1 + 2e-3 * rng.standard_normal(f.shape))


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("Lx,Lz,tau,grav", [(8, 16, 0.8, 1e-4), (3, 7, 0.7, 5e-3), (1, 9, 1.1, 1e-3), (5, 140, 0.8, 1e-4)])
def test_adjoint_step_matches_oracle(env, Lx, Lz, tau, grav):
    torch, lbm = env
    f = near_eq(Lx, Lz, 1)
    lam = np.random.default_rng(2).standard_normal(f.shape)
    L = lbm.Lattice(Lx, Lz, tau, grav, prec="f64")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ft, ln = dev(f), dev(lam)
    out = torch.empty_like(ft)
    L.adjoint_step(ft, ln, out)
    torch.cuda.synchronize()
    ref = oracle.adjoint_step(f, lam, tau, grav)
    assert rel_err(out.cpu().numpy().reshape(f.shape), ref) < 1e-12


def test_loss_and_init_adjoint_match_oracle(env):
    torch, lbm = env
    lat = W.Lattice(12, 48, tau=0.8, grav=1e-3, K=3, sigma=1.0, seed=11)
    a = lat.layer_args()
    f0 = oracle.init_layers(lat.Lx, lat.Lz, **a)
    f = oracle.step(f0, lat.tau, lat.grav, 3)
    _, dL = oracle.widths(oracle.row_mean_T(f), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64")
    fd = torch.from_numpy(f.ravel().copy()).cuda()
    lam = torch.empty_like(fd)
    L.loss_adjoint(fd, dL, lam)
    ref = oracle.loss_adjoint(f, dL)
    assert rel_err(lam.cpu().numpy().reshape(f.shape), ref) < 1e-12
    m = lat.modes()
    g_lo, g_hi = L.init_adjoint(lam, lat.T_u, lat.T_m, lat.T_d, lat.z_lo, lat.z_hi, lat.rho_ref, lat.tanh_w,
                                m.amp_lo, m.ph_lo, m.amp_hi, m.ph_hi)
    o_lo, o_hi = oracle.init_adjoint(lat.Lx, lat.Lz, **a, lam0=ref)
    np.testing.assert_allclose(g_lo, o_lo, rtol=1e-10, atol=1e-12 * np.abs(o_lo).max())
    np.testing.assert_allclose(g_hi, o_hi, rtol=1e-10, atol=1e-12 * np.abs(o_hi).max())


def test_adjoint_rejects_non_f64_context(env):
    torch, lbm = env
    L = lbm.Lattice(4, 16, 0.8, 1e-4, prec="f64_ff")
    x = torch.zeros(37 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        L.adjoint_step(x, x.clone(), x.clone())
    assert e.value.code == lbm.LBM_ESTATE

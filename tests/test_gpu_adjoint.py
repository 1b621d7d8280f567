"""GPU parity of the adjoint kernels (native FP64 and float-float) against the oracle's own CPU
adjoint, and the float-float adjoint's scaling, sparse-input and ragged-shape cases."""
import math

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


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
@pytest.mark.parametrize("Lx,Lz,tau,grav", [(8, 16, 0.8, 1e-4), (3, 7, 0.7, 5e-3), (1, 9, 1.1, 1e-3), (5, 140, 0.8, 1e-4)])
def test_adjoint_step_matches_oracle(env, Lx, Lz, tau, grav, prec):
    torch, lbm = env
    f = near_eq(Lx, Lz, 1)
    lam = np.random.default_rng(2).standard_normal(f.shape)
    L = lbm.Lattice(Lx, Lz, tau, grav, prec=prec)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    ft, ln = dev(f), dev(lam)
    out = torch.empty_like(ft)
    L.adjoint_step(ft, ln, out)
    torch.cuda.synchronize()
    ref = oracle.adjoint_step(f, lam, tau, grav)
    assert rel_err(out.cpu().numpy().reshape(f.shape), ref) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_loss_and_init_adjoint_match_oracle(env, prec):
    torch, lbm = env
    lat = W.Lattice(12, 48, tau=0.8, grav=1e-3, K=3, sigma=1.0, seed=11)
    a = lat.layer_args()
    f0 = oracle.init_layers(lat.Lx, lat.Lz, **a)
    f = oracle.step(f0, lat.tau, lat.grav, 3)
    _, dL = oracle.widths(oracle.row_mean_T(f), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
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


@pytest.mark.parametrize("Lx,Lz", [(8, 16), (3, 7), (5, 140)])
def test_fp32_adjoint_matches_oracle(env, Lx, Lz):
    """FP32 contexts: the adjoint step in FP32 storage and arithmetic against the oracle's
    FP64 adjoint of the same (FP32-representable) inputs, to FP32 accuracy."""
    torch, lbm = env
    f = near_eq(Lx, Lz, 1).astype(np.float32)
    lam = np.random.default_rng(2).standard_normal(f.shape).astype(np.float32)
    L = lbm.Lattice(Lx, Lz, 0.8, 1e-4, prec="f32")
    ft = torch.from_numpy(np.ascontiguousarray(f).ravel()).cuda()
    ln = torch.from_numpy(np.ascontiguousarray(lam).ravel()).cuda()
    out = torch.empty_like(ft)
    L.adjoint_step(ft, ln, out)
    torch.cuda.synchronize()
    ref = oracle.adjoint_step(f.astype(np.float64), lam.astype(np.float64), 0.8, 1e-4)
    assert rel_err(out.cpu().numpy().astype(np.float64).reshape(f.shape), ref) < 2e-6


def evolved_state(torch, lbm, steps=60):
    """The 64x128 parity workload after some steps (a state with flow, all wall cases)."""
    lat = W.PARITY_64x128
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64")
    L.init_from(lat)
    L.step(steps)
    f = L.populations_device().clone()
    L.close()
    return lat, f


def adjoint_of(torch, lbm, lat, prec, f, lam):
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    out = torch.empty_like(f)
    L.adjoint_step(f, lam, out)
    torch.cuda.synchronize()
    L.close()
    return out


def test_ff_adjoint_matches_oracle_on_evolved_state(env):
    """64x128 state with flow (2 x 128-row tiles, wall tiles), random lam: the float-float
    adjoint against the oracle element by element, relative to the largest entry."""
    torch, lbm = env
    lat, f = evolved_state(torch, lbm)
    lam = torch.from_numpy(np.random.default_rng(5).standard_normal(f.numel())).cuda()
    got = adjoint_of(torch, lbm, lat, "f64_ff", f, lam).cpu().numpy().reshape(37, lat.Lx, lat.Lz)
    ref = oracle.adjoint_step(f.cpu().numpy().reshape(37, lat.Lx, lat.Lz),
                              lam.cpu().numpy().reshape(37, lat.Lx, lat.Lz), lat.tau, lat.grav)
    assert rel_err(got, ref) < 1e-13


def test_ff_adjoint_is_scale_invariant(env):
    """The per-site block exponent: lam * 2^k gives the result * 2^k bit for bit, from
    2^-900 to 2^900 (all arithmetic after the scaling is the same)."""
    torch, lbm = env
    lat, f = evolved_state(torch, lbm, 20)
    lam = torch.from_numpy(np.random.default_rng(6).standard_normal(f.numel())).cuda()
    base = adjoint_of(torch, lbm, lat, "f64_ff", f, lam)
    for k in (-900, -300, -40, 40, 300, 900):
        got = adjoint_of(torch, lbm, lat, "f64_ff", f, lam * math.ldexp(1.0, k))   # exact scalings
        assert torch.equal(got * math.ldexp(1.0, -k), base), k


def test_ff_adjoint_sparse_and_mixed_magnitude_lambda(env):
    """lam nonzero in a few rows only (as the width loss starts it), with magnitudes from
    1e-30 to 1 mixed inside sites: zero where the oracle is zero, and within 1e-13 of each
    site's scale elsewhere (entries far below a site's largest count as 0 in the collide
    term, an error below 2^-74 of that largest entry)."""
    torch, lbm = env
    lat, f = evolved_state(torch, lbm, 20)
    rng = np.random.default_rng(7)
    lam = np.zeros((37, lat.Lx, lat.Lz))
    rows = [0, 1, 40, 41, 42, 90, lat.Lz - 1]
    lam[:, :, rows] = rng.standard_normal((37, lat.Lx, len(rows))) * 10.0 ** rng.integers(-30, 1, (37, lat.Lx, len(rows)))
    got = adjoint_of(torch, lbm, lat, "f64_ff", f, torch.from_numpy(lam.ravel()).cuda())
    got = got.cpu().numpy().reshape(lam.shape)
    ref = oracle.adjoint_step(f.cpu().numpy().reshape(lam.shape), lam, lat.tau, lat.grav)
    assert np.array_equal(got == 0, ref == 0)
    assert rel_err(got, ref) < 1e-13


@pytest.mark.parametrize("Lx,Lz", [(48, 300), (7, 133), (2, 40)])
def test_ff_adjoint_matches_native_ragged(env, Lx, Lz):
    """Ragged row tails, narrow lattices (x wrap below 3 columns) and several interior
    tiles per column: float-float against the native FP64 adjoint."""
    torch, lbm = env
    lat = W.Lattice(Lx, Lz, tau=0.7, grav=2e-4, K=3, sigma=1.0, seed=9)
    L = lbm.Lattice(Lx, Lz, lat.tau, lat.grav, prec="f64")
    L.init_from(lat)
    L.step(15)
    f = L.populations_device().clone()
    L.close()
    lam = torch.from_numpy(np.random.default_rng(8).standard_normal(f.numel())).cuda()
    a = adjoint_of(torch, lbm, lat, "f64_ff", f, lam)
    b = adjoint_of(torch, lbm, lat, "f64", f, lam)
    assert float((a - b).abs().max() / b.abs().max()) < 1e-13


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_step_and_adjoint_chains_equal_single_calls(env, prec):
    """lbm_step_chain through caller buffers equals lbm_step, and lbm_adjoint_chain equals
    repeated lbm_adjoint_step (bit for bit: the same kernels on the same inputs)."""
    torch, lbm = env
    lat = W.Lattice(24, 70, tau=0.75, grav=2e-4, K=3, sigma=1.0, seed=12)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    f0 = L.populations_device().clone()
    states = [f0] + [torch.empty_like(f0) for _ in range(4)]
    L.step_chain(states)
    for j in range(1, 5):
        L.step(1)
        assert torch.equal(states[j], L.populations_device())
    lam = torch.from_numpy(np.random.default_rng(13).standard_normal(f0.numel())).cuda()
    a, b = lam.clone(), torch.empty_like(lam)
    idx = L.adjoint_chain(states, a, b)
    ref, tmp = lam.clone(), torch.empty_like(lam)
    for j in range(4, -1, -1):
        L.adjoint_step(states[j], ref, tmp)
        ref, tmp = tmp, ref
    assert idx == 1 and torch.equal((a, b)[idx], ref)
    with pytest.raises(lbm.LBMError):
        L.adjoint_chain([states[0], a], a, b)            # a state aliasing an adjoint buffer
    L.close()


def test_moment_records_give_the_same_adjoint(env):
    """lbm_record_moments steps like lbm_step (bit for bit), and the adjoint from its moment
    records equals the adjoint from the states (the same int64 moments enter the same code)."""
    torch, lbm = env
    lat = W.Lattice(20, 150, tau=0.7, grav=2e-4, K=3, sigma=1.0, seed=14)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    f0 = L.populations_device().clone()
    states = [f0] + [torch.empty_like(f0) for _ in range(4)]
    L.step_chain(states)
    wa, wb = torch.empty_like(f0), torch.empty_like(f0)
    moms = [torch.empty(4 * lat.Lx * lat.Lz, dtype=torch.int64, device=f0.device) for _ in range(5)]
    L.record_moments(f0, wa, wb, moms)
    torch.cuda.synchronize()
    assert torch.equal(wb, states[4])               # after step 3 (odd: work_b)
    lam = torch.from_numpy(np.random.default_rng(15).standard_normal(f0.numel())).cuda()
    a1, b1 = lam.clone(), torch.empty_like(lam)
    i1 = L.adjoint_chain(states, a1, b1)
    a2, b2 = lam.clone(), torch.empty_like(lam)
    i2 = L.adjoint_chain_moments(moms, a2, b2)
    assert i1 == i2 and torch.equal((a1, b1)[i1], (a2, b2)[i2])
    L.close()
    F = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64")
    with pytest.raises(lbm.LBMError) as e:
        F.record_moments(f0, wa, wb, moms)
    assert e.value.code == lbm.LBM_ESTATE

"""Gradient of the two fronts' mixing widths with respect to the interface-mode amplitudes:
the checkpointed GPU adjoint against the oracle's adjoint chain (tiny lattice) and against
centred finite differences of the GPU forward (relative 1e-4, step 1e-6)."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    from paper_1405_1253_b300 import adjoint
    return adjoint


@pytest.mark.parametrize("prec,store", [("f64", "states"), ("f64_ff", "states"), ("f64_ff", "moments"),
                                        ("f64_ff", "tape")])
def test_gradient_matches_oracle_chain(adj, prec, store):
    lat = W.Lattice(12, 48, tau=0.8, grav=1e-3, K=2, sigma=1.0, seed=21)
    nsteps, ckpt = 6, 3
    drv = adj.WidthGradient(lat, nsteps, ckpt, prec=prec, store=store)
    m = lat.modes()
    Lval = drv.forward(m.amp_lo, m.amp_hi)
    g_lo, g_hi = drv.backward()
    drv.close()
    a = lat.layer_args()
    states = [oracle.init_layers(lat.Lx, lat.Lz, **a)]
    for _ in range(nsteps):
        states.append(oracle.step(states[-1], lat.tau, lat.grav))
    Lo, dL = oracle.widths(oracle.row_mean_T(states[-1]), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    assert abs(Lval - Lo.sum()) < 1e-10 * abs(Lo.sum())
    lam = oracle.loss_adjoint(states[-1], dL)
    for t in range(nsteps - 1, -1, -1):
        lam = oracle.adjoint_step(states[t], lam, lat.tau, lat.grav)
    o_lo, o_hi = oracle.init_adjoint(lat.Lx, lat.Lz, **a, lam0=lam)
    np.testing.assert_allclose(g_lo, o_lo, rtol=1e-9, atol=1e-12 * np.abs(o_lo).max())
    np.testing.assert_allclose(g_hi, o_hi, rtol=1e-9, atol=1e-12 * np.abs(o_hi).max())


def fd_gradient(drv, lat, h, ks):
    m = lat.modes()
    fd_lo, fd_hi = np.zeros(lat.K), np.zeros(lat.K)
    for k in ks:
        e = np.zeros(lat.K)
        e[k] = h
        fd_lo[k] = (drv.forward(m.amp_lo + e, m.amp_hi) - drv.forward(m.amp_lo - e, m.amp_hi)) / (2 * h)
        fd_hi[k] = (drv.forward(m.amp_lo, m.amp_hi + e) - drv.forward(m.amp_lo, m.amp_hi - e)) / (2 * h)
    return fd_lo, fd_hi


def fd_check(adj, lat, nsteps, ckpt, tol=1e-4):
    """Adjoint gradient (through torch.autograd) against centred differences:
    normwise relative error < tol with step 1e-6, and componentwise relative error < tol
    with step 1e-4 (at 1e-6 the forward's ~1e-12 rounding noise in L becomes ~1e-6 in each
    difference quotient, which only the normwise measure averages out)."""
    import torch
    drv = adj.WidthGradient(lat, nsteps, ckpt)
    m = lat.modes()
    amp_lo = torch.tensor(m.amp_lo, requires_grad=True)
    amp_hi = torch.tensor(m.amp_hi, requires_grad=True)
    loss = adj.width_loss(amp_lo, amp_hi, drv)
    loss.backward()
    g = np.concatenate([amp_lo.grad.numpy(), amp_hi.grad.numpy()])
    fd6 = np.concatenate(fd_gradient(drv, lat, 1e-6, range(lat.K)))
    assert np.linalg.norm(g - fd6) / np.linalg.norm(fd6) < tol
    fd4 = np.concatenate(fd_gradient(drv, lat, 1e-4, range(lat.K)))
    scale = np.maximum(np.abs(fd4), 1e-3 * np.abs(fd4).max())
    assert np.max(np.abs(g - fd4) / scale) < tol
    drv.close()
    return g


def test_gradient_vs_finite_differences_small(adj):
    lat = W.Lattice(64, 192, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=22)
    fd_check(adj, lat, nsteps=200, ckpt=20)


def test_gradient_vs_finite_differences_256x512_2000_steps(adj):
    """The differentiation workload: 256x512, 2000 steps, checkpoint every 100, 16 modes
    per front, centred differences on every amplitude."""
    lat = W.GRADIENT_256x512
    fd_check(adj, lat, nsteps=W.GRADIENT_STEPS, ckpt=W.GRADIENT_CKPT)


def test_moment_store_gives_the_same_gradient(adj):
    """The three backward stores of the float-float driver (segment states, recomputed moment
    records with and without the recompute overlapped on a second stream, moment records taped
    in the forward) give the same loss and the same amplitude and phase gradients bit for bit;
    the tape recomputes no step."""
    lat = W.Lattice(40, 96, tau=0.8, grav=1e-4, K=3, sigma=1.0, seed=25)
    m = lat.modes()
    out = []
    for store, pipe in (("states", False), ("moments", False), ("moments", True), ("tape", False)):
        drv = adj.WidthGradient(lat, 60, 20, store=store, pipeline=pipe)
        assert drv.pipeline == pipe
        val = drv.forward(m.amp_lo, m.amp_hi)
        g = np.concatenate(drv.backward())
        out.append((val, g, np.concatenate(drv.grad_phases)))
        if store == "tape":
            assert drv.stats.recompute_steps == 0 and drv.stats.adjoint_steps == 60
            assert drv.stats.checkpoint_bytes == 0
        if store == "moments":
            # the forward records its last segments itself, one per record set (one without
            # the overlap, four by default with it); the backward recomputes only the others
            assert drv.n_taped == min(len(drv.moms_sets), 3) == (3 if pipe else 1)
            assert drv.stats.recompute_steps == 20 * (3 - drv.n_taped)
        drv.close()
    for val, g, gp in out[1:]:
        assert val == out[0][0]
        np.testing.assert_array_equal(g, out[0][1])
        np.testing.assert_array_equal(gp, out[0][2])


@pytest.mark.parametrize("nsteps,ckpt", [(40, 20), (20, 20), (30, 10)])
def test_moment_store_segment_counts(adj, nsteps, ckpt):
    """With one, two or three segments the moment store (the forward recording the moments of
    the segments the backward reads first, one per record set) gives the state store's
    gradient bit for bit, with and without the overlap and with more record sets."""
    lat = W.Lattice(24, 72, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=27)
    m = lat.modes()
    out = []
    for store, pipe, nset in (("states", False, None), ("moments", False, None), ("moments", True, None),
                              ("moments", True, 3), ("moments", False, 2)):
        drv = adj.WidthGradient(lat, nsteps, ckpt, store=store, pipeline=pipe, record_sets=nset)
        val = drv.forward(m.amp_lo, m.amp_hi)
        out.append((val, np.concatenate(drv.backward())))
        drv.close()
    for val, g in out[1:]:
        assert val == out[0][0]
        np.testing.assert_array_equal(g, out[0][1])


def test_record_sets_need_two_with_the_overlap(adj):
    lat = W.Lattice(8, 24, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=26)
    with pytest.raises(ValueError):
        adj.WidthGradient(lat, 4, 2, store="moments", pipeline=True, record_sets=1)
    with pytest.raises(ValueError):
        adj.WidthGradient(lat, 4, 2, store="moments", pipeline=False, record_sets=0)


def test_tape_store_refuses_other_precisions_and_walls(adj):
    lat = W.Lattice(8, 24, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=26)
    for kw in ({"prec": "f64"}, {"prec": "f32"}, {"walls": (1.02, 0.98)}):
        with pytest.raises(ValueError):
            adj.WidthGradient(lat, 4, 2, store="tape", **kw)


def test_phase_gradient_matches_oracle_chain_and_finite_differences(adj):
    """dL/dphi from the driver (init adjoint with phases) against the oracle's chain, and
    against centred differences of the GPU forward in each phase."""
    lat = W.Lattice(12, 48, tau=0.8, grav=1e-3, K=2, sigma=1.0, seed=21)
    nsteps, ckpt = 6, 3
    drv = adj.WidthGradient(lat, nsteps, ckpt)
    m = lat.modes()
    drv.forward(m.amp_lo, m.amp_hi)
    drv.backward()
    p_lo, p_hi = drv.grad_phases
    a = lat.layer_args()
    states = [oracle.init_layers(lat.Lx, lat.Lz, **a)]
    for _ in range(nsteps):
        states.append(oracle.step(states[-1], lat.tau, lat.grav))
    _, dL = oracle.widths(oracle.row_mean_T(states[-1]), lat.T_u, lat.T_m, lat.T_d, with_grad=True)
    lam = oracle.loss_adjoint(states[-1], dL)
    for t in range(nsteps - 1, -1, -1):
        lam = oracle.adjoint_step(states[t], lam, lat.tau, lat.grav)
    o_lo, o_hi = oracle.init_adjoint_phases(lat.Lx, lat.Lz, **a, lam0=lam)
    np.testing.assert_allclose(p_lo, o_lo, rtol=1e-9, atol=1e-12 * np.abs(o_lo).max())
    np.testing.assert_allclose(p_hi, o_hi, rtol=1e-9, atol=1e-12 * np.abs(o_hi).max())
    h = 1e-6
    for k in range(lat.K):
        e = np.zeros(lat.K)
        e[k] = h
        fd_lo = (drv.forward(m.amp_lo, m.amp_hi, m.ph_lo + e, m.ph_hi)
                 - drv.forward(m.amp_lo, m.amp_hi, m.ph_lo - e, m.ph_hi)) / (2 * h)
        fd_hi = (drv.forward(m.amp_lo, m.amp_hi, m.ph_lo, m.ph_hi + e)
                 - drv.forward(m.amp_lo, m.amp_hi, m.ph_lo, m.ph_hi - e)) / (2 * h)
        assert abs(fd_lo - p_lo[k]) < 1e-4 * max(1.0, abs(fd_lo))
        assert abs(fd_hi - p_hi[k]) < 1e-4 * max(1.0, abs(fd_hi))
    drv.close()


def test_fp32_gradient_tracks_fp64_gradient(adj):
    """The gradient of an FP32-storage run (FP32 forward, FP32 adjoint) against the
    float-float gradient of the same problem: the same to FP32-level accuracy."""
    lat = W.Lattice(64, 192, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=22)
    m = lat.modes()
    g = {}
    for prec in ("f32", "f64_ff"):
        drv = adj.WidthGradient(lat, 200, 20, prec=prec)
        drv.forward(m.amp_lo, m.amp_hi)
        g[prec] = np.concatenate(drv.backward())
        drv.close()
    assert np.linalg.norm(g["f32"] - g["f64_ff"]) / np.linalg.norm(g["f64_ff"]) < 1e-3

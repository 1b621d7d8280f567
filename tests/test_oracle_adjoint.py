"""Pins of the oracle adjoint: finite differences of the oracle forward step and the
dot-product identity <lam, J v> = <J^T lam, v>."""
import numpy as np
import pytest

import oracle

TU, TM, TD = 0.95, 1.0, 1.05


def near_eq_state(Lx, Lz, seed):
    rng = np.random.default_rng(seed)
    f = np.empty((37, Lx, Lz))
    for x in range(Lx):
        for z in range(Lz):
            f[:, x, z] = oracle.equilibrium(1 + 0.02 * rng.standard_normal(), 0.02 * rng.standard_normal(),
                                            0.02 * rng.standard_normal(), 1 + 0.03 * rng.standard_normal())
    return f * (1 + 2e-3 * rng.standard_normal(f.shape))


@pytest.mark.parametrize("Lx,Lz,tau,grav", [(3, 8, 0.8, 1e-4), (4, 7, 0.7, 5e-3)])
def test_adjoint_step_dot_product(Lx, Lz, tau, grav):
    rng = np.random.default_rng(1)
    f = near_eq_state(Lx, Lz, 2)
    lam = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape)
    h = 1e-6
    Jv = (oracle.step(f + h * v, tau, grav) - oracle.step(f - h * v, tau, grav)) / (2 * h)
    lhs = np.sum(lam * Jv)
    rhs = np.sum(oracle.adjoint_step(f, lam, tau, grav) * v)
    assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs))


def test_adjoint_step_columns_by_finite_differences():
    Lx, Lz, tau, grav = 2, 7, 0.8, 1e-3
    f = near_eq_state(Lx, Lz, 4)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal(f.shape)
    adj = oracle.adjoint_step(f, lam, tau, grav)
    h = 1e-6
    for flat in rng.choice(f.size, 25, replace=False):
        e = np.zeros(f.size); e[flat] = h
        e = e.reshape(f.shape)
        fd = np.sum(lam * (oracle.step(f + e, tau, grav) - oracle.step(f - e, tau, grav))) / (2 * h)
        assert abs(fd - adj.ravel()[flat]) < 1e-7 * max(1.0, abs(fd))


def test_loss_and_init_adjoint_chain_matches_finite_differences():
    """d(L_u + L_d)/dA for a short run on a small lattice: adjoint chain vs centred FD."""
    Lx, Lz, grav, tau, nsteps, K = 12, 48, 1e-3, 0.8, 6, 2
    rng = np.random.default_rng(5)
    a_lo, a_hi = rng.normal(0, 1, K), rng.normal(0, 1, K)
    p_lo, p_hi = rng.uniform(0, 2 * np.pi, K), rng.uniform(0, 2 * np.pi, K)
    args = (Lx, Lz, grav, TU, TM, TD, Lz / 3, 2 * Lz / 3, 1.0, 3.0)

    def loss(al, ah):
        f = oracle.init_layers(*args, al, p_lo, ah, p_hi)
        f = oracle.step(f, tau, grav, nsteps)
        return oracle.widths(oracle.row_mean_T(f), TU, TM, TD).sum()

    f0 = oracle.init_layers(*args, a_lo, p_lo, a_hi, p_hi)
    states = [f0]
    for _ in range(nsteps):
        states.append(oracle.step(states[-1], tau, grav))
    _, dL = oracle.widths(oracle.row_mean_T(states[-1]), TU, TM, TD, with_grad=True)
    lam = oracle.loss_adjoint(states[-1], dL)
    for t in range(nsteps - 1, -1, -1):
        lam = oracle.adjoint_step(states[t], lam, tau, grav)
    g_lo, g_hi = oracle.init_adjoint(*args, a_lo, p_lo, a_hi, p_hi, lam)
    h = 1e-6
    for k in range(K):
        e = np.zeros(K); e[k] = h
        fd_lo = (loss(a_lo + e, a_hi) - loss(a_lo - e, a_hi)) / (2 * h)
        fd_hi = (loss(a_lo, a_hi + e) - loss(a_lo, a_hi - e)) / (2 * h)
        assert abs(fd_lo - g_lo[k]) < 1e-5 * max(1.0, abs(fd_lo)), (k, fd_lo, g_lo[k])
        assert abs(fd_hi - g_hi[k]) < 1e-5 * max(1.0, abs(fd_hi)), (k, fd_hi, g_hi[k])


WALLS = (1.04, 0.97)


@pytest.mark.parametrize("Lx,Lz,tau,grav", [(3, 8, 0.8, 1e-4), (5, 7, 0.7, 5e-3)])
def test_thermal_adjoint_step_dot_product(Lx, Lz, tau, grav):
    """The adjoint step with thermal walls against a directional finite difference of the
    oracle's thermal-wall step."""
    rng = np.random.default_rng(11)
    f = near_eq_state(Lx, Lz, 12)
    lam = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape)
    h = 1e-6
    Jv = (oracle.step(f + h * v, tau, grav, walls=WALLS) - oracle.step(f - h * v, tau, grav, walls=WALLS)) / (2 * h)
    lhs = np.sum(lam * Jv)
    rhs = np.sum(oracle.adjoint_step(f, lam, tau, grav, walls=WALLS) * v)
    assert abs(lhs - rhs) < 1e-7 * max(1.0, abs(lhs))


def test_thermal_adjoint_columns_by_finite_differences():
    """Columns of the thermal adjoint, including populations that leave through a wall (which
    only the ghost densities take up) and wall-row destinations, by finite differences."""
    Lx, Lz, tau, grav = 4, 8, 0.8, 1e-3
    f = near_eq_state(Lx, Lz, 13)
    rng = np.random.default_rng(14)
    lam = rng.standard_normal(f.shape)
    adj = oracle.adjoint_step(f, lam, tau, grav, walls=WALLS)
    h = 1e-6
    c, _ = oracle.velocities()
    leaving = [np.ravel_multi_index((l, x, z), f.shape) for l in range(37) for x in range(Lx) for z in (0, 1, 2)
               if z + c[l, 1] < 0]
    picks = list(rng.choice(leaving, 10, replace=False)) + list(rng.choice(f.size, 20, replace=False))
    for flat in picks:
        e = np.zeros(f.size); e[flat] = h
        e = e.reshape(f.shape)
        fd = np.sum(lam * (oracle.step(f + e, tau, grav, walls=WALLS) - oracle.step(f - e, tau, grav, walls=WALLS))) / (2 * h)
        assert abs(fd - adj.ravel()[flat]) < 1e-7 * max(1.0, abs(fd))


def test_thermal_propagate_transpose_is_exact():
    """With tau -> infinity and no gravity the collide is the identity, so the adjoint is the
    transpose of propagate + thermal bc, a linear map: <P v, w> = <v, P^T w> to rounding."""
    Lx, Lz = 5, 9
    rng = np.random.default_rng(15)
    f = near_eq_state(Lx, Lz, 16)
    v, w = rng.standard_normal(f.shape), rng.standard_normal(f.shape)
    Pv = oracle.bc_thermal(v, oracle.propagate(v), *WALLS)
    PTw = oracle.adjoint_step(f, w, 1e15, 0.0, walls=WALLS)
    lhs, rhs = np.sum(Pv * w), np.sum(v * PTw)
    assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(Pv * w))


def test_phase_gradient_chain_matches_finite_differences():
    """d(L_u + L_d)/dphi for a short run: the adjoint chain (init_adjoint_phases) against
    centred finite differences in each phase of both fronts."""
    Lx, Lz, grav, tau, nsteps, K = 12, 48, 1e-3, 0.8, 6, 2
    rng = np.random.default_rng(6)
    a_lo, a_hi = rng.normal(0, 1, K), rng.normal(0, 1, K)
    p_lo, p_hi = rng.uniform(0, 2 * np.pi, K), rng.uniform(0, 2 * np.pi, K)
    args = (Lx, Lz, grav, TU, TM, TD, Lz / 3, 2 * Lz / 3, 1.0, 3.0)

    def loss(pl, ph):
        f = oracle.step(oracle.init_layers(*args, a_lo, pl, a_hi, ph), tau, grav, nsteps)
        return oracle.widths(oracle.row_mean_T(f), TU, TM, TD).sum()

    states = [oracle.init_layers(*args, a_lo, p_lo, a_hi, p_hi)]
    for _ in range(nsteps):
        states.append(oracle.step(states[-1], tau, grav))
    _, dL = oracle.widths(oracle.row_mean_T(states[-1]), TU, TM, TD, with_grad=True)
    lam = oracle.loss_adjoint(states[-1], dL)
    for t in range(nsteps - 1, -1, -1):
        lam = oracle.adjoint_step(states[t], lam, tau, grav)
    g_lo, g_hi = oracle.init_adjoint_phases(*args, a_lo, p_lo, a_hi, p_hi, lam)
    h = 1e-6
    for k in range(K):
        e = np.zeros(K); e[k] = h
        fd_lo = (loss(p_lo + e, p_hi) - loss(p_lo - e, p_hi)) / (2 * h)
        fd_hi = (loss(p_lo, p_hi + e) - loss(p_lo, p_hi - e)) / (2 * h)
        assert abs(fd_lo - g_lo[k]) < 1e-5 * max(1.0, abs(fd_lo)), (k, fd_lo, g_lo[k])
        assert abs(fd_hi - g_hi[k]) < 1e-5 * max(1.0, abs(fd_hi)), (k, fd_hi, g_hi[k])

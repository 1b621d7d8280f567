"""Physics regressions of the GPU step (Sec. III.A), in every precision:
* the exact budget of the collide: it conserves mass, adds exactly -g rho / r to the z
  momentum sum of the lattice vectors (rho u gains rho g_vec) and raises the energy by exactly
  rho (u . g_vec + g^2 / 2) per site, u the pre-collision velocity (the force-shifted
  equilibrium keeps T); propagation with the wall rule conserves mass and energy;
* an unperturbed isothermal layer stays at rest (renormalised velocity small, no growth)."""
import numpy as np
import pytest

import oracle
from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu

# tolerance of the budgets, relative to the size of the summed quantity: FP64-accurate steps
# carry ~1e-14 per population; FP32 storage rounds every population to 2^-24
TOL = {"f64": 1e-12, "f64_ff": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    return lbm


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
def test_one_step_budget(lbm, prec):
    lat = W.Lattice(32, 96, tau=0.8, grav=2e-4, K=4, sigma=1.5, seed=17)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    L.step(40)                                   # a state with flow
    f0 = L.populations()
    L.step(1)
    f1 = L.populations()
    c, _ = oracle.velocities()                   # [37, 2] integer lattice vectors
    _, r = oracle.weights()                      # lattice constant, xi = r c
    g = oracle.bc(f0, oracle.propagate(f0))      # pre-collision populations
    rho, ux, uz, T = oracle.moments(g, lat.grav)
    xi2 = (r * r) * (c ** 2).sum(axis=1)
    # the budgets hold for the collide, between the pre-collision state g = P f0 and the
    # stored post-collision f1; propagation conserves mass and energy but not momentum (the
    # walls reverse populations)
    mass0, mass1 = g.sum(), f1.sum()
    jz0 = np.tensordot(c[:, 1].astype(float), g, axes=1).sum()
    jz1 = np.tensordot(c[:, 1].astype(float), f1, axes=1).sum()
    e0 = 0.5 * np.tensordot(xi2, g, axes=1).sum()
    e1 = 0.5 * np.tensordot(xi2, f1, axes=1).sum()
    assert abs(g.sum() - f0.sum()) < 1e-13 * f0.sum()
    assert abs(0.5 * np.tensordot(xi2, f0, axes=1).sum() - e0) < 1e-13 * e0
    tol = TOL[prec]
    assert abs(mass1 - mass0) < tol * mass0
    # z momentum of the lattice vectors: rho u_z = r sum c_z f gains -g rho per site
    djz = -lat.grav * rho.sum() / r
    assert abs((jz1 - jz0) - djz) < tol * np.abs(np.tensordot(np.abs(c[:, 1]).astype(float), f0, axes=1)).sum()
    # energy: + rho (u . g_vec + g^2/2) = rho (-g u_z + g^2/2) per site
    de = (rho * (-lat.grav * uz + 0.5 * lat.grav ** 2)).sum()
    assert abs((e1 - e0) - de) < tol * e0


@pytest.mark.parametrize("prec", ["f64", "f64_ff", "f32"])
def test_isothermal_layer_stays_at_rest(lbm, prec):
    lat = W.Lattice(4, 64, tau=0.8, grav=1e-4, K=0, sigma=0.0, seed=0, T_u=1.0, T_m=1.0, T_d=1.0)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    inner = slice(6, lat.Lz - 6)
    peaks = []
    for _ in range(6):
        L.step(250)
        _, ux, uz, T = L.moments(renormalised=True)
        assert np.abs(ux).max() < 1e-10
        assert np.abs(uz[:, inner]).max() < 1e-6
        assert np.abs(uz).max() < 1e-5
        assert np.abs(T - 1).max() < 5e-5
        peaks.append(np.abs(uz).max())
    assert max(peaks[3:]) < 1.2 * max(peaks[:3])

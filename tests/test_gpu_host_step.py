"""Streamed host-buffer stepping (lbm_step_host): every output equals set_populations +
one step + get_populations of its input, bit for bit, also when the copies of consecutive
steps overlap; FP32 storage and NULL buffers are rejected."""
import numpy as np
import pytest

from paper_1405_1253_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1405_1253_b300 import lbm
    return lbm


@pytest.mark.parametrize("prec", ["f64", "f64_ff"])
def test_step_host_matches_sequential(lbm, prec):
    import torch
    lat = W.Lattice(32, 96, tau=0.8, grav=1e-4, K=4, sigma=1.0, seed=13)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    rng = np.random.default_rng(3)
    base = L.populations()
    n = 5
    ins = [torch.from_numpy(base * (1 + 1e-3 * rng.standard_normal(base.shape))).reshape(-1).pin_memory()
           for _ in range(n)]
    outs = [torch.empty_like(a).pin_memory() for a in ins]
    L.step_host(ins, outs)
    last = outs[-1].numpy().reshape(base.shape).copy()
    assert np.array_equal(L.populations(), last)      # the device holds the last output
    for a, b in zip(ins, outs):
        L.set_populations(a.numpy().reshape(base.shape))
        L.step(1)
        assert np.array_equal(L.populations(), b.numpy().reshape(base.shape))


def test_step_host_pageable_buffers(lbm):
    lat = W.Lattice(16, 48, tau=0.8, grav=1e-4, K=2, sigma=1.0, seed=14)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec="f64_ff")
    L.init_from(lat)
    f0 = L.populations().reshape(-1).copy()
    out = np.empty_like(f0)
    L.step_host([f0, f0], [out, out])
    L.set_populations(f0.reshape(37, lat.Lx, lat.Lz))
    L.step(1)
    assert np.array_equal(L.populations().reshape(-1), out)


def test_step_host_rejects_fp32(lbm):
    L = lbm.Lattice(16, 48, 0.8, 1e-4, prec="f32")
    a = np.zeros(37 * 16 * 48)
    with pytest.raises(lbm.LBMError):
        L.step_host([a], [a])

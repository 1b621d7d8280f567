"""Thin ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA library ``csrc/liblbm.so``; PyTorch only
provides device memory and the stream.  Importing this module loads the library and
raises ImportError when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the same library (the bounds-checked one in tests)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_HERE, "csrc", "liblbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1405_1253_b300.build` "
                      "(or __graft_entry__.build()); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

Q = 37
LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENOMEM, LBM_ETIMEOUT, LBM_ENUMERIC, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
PREC = {"f64": 0, "f32": 1, "f32_dev": 2, "f64_ff": 3}   # lbm_prec of include/lbm.h
POP_BYTES = {"f64": 8, "f64_ff": 8, "f32": 4, "f32_dev": 4}

_vp, _dp, _ip, _i, _d, _sz = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                              ctypes.c_int, ctypes.c_double, ctypes.c_size_t)


class LayersDesc(ctypes.Structure):
    _fields_ = [("T_u", _d), ("T_m", _d), ("T_d", _d), ("z_lo", _d), ("z_hi", _d), ("rho_ref", _d),
                ("tanh_w", _d), ("n_modes", _i), ("amp_lo", _dp), ("phase_lo", _dp), ("amp_hi", _dp),
                ("phase_hi", _dp)]


_SIGS = {
    "lbm_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _d, _d, _vp, _vp, _sz, _vp]),
    "lbm_destroy": (_i, [_vp]),
    "lbm_init_layers": (_i, [_vp, ctypes.POINTER(LayersDesc)]),
    "lbm_step": (_i, [_vp, _i]),
    "lbm_step_push": (_i, [_vp, _i]),
    "lbm_set_walls": (_i, [_vp, _i, _d, _d]),
    "lbm_step_chain": (_i, [_vp, _vp, _i]),
    "lbm_adjoint_chain": (_i, [_vp, _vp, _i, _vp, _vp, ctypes.POINTER(_i)]),
    "lbm_record_moments": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "lbm_adjoint_chain_moments": (_i, [_vp, _vp, _i, _vp, _vp, ctypes.POINTER(_i)]),
    "lbm_step_host": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i]),
    "lbm_propagate": (_i, [_vp]),
    "lbm_current": (_vp, [_vp]),
    "lbm_get_populations": (_i, [_vp, _vp, _i]),
    "lbm_set_populations": (_i, [_vp, _vp, _i]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i]),
    "lbm_row_mean_T": (_i, [_vp, _vp, _i]),
    "lbm_widths": (_i, [_vp, _d, _d, _d, _dp, _dp]),
    "lbm_tent_widths": (_i, [_vp, _d, _d, _d, _dp]),
    "lbm_row_stats": (_i, [_vp, _dp, _dp, _dp, _dp, _i]),
    "lbm_global_sums": (_i, [_vp, _dp]),
    "lbm_adjoint_step": (_i, [_vp, _vp, _vp, _vp]),
    "lbm_loss_adjoint": (_i, [_vp, _vp, _dp, _vp]),
    "lbm_init_adjoint": (_i, [_vp, ctypes.POINTER(LayersDesc), _vp, _dp, _dp]),
    "lbm_init_adjoint_full": (_i, [_vp, ctypes.POINTER(LayersDesc), _vp, _dp, _dp, _dp, _dp]),
    "lbm_sync": (_i, [_vp]),
    "lbm_lattice": (_i, [_ip, _dp, _dp]),
    "lbm_row_mean_T_noalloc": (_i, [_vp, _i, _i, _vp, _vp]),
    "lbm_ensemble_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "lbm_ensemble_destroy": (_i, [_vp]),
    "lbm_ensemble_config": (_i, [_vp, _i, _i, _i]),
    "lbm_ensemble_tune": (_i, [_vp, _i, _dp, _ip, _ip, _ip]),
    "lbm_ensemble_step": (_i, [_vp, _i]),
    "lbm_ensemble_capture": (_i, [_vp, _i]),
    "lbm_ensemble_graph_launch": (_i, [_vp]),
    "lbm_ensemble_sync": (_i, [_vp]),
    "lbm_ensemble_set_wait": (_i, [_vp, ctypes.c_longlong, ctypes.c_uint]),
    "lbm_slabs_create": (_i, [ctypes.POINTER(_vp), _vp, _i]),
    "lbm_slabs_destroy": (_i, [_vp]),
    "lbm_slabs_scatter": (_i, [_vp]),
    "lbm_slabs_step": (_i, [_vp, _i, _i]),
    "lbm_slabs_gather": (_i, [_vp]),
    "lbm_test_fail_alloc": (_i, [_i]),
    "lbm_test_packed_ff": (_i, [_i, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ulonglong)]),
    "lbm_test_oob_count": (_i, [ctypes.POINTER(ctypes.c_uint)]),
    "lbm_probe_fp64_rate": (_i, [_i, ctypes.POINTER(ctypes.c_double)]),
    "lbm_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def test_fail_alloc(n: int):
    """Refuse the n-th next device allocation of the library (n < 0: cancel); for tests of
    the error paths."""
    _lib.lbm_test_fail_alloc(int(n))


def test_packed_ff(n: int, seed: int) -> int:
    """Result words in which a packed float-float operation differs from its scalar form, over
    n seeded operand pairs (lbm_test_packed_ff)."""
    out = ctypes.c_ulonglong(0)
    _check(_lib.lbm_test_packed_ff(int(n), ctypes.c_ulonglong(seed), ctypes.byref(out)))
    return out.value


def probe_fp64_rate(iters: int = 2048) -> float:
    """FP64 FMAs per second of the current device's FP64 pipe (lbm_probe_fp64_rate)."""
    out = ctypes.c_double(0.0)
    _check(_lib.lbm_probe_fp64_rate(int(iters), ctypes.byref(out)))
    return out.value


def test_oob_count() -> int:
    """Out-of-range population indices met since the last call (bounds-checked builds
    only; raises LBMError otherwise)."""
    v = ctypes.c_uint()
    _check(_lib.lbm_test_oob_count(ctypes.byref(v)))
    return v.value


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _check(rc: int):
    if rc != LBM_OK:
        raise LBMError(rc, _lib.lbm_last_error().decode())


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def exported_symbols():
    return list(_SIGS)


def lattice():
    """(c[37,2], w[37], r) from the library's own quadrature (host only)."""
    c = np.zeros(2 * Q, dtype=np.int32)
    w = np.zeros(Q)
    r = np.zeros(1)
    _check(_lib.lbm_lattice(c.ctypes.data_as(_ip), _dptr(w), _dptr(r)))
    return c.reshape(Q, 2), w, float(r[0])


def row_mean_T_noalloc(f_dev_ptr: int, Lx: int, Lz: int, Tbar_dev_ptr: int, stream_ptr: int = 0):
    """Allocation-free horizontal mean of T of an FP64 population array (device pointers)."""
    _check(_lib.lbm_row_mean_T_noalloc(f_dev_ptr, int(Lx), int(Lz), Tbar_dev_ptr, stream_ptr or None))


def layers_desc(T_u, T_m, T_d, z_lo, z_hi, rho_ref, tanh_w, amp_lo, ph_lo, amp_hi, ph_hi):
    """Build an lbm_layers_desc; returns (desc, keepalive arrays)."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (amp_lo, ph_lo, amp_hi, ph_hi)]
    K = len(arrs[0])
    assert all(len(a) == K for a in arrs)
    d = LayersDesc(float(T_u), float(T_m), float(T_d), float(z_lo), float(z_hi), float(rho_ref),
                   float(tanh_w), K, *[_dptr(a) if K else None for a in arrs])
    return d, arrs


class Lattice:
    """One lattice on one GPU: two torch-owned population buffers and a library context."""

    def __init__(self, Lx: int, Lz: int, tau: float, grav: float, prec: str = "f64",
                 device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.Lx, self.Lz, self.tau, self.grav, self.prec = int(Lx), int(Lz), float(tau), float(grav), prec
        self.device = torch.device("cuda", device)
        n = Q * self.Lx * self.Lz
        dt = torch.float64 if POP_BYTES[prec] == 8 else torch.float32
        self.bufs = [torch.empty(n, dtype=dt, device=self.device) for _ in range(2)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = _vp()
        nbytes = n * POP_BYTES[prec]
        _check(_lib.lbm_create(ctypes.byref(ctx), self.Lx, self.Lz, PREC[prec], self.tau, self.grav,
                               self.bufs[0].data_ptr(), self.bufs[1].data_ptr(), nbytes,
                               self.stream.cuda_stream))
        self.ctx = ctx

    # -- lifecycle ---------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            _lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- method --------------------------------------------------------------------
    def init_layers(self, T_u, T_m, T_d, z_lo, z_hi, rho_ref, tanh_w, amp_lo, ph_lo, amp_hi, ph_hi):
        d, keep = layers_desc(T_u, T_m, T_d, z_lo, z_hi, rho_ref, tanh_w, amp_lo, ph_lo, amp_hi, ph_hi)
        _check(_lib.lbm_init_layers(self.ctx, ctypes.byref(d)))

    def init_from(self, lat):
        """Initial state of a workloads.Lattice description."""
        m = lat.modes()
        self.init_layers(lat.T_u, lat.T_m, lat.T_d, lat.z_lo, lat.z_hi, lat.rho_ref, lat.tanh_w,
                         m.amp_lo, m.ph_lo, m.amp_hi, m.ph_hi)

    def step(self, n: int = 1):
        _check(_lib.lbm_step(self.ctx, int(n)))

    def step_host(self, host_in, host_out):
        """One step per (input, output) pair of host buffers (pinned torch tensors or
        contiguous float64 numpy arrays of 37*Lx*Lz elements): copy in, step, copy out,
        the copies of consecutive steps overlapped (lbm_step_host)."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        n = len(host_in)
        if len(host_out) != n:
            raise ValueError("host_in and host_out differ in length")
        ins = (_vp * n)(*[ptr(a) for a in host_in])
        outs = (_vp * n)(*[ptr(a) for a in host_out])
        _check(_lib.lbm_step_host(self.ctx, ins, outs, n))

    def set_walls(self, thermal: bool, T_bottom: float = 1.0, T_top: float = 1.0):
        """Wall rule of step(): half-way bounce-back (thermal=False, the default) or
        isothermal walls at T_bottom / T_top (see lbm_set_walls)."""
        _check(_lib.lbm_set_walls(self.ctx, int(bool(thermal)), float(T_bottom), float(T_top)))

    def step_push(self, n: int = 1):
        """Push-form steps of a post-propagation state (see lbm_step_push)."""
        _check(_lib.lbm_step_push(self.ctx, int(n)))

    def propagate(self):
        """One propagate + bc without collide (pull-form state -> push-form state)."""
        _check(_lib.lbm_propagate(self.ctx))

    def sync(self):
        _check(_lib.lbm_sync(self.ctx))

    def current(self):
        """The torch buffer holding the current state (storage precision, flat)."""
        ptr = _lib.lbm_current(self.ctx)
        return self.bufs[0] if ptr == self.bufs[0].data_ptr() else self.bufs[1]

    def populations(self) -> np.ndarray:
        out = np.empty((Q, self.Lx, self.Lz))
        _check(_lib.lbm_get_populations(self.ctx, out.ctypes.data, 0))
        return out

    def populations_device(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty(Q * self.Lx * self.Lz, dtype=torch.float64, device=self.device)
        _check(_lib.lbm_get_populations(self.ctx, out.data_ptr(), 1))
        return out

    def set_populations(self, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            assert f.size == Q * self.Lx * self.Lz
            _check(_lib.lbm_set_populations(self.ctx, f.ctypes.data, 0))
        else:
            assert f.dtype == self.torch.float64 and f.is_contiguous() and f.numel() == Q * self.Lx * self.Lz
            _check(_lib.lbm_set_populations(self.ctx, f.data_ptr(), 1))

    def moments(self, renormalised: bool = False):
        outs = [np.empty((self.Lx, self.Lz)) for _ in range(4)]
        _check(_lib.lbm_moments(self.ctx, *[o.ctypes.data for o in outs], int(bool(renormalised)), 0))
        return tuple(outs)

    def row_mean_T(self) -> np.ndarray:
        out = np.empty(self.Lz)
        _check(_lib.lbm_row_mean_T(self.ctx, out.ctypes.data, 0))
        return out

    def widths(self, T_u, T_m, T_d, with_grad: bool = False):
        out = np.zeros(2)
        dL = np.zeros(self.Lz) if with_grad else None
        _check(_lib.lbm_widths(self.ctx, float(T_u), float(T_m), float(T_d), _dptr(out),
                               _dptr(dL) if with_grad else None))
        return (out, dL) if with_grad else out

    def tent_widths(self, T_u, T_m, T_d) -> np.ndarray:
        """(L_u, L_d) by the tent-map integral of Eq. (3L), in sites."""
        out = np.zeros(2)
        _check(_lib.lbm_tent_widths(self.ctx, float(T_u), float(T_m), float(T_d), _dptr(out)))
        return out

    def row_stats(self) -> dict:
        """Per-row mean and rms fluctuation over x of T and of E_k = |u^H|^2 / 2."""
        outs = {k: np.empty(self.Lz) for k in ("T_mean", "T_rms", "Ek_mean", "Ek_rms")}
        _check(_lib.lbm_row_stats(self.ctx, *[_dptr(outs[k]) for k in ("T_mean", "T_rms", "Ek_mean", "Ek_rms")], 0))
        return outs

    def global_sums(self) -> np.ndarray:
        out = np.zeros(2)
        _check(_lib.lbm_global_sums(self.ctx, _dptr(out)))
        return out

    # -- adjoint (FP64 contexts) -------------------------------------------------------
    def step_chain(self, states):
        """states[j + 1] = step(states[j]) through the given device tensors (lbm_step_chain)."""
        ptrs = (_vp * len(states))(*[t.data_ptr() for t in states])
        _check(_lib.lbm_step_chain(self.ctx, ptrs, len(states)))

    def adjoint_chain(self, states, lam_a, lam_b) -> int:
        """len(states) adjoint steps from lam_a (lam_n) back to lam_0; returns 0 or 1, the
        index of the tensor (lam_a, lam_b) that holds lam_0 (lbm_adjoint_chain)."""
        ptrs = (_vp * len(states))(*[t.data_ptr() for t in states])
        idx = _i(0)
        _check(_lib.lbm_adjoint_chain(self.ctx, ptrs, len(states), lam_a.data_ptr(), lam_b.data_ptr(),
                                      ctypes.byref(idx)))
        return idx.value

    def record_moments(self, f0, work_a, work_b, moments):
        """len(moments) steps from f0 through work_a / work_b, recording each step's moments
        (int64 tensors of 4 Lx Lz) for the adjoint (lbm_record_moments)."""
        ptrs = (_vp * len(moments))(*[t.data_ptr() for t in moments])
        _check(_lib.lbm_record_moments(self.ctx, f0.data_ptr(), len(moments), work_a.data_ptr(), work_b.data_ptr(),
                                       ptrs))

    def adjoint_chain_moments(self, moments, lam_a, lam_b) -> int:
        """adjoint_chain with f_t given by its moment records; returns the index of the
        tensor (lam_a, lam_b) holding lam_0 (lbm_adjoint_chain_moments)."""
        ptrs = (_vp * len(moments))(*[t.data_ptr() for t in moments])
        idx = _i(0)
        _check(_lib.lbm_adjoint_chain_moments(self.ctx, ptrs, len(moments), lam_a.data_ptr(), lam_b.data_ptr(),
                                              ctypes.byref(idx)))
        return idx.value

    def adjoint_step(self, f_t, lam_next, lam_out):
        _check(_lib.lbm_adjoint_step(self.ctx, f_t.data_ptr(), lam_next.data_ptr(), lam_out.data_ptr()))

    def loss_adjoint(self, f, dL_dTbar: np.ndarray, lam_out):
        dL = np.ascontiguousarray(dL_dTbar, dtype=np.float64)
        assert dL.size == self.Lz
        _check(_lib.lbm_loss_adjoint(self.ctx, f.data_ptr(), _dptr(dL), lam_out.data_ptr()))

    def init_adjoint(self, lam0, T_u, T_m, T_d, z_lo, z_hi, rho_ref, tanh_w, amp_lo, ph_lo, amp_hi, ph_hi,
                     phases: bool = False):
        """dL/dA of both fronts from lam0 = dL/df_0; with phases=True also dL/dphi
        (returns dA_lo, dA_hi, dphi_lo, dphi_hi)."""
        d, keep = layers_desc(T_u, T_m, T_d, z_lo, z_hi, rho_ref, tanh_w, amp_lo, ph_lo, amp_hi, ph_hi)
        K = d.n_modes
        dlo, dhi = np.zeros(max(K, 1)), np.zeros(max(K, 1))
        if not phases:
            _check(_lib.lbm_init_adjoint(self.ctx, ctypes.byref(d), lam0.data_ptr(), _dptr(dlo), _dptr(dhi)))
            return dlo[:K], dhi[:K]
        plo, phi = np.zeros(max(K, 1)), np.zeros(max(K, 1))
        _check(_lib.lbm_init_adjoint_full(self.ctx, ctypes.byref(d), lam0.data_ptr(), _dptr(dlo), _dptr(dhi),
                                          _dptr(plo), _dptr(phi)))
        return dlo[:K], dhi[:K], plo[:K], phi[:K]


class Ensemble:
    """Independent lattices advanced together (one launch per step, or one persistent
    launch under an optional CUDA graph).  `lattices` are Lattice objects sharing the
    device, precision ("f64_ff" or "f32"), tau, g and stream."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        arr = (_vp * len(self.lattices))(*[L.ctx for L in self.lattices])
        e = _vp()
        _check(_lib.lbm_ensemble_create(ctypes.byref(e), len(self.lattices), arr))
        self.e = e

    def config(self, mode: int = 1, tile_z: int = 128, ctas_per_sm: int = 0):
        _check(_lib.lbm_ensemble_config(self.e, int(mode), int(tile_z), int(ctas_per_sm)))

    def tune(self, steps: int = 5):
        ms = ctypes.c_double()
        mode, tz, ctas = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.lbm_ensemble_tune(self.e, int(steps), ctypes.byref(ms), ctypes.byref(mode),
                                      ctypes.byref(tz), ctypes.byref(ctas)))
        return {"ms_per_step": ms.value, "mode": mode.value, "tile_z": tz.value, "ctas_per_sm": ctas.value}

    def step(self, n: int = 1):
        _check(_lib.lbm_ensemble_step(self.e, int(n)))

    def capture(self, n: int):
        _check(_lib.lbm_ensemble_capture(self.e, int(n)))

    def graph_launch(self):
        _check(_lib.lbm_ensemble_graph_launch(self.e))

    def sync(self):
        _check(_lib.lbm_ensemble_sync(self.e))

    def set_wait(self, spin_limit_cycles: int, extra_wait: int = 0):
        _check(_lib.lbm_ensemble_set_wait(self.e, int(spin_limit_cycles), int(extra_wait)))

    def close(self):
        if getattr(self, "e", None):
            _lib.lbm_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slabs:
    """The lattice of `lattice` split into `n` x-slabs with halo exchange (Sec. III.B),
    emulating the paper's multi-GPU layout on this device."""

    def __init__(self, lattice: Lattice, n: int):
        self.lattice = lattice
        s = _vp()
        _check(_lib.lbm_slabs_create(ctypes.byref(s), lattice.ctx, int(n)))
        self.s = s

    def scatter(self):
        _check(_lib.lbm_slabs_scatter(self.s))

    def step(self, n: int = 1, overlap: bool = True):
        _check(_lib.lbm_slabs_step(self.s, int(n), int(bool(overlap))))

    def gather(self):
        _check(_lib.lbm_slabs_gather(self.s))

    def close(self):
        if getattr(self, "s", None):
            _lib.lbm_slabs_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

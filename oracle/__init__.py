"""Plain FP64 CPU oracle for the D2Q37 thermal lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package, and this package imports
nothing from the product.

The arithmetic lives in ``d2q37_oracle.c`` (plain C, FP64, one function per passage of
the paper); this module compiles it with gcc on first use and exposes numpy wrappers.
Arrays use the paper's structure-of-arrays, column-major layout ``f[l, x, z]``.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  velocity set, quadrature ..... pinned (paper's r ~ 1.1969, Gaussian moments to degree 9)
  equilibrium .................. pinned (Gaussian moments up to order 4, closed form)
  propagate, bc ................ pinned (np.roll interior, bijection, reversibility, rest state);
                                 the wall RULE is a reading: the paper names the rows only
  collide ...................... pinned (mass, momentum + rho g, temperature invariants)
  init_layers, init_columns .... pinned (isothermal hydrostatic slopes, pressure continuity;
                                 the column form equals the listed columns of the full one)
  moments ...................... pinned (round trip through the pinned equilibrium)
  row_mean_T ................... pinned (closed-form tanh profile of the initial state, its
                                 column average with modes, equilibria of chosen fields)
  widths ....................... pinned (closed form on a tanh profile)
  adjoint_step, loss/init adjoint  pinned (finite differences, dot-product identity)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d2q37_oracle.c")
_LIB = os.path.join(_HERE, "_d2q37_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 37


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP over x columns)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "oracle_setup": (i, []),
                "oracle_velocities": (i, [ip, ip]),
                "oracle_weights": (i, [dp, dp]),
                "oracle_equilibrium": (None, [d, d, d, d, dp]),
                "oracle_site_moments": (None, [dp, dp]),
                "oracle_propagate": (None, [i, i, dp, dp]),
                "oracle_bc": (None, [i, i, dp, dp]),
                "oracle_bc_thermal": (None, [i, i, dp, dp, d, d]),
                "oracle_step_thermal": (None, [i, i, d, d, i, dp, dp, d, d]),
                "oracle_collide": (None, [i, i, d, d, dp, dp]),
                "oracle_step": (None, [i, i, d, d, i, dp, dp]),
                "oracle_init_layers": (None, [i, i, d, d, d, d, d, d, d, d, i, dp, dp, dp, dp, dp]),
                "oracle_init_columns": (None, [i, i, d, d, d, d, d, d, d, d, i, dp, dp, dp, dp,
                                               i, ip, dp]),
                "oracle_moments": (None, [i, i, d, dp, dp, dp, dp, dp, i]),
                "oracle_row_mean_T": (None, [i, i, dp, dp]),
                "oracle_widths": (i, [i, dp, d, d, d, dp, dp]),
                "oracle_tent_widths": (None, [i, dp, d, d, d, dp]),
                "oracle_adjoint_step": (None, [i, i, d, d, dp, dp, dp]),
                "oracle_adjoint_step_thermal": (None, [i, i, d, d, dp, dp, dp, d, d]),
                "oracle_loss_adjoint": (None, [i, i, dp, dp, dp]),
                "oracle_init_adjoint": (None, [i, i, d, d, d, d, d, d, d, d, i,
                                               dp, dp, dp, dp, dp, dp, dp]),
                "oracle_init_adjoint_phases": (None, [i, i, d, d, d, d, d, d, d, d, i,
                                                      dp, dp, dp, dp, dp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            rc = lib.oracle_setup()
            if rc != 0:
                raise RuntimeError(f"oracle_setup failed ({rc})")
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def velocities():
    """(c[37,2] int, opp[37] int) in canonical order."""
    lib = _load()
    c = np.zeros(2 * Q, dtype=np.int32)
    opp = np.zeros(Q, dtype=np.int32)
    lib.oracle_velocities(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c.reshape(Q, 2).astype(np.int64), opp.astype(np.int64)


def weights():
    """(w[37], r) from the oracle's own quadrature solve."""
    lib = _load()
    w = np.zeros(Q)
    r = np.zeros(1)
    lib.oracle_weights(_p(w), _p(r))
    return w, float(r[0])


def equilibrium(rho, ux, uz, T) -> np.ndarray:
    lib = _load()
    out = np.zeros(Q)
    lib.oracle_equilibrium(float(rho), float(ux), float(uz), float(T), _p(out))
    return out


def site_moments(fs) -> np.ndarray:
    """(rho, ux, uz, T) of one site's 37 populations."""
    lib = _load()
    fs = _f64(fs)
    out = np.zeros(4)
    lib.oracle_site_moments(_p(fs), _p(out))
    return out


def propagate(f: np.ndarray, fill=np.nan) -> np.ndarray:
    lib = _load()
    f = _f64(f)
    _, Lx, Lz = f.shape
    g = np.full_like(f, fill)
    lib.oracle_propagate(Lx, Lz, _p(f), _p(g))
    return g


def bc(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    lib = _load()
    f = _f64(f)
    g = _f64(g).copy()
    _, Lx, Lz = f.shape
    lib.oracle_bc(Lx, Lz, _p(f), _p(g))
    return g


def bc_thermal(f: np.ndarray, g: np.ndarray, T_bot: float, T_top: float) -> np.ndarray:
    """Thermal-wall variant of bc: ghost rows at rest at T_bot / T_top, mass-balanced."""
    lib = _load()
    f = _f64(f)
    g = _f64(g).copy()
    _, Lx, Lz = f.shape
    lib.oracle_bc_thermal(Lx, Lz, _p(f), _p(g), float(T_bot), float(T_top))
    return g


def collide(g: np.ndarray, tau: float, grav: float) -> np.ndarray:
    lib = _load()
    g = _f64(g)
    _, Lx, Lz = g.shape
    out = np.empty_like(g)
    lib.oracle_collide(Lx, Lz, float(tau), float(grav), _p(g), _p(out))
    return out


def step(f: np.ndarray, tau: float, grav: float, nsteps: int = 1, walls=None) -> np.ndarray:
    """nsteps full steps; walls=None: bounce-back walls, walls=(T_bot, T_top): thermal walls."""
    lib = _load()
    f = _f64(f).copy()
    _, Lx, Lz = f.shape
    work = np.empty_like(f)
    if walls is None:
        lib.oracle_step(Lx, Lz, float(tau), float(grav), int(nsteps), _p(f), _p(work))
    else:
        lib.oracle_step_thermal(Lx, Lz, float(tau), float(grav), int(nsteps), _p(f), _p(work),
                                float(walls[0]), float(walls[1]))
    return f


def init_layers(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt,
                amp_lo, ph_lo, amp_hi, ph_hi) -> np.ndarray:
    lib = _load()
    amp_lo, ph_lo, amp_hi, ph_hi = map(_f64, (amp_lo, ph_lo, amp_hi, ph_hi))
    K = len(amp_lo)
    assert len(ph_lo) == K and len(amp_hi) == K and len(ph_hi) == K
    f = np.empty((Q, Lx, Lz))
    lib.oracle_init_layers(int(Lx), int(Lz), float(grav), float(Tu), float(Tm), float(Td),
                           float(zlo0), float(zhi0), float(rho_ref), float(wt), K,
                           _p(amp_lo), _p(ph_lo), _p(amp_hi), _p(ph_hi), _p(f))
    return f


def init_columns(Lx, Lz, cols, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt,
                 amp_lo, ph_lo, amp_hi, ph_hi) -> np.ndarray:
    """Columns `cols` of the Lx x Lz initial state, as a [37, len(cols), Lz] array."""
    lib = _load()
    amp_lo, ph_lo, amp_hi, ph_hi = map(_f64, (amp_lo, ph_lo, amp_hi, ph_hi))
    K = len(amp_lo)
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int32) % int(Lx))
    f = np.empty((Q, len(cols), Lz))
    lib.oracle_init_columns(int(Lx), int(Lz), float(grav), float(Tu), float(Tm), float(Td),
                            float(zlo0), float(zhi0), float(rho_ref), float(wt), K,
                            _p(amp_lo), _p(ph_lo), _p(amp_hi), _p(ph_hi), len(cols),
                            cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(f))
    return f


def moments(f: np.ndarray, grav: float, renormalised: bool = False):
    """rho, ux, uz, T as [Lx, Lz] arrays."""
    lib = _load()
    f = _f64(f)
    _, Lx, Lz = f.shape
    out = [np.empty((Lx, Lz)) for _ in range(4)]
    lib.oracle_moments(Lx, Lz, float(grav), _p(f), *[_p(o) for o in out], int(bool(renormalised)))
    return tuple(out)


def row_mean_T(f: np.ndarray) -> np.ndarray:
    lib = _load()
    f = _f64(f)
    _, Lx, Lz = f.shape
    out = np.empty(Lz)
    lib.oracle_row_mean_T(Lx, Lz, _p(f), _p(out))
    return out


def widths(Tbar, Tu, Tm, Td, with_grad: bool = False):
    """(L_u, L_d) threshold widths; with_grad also returns d(L_u+L_d)/dTbar."""
    lib = _load()
    Tbar = _f64(Tbar)
    out = np.zeros(2)
    dL = np.zeros(len(Tbar))
    rc = lib.oracle_widths(len(Tbar), _p(Tbar), float(Tu), float(Tm), float(Td), _p(out), _p(dL))
    if rc != 0:
        raise ValueError("mixing-width crossing not found")
    return (out, dL) if with_grad else out


def tent_widths(Tbar, Tu, Tm, Td) -> np.ndarray:
    lib = _load()
    Tbar = _f64(Tbar)
    out = np.zeros(2)
    lib.oracle_tent_widths(len(Tbar), _p(Tbar), float(Tu), float(Tm), float(Td), _p(out))
    return out


def adjoint_step(f_t: np.ndarray, lam_next: np.ndarray, tau: float, grav: float, walls=None) -> np.ndarray:
    """lam_t = P^T J_C^T lam_next at state f_t; walls=(T_bot, T_top) for the thermal walls."""
    lib = _load()
    f_t, lam_next = _f64(f_t), _f64(lam_next)
    _, Lx, Lz = f_t.shape
    out = np.empty_like(f_t)
    if walls is None:
        lib.oracle_adjoint_step(Lx, Lz, float(tau), float(grav), _p(f_t), _p(lam_next), _p(out))
    else:
        lib.oracle_adjoint_step_thermal(Lx, Lz, float(tau), float(grav), _p(f_t), _p(lam_next), _p(out),
                                        float(walls[0]), float(walls[1]))
    return out


def loss_adjoint(f: np.ndarray, dL_dTbar) -> np.ndarray:
    lib = _load()
    f, dL_dTbar = _f64(f), _f64(dL_dTbar)
    _, Lx, Lz = f.shape
    out = np.empty_like(f)
    lib.oracle_loss_adjoint(Lx, Lz, _p(f), _p(dL_dTbar), _p(out))
    return out


def init_adjoint_phases(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt,
                        amp_lo, ph_lo, amp_hi, ph_hi, lam0):
    """dL/dphi of the lower and upper interface modes, given lam0 = dL/df_0."""
    lib = _load()
    amp_lo, ph_lo, amp_hi, ph_hi, lam0 = map(_f64, (amp_lo, ph_lo, amp_hi, ph_hi, lam0))
    K = len(amp_lo)
    dlo, dhi = np.zeros(K), np.zeros(K)
    lib.oracle_init_adjoint_phases(int(Lx), int(Lz), float(grav), float(Tu), float(Tm), float(Td),
                                   float(zlo0), float(zhi0), float(rho_ref), float(wt), K,
                                   _p(amp_lo), _p(ph_lo), _p(amp_hi), _p(ph_hi), _p(lam0),
                                   _p(dlo), _p(dhi))
    return dlo, dhi


def init_adjoint(Lx, Lz, grav, Tu, Tm, Td, zlo0, zhi0, rho_ref, wt,
                 amp_lo, ph_lo, amp_hi, ph_hi, lam0):
    lib = _load()
    amp_lo, ph_lo, amp_hi, ph_hi, lam0 = map(_f64, (amp_lo, ph_lo, amp_hi, ph_hi, lam0))
    K = len(amp_lo)
    dlo, dhi = np.zeros(K), np.zeros(K)
    lib.oracle_init_adjoint(int(Lx), int(Lz), float(grav), float(Tu), float(Tm), float(Td),
                            float(zlo0), float(zhi0), float(rho_ref), float(wt), K,
                            _p(amp_lo), _p(ph_lo), _p(amp_hi), _p(ph_hi), _p(lam0),
                            _p(dlo), _p(dhi))
    return dlo, dhi

"""Seeded synthetic workloads for the three-layer Rayleigh-Taylor runs.

This module holds no lattice Boltzmann arithmetic: it only names the run
configurations (sizes, relaxation time, gravity, layer temperatures, mode counts)
and draws the random interface modes.  Both the CUDA path and the oracle receive
the drawn arrays as plain inputs, so neither depends on the random generator.

Recipe (the paper's "white noise" interface perturbations, Sec. V, with the layer
set-up of Sec. I and Table II scaled to single-GPU sizes):
  T_d = 1.05 (bottom), T_m = 1.00, T_u = 0.95 (top); equal layer heights
  (interfaces at Lz/3 and 2Lz/3); rho_ref = 1 at the bottom wall; tanh half-width
  3 sites.  Modes k = 1..K per front: rng = numpy.random.default_rng(seed); for the
  lower front first, then the upper: phases U[0, 2 pi), then amplitudes N(0, sigma^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

T_D, T_M, T_U = 1.05, 1.00, 0.95
RHO_REF = 1.0
TANH_W = 3.0


@dataclass(frozen=True)
class Modes:
    amp_lo: np.ndarray
    ph_lo: np.ndarray
    amp_hi: np.ndarray
    ph_hi: np.ndarray

    @property
    def K(self) -> int:
        return len(self.amp_lo)


def draw_modes(seed: int, K: int, sigma: float) -> Modes:
    rng = np.random.default_rng(seed)
    ph_lo = rng.uniform(0.0, 2.0 * np.pi, K)
    amp_lo = rng.normal(0.0, sigma, K)
    ph_hi = rng.uniform(0.0, 2.0 * np.pi, K)
    amp_hi = rng.normal(0.0, sigma, K)
    return Modes(amp_lo, ph_lo, amp_hi, ph_hi)


@dataclass(frozen=True)
class Lattice:
    """One three-layer lattice: shape, physics parameters and its seeded modes."""
    Lx: int
    Lz: int
    tau: float
    grav: float
    K: int
    sigma: float
    seed: int
    T_u: float = T_U
    T_m: float = T_M
    T_d: float = T_D
    rho_ref: float = RHO_REF
    tanh_w: float = TANH_W
    z_lo_rows: float | None = None   # unperturbed interface heights in sites (default Lz/3, 2 Lz/3)
    z_hi_rows: float | None = None

    @property
    def z_lo(self) -> float:
        return self.Lz / 3.0 if self.z_lo_rows is None else self.z_lo_rows

    @property
    def z_hi(self) -> float:
        return 2.0 * self.Lz / 3.0 if self.z_hi_rows is None else self.z_hi_rows

    @property
    def sites(self) -> int:
        return self.Lx * self.Lz

    def modes(self) -> Modes:
        return draw_modes(self.seed, self.K, self.sigma)

    def layer_args(self):
        """Positional arguments shared by the oracle and the CUDA init."""
        m = self.modes()
        return dict(grav=self.grav, Tu=self.T_u, Tm=self.T_m, Td=self.T_d,
                    zlo0=self.z_lo, zhi0=self.z_hi, rho_ref=self.rho_ref, wt=self.tanh_w,
                    amp_lo=m.amp_lo, ph_lo=m.ph_lo, amp_hi=m.amp_hi, ph_hi=m.ph_hi)


# The five run configurations (lattice units).
PARITY_64x128 = Lattice(64, 128, tau=0.8, grav=1e-4, K=8, sigma=1.0, seed=1)
PARITY_STEPS = 100
THROUGHPUT_1024x2048 = Lattice(1024, 2048, tau=0.7, grav=5e-5, K=64, sigma=0.5, seed=2)
THROUGHPUT_STEPS = 5000
PRECISION_4096x8192 = Lattice(4096, 8192, tau=0.7, grav=5e-5, K=128, sigma=0.5, seed=3)
PRECISION_STEPS = 2000
GRADIENT_256x512 = Lattice(256, 512, tau=0.8, grav=1e-4, K=16, sigma=1.0, seed=5)
GRADIENT_STEPS = 2000
GRADIENT_CKPT = 100
ENSEMBLE_STEPS = 3000


def fronts(case: str, seed: int, Lx: int = 384, Lz: int = 1024, tau: float = 0.6) -> Lattice:
    """Table II's two cases scaled to Lx x Lz (aspect ~ 2400:6144), Atwood number 0.025:
    T_u = 0.975, T_d = 1.025; "double": a middle layer at T_m = 1 of depth Lz/12 centred at
    Lz/2; "single": T_u above Lz/2, T_d below (T_m = T_u, no second jump).  Gravity keeps the
    adiabatic length 2 (T_d - T_u) / g at ~1.085 Lz as in Table II; white-noise interfaces of
    K = Lx/2 modes with an rms displacement of one site."""
    K = Lx // 2
    g = 2.0 * 0.05 / (1.085 * Lz)
    sigma = float(np.sqrt(2.0 / K))
    if case == "double":
        d = Lz / 12.0
        return Lattice(Lx, Lz, tau=tau, grav=g, K=K, sigma=sigma, seed=seed, T_u=0.975, T_m=1.0, T_d=1.025,
                       z_lo_rows=Lz / 2.0 - d / 2.0, z_hi_rows=Lz / 2.0 + d / 2.0)
    if case == "single":
        return Lattice(Lx, Lz, tau=tau, grav=g, K=K, sigma=sigma, seed=seed, T_u=0.975, T_m=0.975, T_d=1.025,
                       z_lo_rows=Lz / 2.0, z_hi_rows=float(Lz))
    raise ValueError(case)


def ensemble_48() -> list[Lattice]:
    """16 x 256x512, 16 x 512x1024, 16 x 384x1536, seeds 100..147."""
    shapes = [(256, 512)] * 16 + [(512, 1024)] * 16 + [(384, 1536)] * 16
    return [Lattice(lx, lz, tau=0.8, grav=1e-4, K=16, sigma=1.0, seed=100 + i)
            for i, (lx, lz) in enumerate(shapes)]

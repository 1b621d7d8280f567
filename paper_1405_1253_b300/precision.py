"""FP32-storage step (or, --low f32_dev, FP32 storage of the deviation from the per-row
reference) against the FP64-accurate step on the same seeded initial state.

  python -m paper_1405_1253_b300.precision [--Lx 4096 --Lz 8192 --steps 2000] [--low f32_dev]

Prints one JSON line: relative L2 errors of rho and T, relative errors of both fronts'
mixing widths, the maximum over sites of |T32 - T64|, and the time of each run (CUDA
events around the stepping only) with the speedup.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import workloads as W


def run(lat, steps, prec, lbm, torch):
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
    L.init_from(lat)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    L.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    rho, _, _, T = L.moments()
    widths = L.widths(lat.T_u, lat.T_m, lat.T_d)
    mass = L.global_sums()[0]
    L.close()
    return rho, T, widths, ms, mass


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--Lx", type=int, default=W.PRECISION_4096x8192.Lx)
    ap.add_argument("--Lz", type=int, default=W.PRECISION_4096x8192.Lz)
    ap.add_argument("--steps", type=int, default=W.PRECISION_STEPS)
    ap.add_argument("--low", default="f32", choices=["f32", "f32_dev"])
    args = ap.parse_args()
    import torch
    from . import lbm
    base = W.PRECISION_4096x8192
    lat = W.Lattice(args.Lx, args.Lz, tau=base.tau, grav=base.grav, K=base.K, sigma=base.sigma, seed=base.seed)
    r64, T64, w64, ms64, m64 = run(lat, args.steps, "f64_ff", lbm, torch)
    r32, T32, w32, ms32, m32 = run(lat, args.steps, args.low, lbm, torch)
    out = {
        "lattice": [lat.Lx, lat.Lz], "steps": args.steps, "tau": lat.tau, "grav": lat.grav, "modes": lat.K,
        "low": args.low,
        "rho_rel_l2": float(np.linalg.norm(r32 - r64) / np.linalg.norm(r64)),
        "T_rel_l2": float(np.linalg.norm(T32 - T64) / np.linalg.norm(T64)),
        "T_max_abs": float(np.abs(T32 - T64).max()),
        "widths_f64": [float(v) for v in w64], "widths_low": [float(v) for v in w32],
        "width_rel_err": [float(abs(a - b) / abs(b)) for a, b in zip(w32, w64)],
        "mass_rel_drift_low": float(abs(m32 - m64) / m64),
        "ms_f64": ms64, "ms_low": ms32, "speedup": ms64 / ms32,
        "mlups_f64": lat.sites * args.steps / (ms64 * 1e-3) / 1e6,
        "mlups_low": lat.sites * args.steps / (ms32 * 1e-3) / 1e6,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()

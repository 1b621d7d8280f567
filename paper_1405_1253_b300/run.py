"""Command-line runner: initialise a three-layer lattice and advance it; optionally apply
the adjoint step to a seeded random field at the final state (in the storage precision).

  python -m paper_1405_1253_b300.run --prec f64_ff --Lx 1024 --Lz 2048 --steps 3
  python -m paper_1405_1253_b300.run --prec f64_ff --steps 1 --adjoint 3 [--store moments]
  python -m paper_1405_1253_b300.run --prec f64_ff --steps 3 --walls      (thermal walls)
  python -m paper_1405_1253_b300.run --prec f64_ff --steps 3 --push       (push form)
  python -m paper_1405_1253_b300.run --prec f64_ff --steps 20 --ensemble 16 --ens-mode 1
      (the first 16 lattices of the 48-lattice ensemble: --steps steps in one launch per step
       (--ens-mode 0) or one persistent launch (1), tile height 128)

Used as the profiled program of the ncu summaries under profiles/.
"""
from __future__ import annotations

import argparse
import json

from . import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", default="f64_ff", choices=["f64", "f64_ff", "f32", "f32_dev"])
    ap.add_argument("--Lx", type=int, default=1024)
    ap.add_argument("--Lz", type=int, default=2048)
    ap.add_argument("--tau", type=float, default=0.7)
    ap.add_argument("--grav", type=float, default=5e-5)
    ap.add_argument("--modes", type=int, default=64)
    ap.add_argument("--sigma", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--adjoint", type=int, default=0, help="adjoint steps after the forward steps")
    ap.add_argument("--store", default="states", choices=["states", "moments"],
                    help="the adjoint reads the state (gathers f_t) or a moment record of the step")
    ap.add_argument("--walls", action="store_true", help="thermal walls at the bottom and top layer temperatures")
    ap.add_argument("--push", action="store_true",
                    help="push form: one propagate into the push convention, then --steps push steps")
    ap.add_argument("--ensemble", type=int, default=0, help="run the first N lattices of the 48-lattice ensemble")
    ap.add_argument("--ens-mode", type=int, default=1, choices=[0, 1],
                    help="0: one launch per step, 1: one persistent launch")
    args = ap.parse_args()
    from . import lbm
    if args.ensemble > 0:
        lats = W.ensemble_48()[:args.ensemble]
        Ls = []
        for d in lats:
            Ls.append(lbm.Lattice(d.Lx, d.Lz, d.tau, d.grav, prec=args.prec))
            Ls[-1].init_from(d)
        ens = lbm.Ensemble(Ls)
        ens.config(mode=args.ens_mode, tile_z=128)
        ens.step(args.steps)
        ens.sync()
        mass = sum(L.global_sums()[0] for L in Ls)
        print(json.dumps({"prec": args.prec, "ensemble": len(Ls), "sites": sum(d.sites for d in lats),
                          "mode": args.ens_mode, "steps": args.steps, "mass": mass}))
        return
    lat = W.Lattice(args.Lx, args.Lz, tau=args.tau, grav=args.grav, K=args.modes, sigma=args.sigma, seed=args.seed)
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=args.prec)
    L.init_from(lat)
    if args.walls:
        L.set_walls(True, lat.T_d, lat.T_u)
    if args.push:
        L.propagate()
        L.step_push(args.steps)
    else:
        L.step(args.steps)
    L.sync()
    mass, energy = L.global_sums()
    out = {"prec": args.prec, "Lx": lat.Lx, "Lz": lat.Lz, "steps": args.steps, "walls": args.walls,
           "push": args.push, "mass": mass, "energy": energy}
    if args.adjoint > 0:
        import torch
        f = L.current().clone()                   # the state in the storage precision
        gen = torch.Generator(device=f.device).manual_seed(args.seed)
        lam = [torch.rand(f.numel(), dtype=f.dtype, device=f.device, generator=gen), torch.empty_like(f)]
        if args.store == "moments":
            mom = [torch.empty(4 * lat.Lx * lat.Lz, dtype=torch.int64, device=f.device)]
            L.record_moments(f, torch.empty_like(f), torch.empty_like(f), mom)
        for i in range(args.adjoint):
            if args.store == "moments":
                L.adjoint_chain_moments(mom, lam[i & 1], lam[(i + 1) & 1])
            else:
                L.adjoint_step(f, lam[i & 1], lam[(i + 1) & 1])
        L.sync()
        out.update(adjoint_steps=args.adjoint, lam_sum=float(lam[args.adjoint & 1].sum()))
    print(json.dumps(out))
    L.close()


if __name__ == "__main__":
    main()

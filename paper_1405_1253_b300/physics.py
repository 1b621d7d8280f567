"""Mixing of the double-front (three-layer) and single-front Rayleigh-Taylor runs (Sec. IV).

Both cases of Table II, scaled to one GPU (workloads.fronts), are advanced together as one
ensemble of N_conf realisations each.  At fixed intervals the driver records, per lattice:
  * the tent-map widths L_u, L_d of Eq. (3L) (for the single front with the virtual
    middle temperature T_m = (T_u + T_d)/2) and L_tot = L_u + L_d;
  * for the double front, the fill-in of the gap between the two fronts: the minimum of the
    rms temperature fluctuation over the rows between the unperturbed interfaces, divided
    by its maximum over all rows (near 0 while the middle layer separates the fronts, of
    order 1 once they are in contact; "contact" is taken as the first time it exceeds 1/2);
and at a few times the rms fluctuation profiles of T and of the kinetic energy.  From the
ensemble mean of L_tot it forms the growth-rate estimate alpha_tot = Ldot_tot^2 / (4 g At L_tot)
(the self-similar relation Ldot^2 = 4 alpha g At L), with Ldot by centred differences.
Times are in units of tau_RT = sqrt(Lx / (g At)).  Every step and every per-row reduction
runs in the CUDA library; this module orders the calls and averages the small results.

    python -m paper_1405_1253_b300.physics --nconf 7 --t-end 5 --out fronts.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as W


def run(nconf: int = 7, t_end: float = 5.0, per_tau: int = 20, Lx: int = 384, Lz: int = 1024,
        tau: float = 0.6, prec: str = "f64_ff", profile_times=(0, 1, 2, 3, 4, 5), seed0: int = 200):
    import torch
    from . import lbm

    cases = ("double", "single")
    descs = {c: [W.fronts(c, seed0 + i, Lx, Lz, tau) for i in range(nconf)] for c in cases}
    d0 = descs["double"][0]
    g = d0.grav
    T_u, T_d = d0.T_u, d0.T_d
    T_m = 0.5 * (T_u + T_d)                       # real (double) or virtual (single) middle
    At = (T_d - T_u) / (T_d + T_u)
    tau_rt = math.sqrt(Lx / (g * At))
    dt = max(1, int(round(tau_rt / per_tau)))
    nsamp = int(round(t_end * per_tau))
    z0, z1 = int(d0.z_lo), int(math.ceil(d0.z_hi))

    stream = torch.cuda.Stream()
    lats = {c: [] for c in cases}
    with torch.cuda.stream(stream):
        for c in cases:
            for d in descs[c]:
                L = lbm.Lattice(Lx, Lz, tau, g, prec=prec, stream=stream)
                L.init_from(d)
                lats[c].append(L)
    ens = lbm.Ensemble(lats["double"] + lats["single"])
    tuned = ens.tune(3)
    for c in cases:                     # the tuning trials advanced the states: start again
        for L, d in zip(lats[c], descs[c]):
            L.init_from(d)

    series = {c: {"L_u": [], "L_d": []} for c in cases}
    gap = []
    profiles = {c: {} for c in cases}
    want = {int(round(t * per_tau)): t for t in profile_times}
    t0 = time.perf_counter()
    steps_done = 0
    for k in range(nsamp + 1):
        if k:
            ens.step(dt)
            steps_done += dt
        ens.sync()
        for c in cases:
            w = np.array([L.tent_widths(T_u, T_m, T_d) for L in lats[c]])
            series[c]["L_u"].append(w[:, 0].tolist())
            series[c]["L_d"].append(w[:, 1].tolist())
            if k in want or c == "double":
                st = [L.row_stats() for L in lats[c]]
                if c == "double":
                    gap.append([float(s["T_rms"][z0:z1].min() / max(s["T_rms"].max(), 1e-300)) for s in st])
                if k in want:
                    profiles[c][str(want[k])] = {
                        key: np.mean([s[key] for s in st], axis=0).tolist() for key in ("T_mean", "T_rms", "Ek_rms")}
    wall = time.perf_counter() - t0
    ens.close()

    times = (np.arange(nsamp + 1) * dt / tau_rt).tolist()
    out = {"config": {"Lx": Lx, "Lz": Lz, "tau": tau, "g": g, "At": At, "T_u": T_u, "T_m": T_m, "T_d": T_d,
                      "tau_rt_steps": tau_rt, "sample_every_steps": dt, "nconf": nconf, "prec": prec,
                      "ensemble_launch": tuned},
           "t_over_tau": times, "steps": steps_done, "wall_s": wall,
           "mlups": 2 * nconf * Lx * Lz * steps_done / wall / 1e6}
    for c in cases:
        Lu = np.array(series[c]["L_u"]).mean(axis=1)
        Ld = np.array(series[c]["L_d"]).mean(axis=1)
        Lt = Lu + Ld
        Ldot = np.full_like(Lt, np.nan)
        Ldot[1:-1] = (Lt[2:] - Lt[:-2]) / (2 * dt)
        alpha = Ldot ** 2 / (4 * g * At * Lt)
        out[c] = {"L_u": Lu.tolist(), "L_d": Ld.tolist(), "L_tot": Lt.tolist(),
                  "alpha_tot": [None if not np.isfinite(a) else float(a) for a in alpha],
                  "profiles": profiles[c]}
    gp = np.array(gap)                              # [sample][config]
    out["double"]["gap_fill"] = gp.mean(axis=1).tolist()
    touch = [times[int(np.argmax(gp[1:, i] > 0.5)) + 1] if (gp[1:, i] > 0.5).any() else None for i in range(nconf)]
    out["double"]["t_touch_over_tau"] = touch
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--nconf", type=int, default=7)
    ap.add_argument("--t-end", type=float, default=5.0)
    ap.add_argument("--per-tau", type=int, default=20)
    ap.add_argument("--Lx", type=int, default=384)
    ap.add_argument("--Lz", type=int, default=1024)
    ap.add_argument("--tau", type=float, default=0.6)
    ap.add_argument("--prec", default="f64_ff", choices=["f64_ff", "f32"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = run(a.nconf, a.t_end, a.per_tau, a.Lx, a.Lz, a.tau, a.prec)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt)
    # summary: L_tot and alpha_tot of both cases at whole multiples of tau_RT
    t = np.array(res["t_over_tau"])
    for c in ("double", "single"):
        for tt in range(int(a.t_end) + 1):
            i = int(np.argmin(np.abs(t - tt)))
            al = res[c]["alpha_tot"][i]
            print(f"{c:6s} t/tau={t[i]:.2f}  L_u={res[c]['L_u'][i]:8.2f}  L_d={res[c]['L_d'][i]:8.2f}  "
                  f"L_tot={res[c]['L_tot'][i]:8.2f}  alpha_tot={al if al is None else round(al, 4)}")
    print("double: gap fill-in (mean) at t/tau = 0, 1, ...", [round(v, 3) for v in res["double"]["gap_fill"][::a.per_tau]])
    print("double: t_touch/tau per realisation", res["double"]["t_touch_over_tau"])
    print(f"steps {res['steps']}  wall {res['wall_s']:.1f} s  {res['mlups']:.0f} MLUPS incl. diagnostics")


if __name__ == "__main__":
    main()

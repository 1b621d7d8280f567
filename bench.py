#!/usr/bin/env python
"""Benchmark of the D2Q37 thermal lattice Boltzmann step on B300.

One benchmark step = one fused propagate + bc + collide launch (lbm_step(1)) over the
whole 1024 x 2048 three-layer Rayleigh-Taylor lattice (tau = 0.7, g = 5e-5, 64 seeded
interface modes of amplitude std 0.5).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f64_ff|f64|f32] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank advances its own independent replica
(weak scaling; the lattices do not exchange data) and rank 0 reports the aggregate.
--impl reference times the plain FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1405_1253_b300 import workloads as W  # noqa: E402

Q = 37
METRIC = "MLUPS and % HBM roofline, FP64 vs FP32-storage (stated error), adjoint/forward"
REF_BUDGET_S = 120.0        # oracle seconds of one reference-arm run (warmup + timed steps)
SPEC_HBM_GBS = 7700.0       # nominal B300 HBM3e bandwidth (context beside the measured copy peak)
# The paper's own throughput for this step (Table I, FP64, its D2Q37 RT code): context beside
# the B300 numbers, not a target (other hardware, other code).
PAPER_TABLE_I = [{"hardware": "NVIDIA C2050 (Fermi)", "mlups": 22.0, "precision": "f64"},
                 {"hardware": "NVIDIA K20X (Kepler)", "mlups": 124.0, "precision": "f64"},
                 {"hardware": "2x Intel Sandy Bridge", "mlups": 21.7, "precision": "f64"}]
BYTES_PER_POP = {"f64": 8, "f64_ff": 8, "f32": 4, "f32_dev": 4}
ARITH = {"f64": "f64", "f64_ff": "f64+f32x2", "f32": "f32", "f32_dev": "f32"}
KERNEL = {"f64": "k_step_f64", "f64_ff": "k_step_ff", "f32": "k_step_f32", "f32_dev": "k_step_f32dev"}
# FP64-pipe instructions per site update.  The float-float step converts its four integer
# moment sums to binary64 and makes one FMA for T - 1 and one per population; its adjoint adds
# one binary64 add per population but the rest one (ncu's thread-level FP64-pipe instruction
# count per site, sm__thread_inst_executed_pipe_fp64_pred_on, gives the same 42 and 78).  The
# native FP64 step's count is ncu's alone: 174 FMAs, 86 multiplies, 17 adds, 4 conversions.
FP64_INSTR_PER_SITE = {"k_step_ff": 4 + 1 + Q, "k_adjoint_ff": 4 + 1 + Q + (Q - 1),
                       "k_adjoint_ff_moments": 4 + 1 + Q + (Q - 1), "k_step_f64": 281}


def fp64_roof(kernel, sites, ms, rate):
    """The second roof of an FP64-storage kernel: its FP64 instructions per second against the
    FP64 FMA rate measured in this run (lbm_probe_fp64_rate); None where the kernel's count is
    not stated or no rate was measured."""
    n = FP64_INSTR_PER_SITE.get(kernel)
    if n is None or not rate:
        return None
    achieved = n * sites / (ms * 1e-3) / 1e9
    return {"bound": "fp64_pipe", "kernel": kernel, "instr_per_site": n, "achieved": achieved,
            "peak": rate / 1e9, "unit": "G FP64 instr/s", "frac": achieved / (rate / 1e9),
            "peak_source": "measured in this run: independent FP64 FMA chains on every SM (lbm_probe_fp64_rate)"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "fallback"


# The sources that define each step kernel (its counters stay valid while these are unchanged).
KERNEL_SOURCES = {
    "k_step_ff": ("lattice.cuh", "common.cuh", "ff.cuh", "moments_fix.cuh", "step_ff.cuh"),
    "k_step_f64": ("lattice.cuh", "common.cuh", "ff.cuh", "moments_fix.cuh", "step_f64.cuh"),
    "k_step_f32": ("lattice.cuh", "common.cuh", "step_f32.cuh"),
    "k_step_f32dev": ("lattice.cuh", "common.cuh", "init_diag.cuh", "step_f32dev.cuh"),
    "k_adjoint_ff": ("lattice.cuh", "common.cuh", "ff.cuh", "moments_fix.cuh", "step_ff.cuh", "adjoint_ff.cuh"),
    "k_adjoint_ff_moments": ("lattice.cuh", "common.cuh", "ff.cuh", "moments_fix.cuh", "step_ff.cuh", "adjoint_ff.cuh"),
}


def code_of(text: str) -> str:
    """C++ source without comments and with whitespace runs collapsed (string literals in the
    kernel headers hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash(kernel: str) -> str:
    """Hash of the code (not the comments) of the sources that define a kernel."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1405_1253_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(code_of(open(os.path.join(d, f)).read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, sites: int):
    """Per-launch DRAM bytes from profiles/, if taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path) or kernel not in KERNEL_SOURCES:
        return None
    want = kernel_hash(kernel)
    for line in open(path):
        m = re.match(r"TRAFFIC kernel=(\S+) src=(\S+) bytes_per_site=([0-9.eE+-]+)", line.strip())
        if m and m.group(1) == kernel and m.group(2) == want:
            return float(m.group(3)) * sites
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s: float = 3.0):
        """Block until the sampler has produced its first line (nvidia-smi takes a few hundred
        ms to start), so that the timed region that follows is covered from its start."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.02)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_ranks(ms_total: float, steps: int, sites_per_rank: int, world_size: int, device=None):
    """Whole-job figures from one rank's timed region: the slowest rank's time (max over
    ranks, a collective when world_size > 1) and the aggregate MLUPS of all ranks'
    independent lattices.  Returns (ms_total_max, ms_per_step, mlups)."""
    if world_size > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / steps
    return ms_total, ms_step, world_size * sites_per_rank / (ms_step * 1e-3) / 1e6


def repeats_for(est_region_ms: float, window_s: float, world_size: int, lo: int = 3, hi: int = 2000,
                device="cuda") -> int:
    """Number of repeats of a timed region of about est_region_ms for window_s seconds of
    coverage (at least lo, at most hi); with several ranks the largest estimate wins, so that
    every rank runs the same number."""
    r = int(np.ceil(window_s * 1e3 / max(est_region_ms, 1e-3)))
    r = max(lo, min(hi, r))
    if world_size > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([r], dtype=torch.int64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        r = int(t.item())
    return r


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cores_used() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    if os.environ.get("OMP_NUM_THREADS"):
        n = min(n, int(os.environ["OMP_NUM_THREADS"]))
    return n


def time_oracle(lat, ncols: int, nsteps: int):
    """Oracle MLUPS on an ncols-column window of the lattice (periodic in the window)."""
    import oracle
    a = lat.layer_args()
    f = oracle.init_layers(lat.Lx, lat.Lz, **a)
    win = np.ascontiguousarray(f[:, :ncols, :])
    t0 = time.perf_counter()
    oracle.step(win, lat.tau, lat.grav, nsteps)
    dt = time.perf_counter() - t0
    return ncols * lat.Lz * nsteps / dt / 1e6, dt


def run_reference(args):
    """The oracle as the reference arm: every step one oracle step of a column window of the
    workload (periodic in the window), the window width chosen from a probe so that the whole
    run of warmup + steps takes about REF_BUDGET_S seconds of oracle work."""
    import oracle
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    lat = W.THROUGHPUT_1024x2048
    f = oracle.init_layers(lat.Lx, lat.Lz, **lat.layer_args())
    probe = np.ascontiguousarray(f[:, :16, :])
    t0 = time.perf_counter()
    oracle.step(probe, lat.tau, lat.grav, 1)
    per_col_s = (time.perf_counter() - t0) / 16
    nstep = max(1, args.steps + args.warmup)
    ncols = int(REF_BUDGET_S / (nstep * per_col_s)) // 16 * 16
    ncols = max(16, min(256, ncols))
    win = np.ascontiguousarray(f[:, :ncols, :])
    del f
    for _ in range(args.warmup):
        win = oracle.step(win, lat.tau, lat.grav, 1)
    tot = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        win = oracle.step(win, lat.tau, lat.grav, 1)
        tot += time.perf_counter() - t0
    mlups = ncols * lat.Lz * args.steps / tot / 1e6
    sample = (f"{ncols}x{lat.Lz} column window of the {lat.Lx}x{lat.Lz} workload (periodic in the window), "
              f"1 oracle step per timed step, {tot:.1f} s in all")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded three-layer Rayleigh-Taylor initial state)",
            "config": {"workload": "three-layer RT, D2Q37, 1024x2048, tau=0.7, g=5e-5, 64 modes",
                       "Lx": lat.Lx, "Lz": lat.Lz, "sample": sample},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_variant(torch, lbm, lat, prec, steps, warmup, stream):
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
    L.init_from(lat)
    L.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    L.close()
    return ms


def bench_precision(torch, lbm, steps, stream):
    """The precision configuration: 4096 x 8192 (33.6 M sites, 128 modes), `steps` steps of
    the FP64-accurate (float-float) step, the FP32-storage step and the FP32 deviation-storage
    step from the same seeded initial state; relative L2 errors of rho and T and relative
    errors of both fronts' widths of each FP32 run against the FP64-accurate one (FP32 storage
    at the top level, deviation storage under f32_dev_errors), the mass drift, and the
    throughput of each (CUDA events around the stepping only; ~222 waves of blocks per launch
    against ~14 on 1024 x 2048)."""
    lat = W.PRECISION_4096x8192
    peak = float(measured_peaks()[0].get("hbm_gbs", 6400.0))
    out = {"workload": f"{lat.Lx}x{lat.Lz}, {steps} steps, tau={lat.tau}, g={lat.grav}, {lat.K} modes (seed {lat.seed})"}
    fields = {}
    for prec in ("f64_ff", "f32", "f32_dev"):
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        m0 = L.global_sums()[0]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rho, _, _, T = L.moments()
        widths = L.widths(lat.T_u, lat.T_m, lat.T_d)
        m1 = L.global_sums()[0]
        L.close()
        torch.cuda.empty_cache()
        gbs = 2 * Q * BYTES_PER_POP[prec] * lat.sites / (ms * 1e-3) / 1e9
        out[prec] = {"ms_per_step": ms, "mlups": lat.sites / (ms * 1e-3) / 1e6, "gbs": gbs, "hbm_frac": gbs / peak,
                     "widths": [float(v) for v in widths], "mass_rel_drift": float(abs(m1 - m0) / m0)}
        fields[prec] = (rho, T, widths)
    (r64, T64, w64) = fields["f64_ff"]
    for low in ("f32", "f32_dev"):
        r32, T32, w32 = fields[low]
        err = {"rho_rel_l2": float(np.linalg.norm(r32 - r64) / np.linalg.norm(r64)),
               "T_rel_l2": float(np.linalg.norm(T32 - T64) / np.linalg.norm(T64)),
               "T_max_abs": float(np.abs(T32 - T64).max()),
               "width_rel_err": [float(abs(a - b) / abs(b)) for a, b in zip(w32, w64)]}
        if low == "f32":      # the FP32-storage figures at the top level, as before
            out.update(err)
        else:
            out["f32_dev_errors"] = err
        out["speedup_" + low] = out["f64_ff"]["ms_per_step"] / out[low]["ms_per_step"]
    out["error_bound"] = 1e-5
    out["fields_within_bound"] = bool(out["rho_rel_l2"] < 1e-5 and out["T_rel_l2"] < 1e-5)
    out["f32_dev_fields_within_bound"] = bool(out["f32_dev_errors"]["rho_rel_l2"] < 1e-5 and
                                              out["f32_dev_errors"]["T_rel_l2"] < 1e-5)
    return out


def bench_ensemble(torch, lbm, prec, steps, stream, tune_steps=20):
    """The 48-lattice ensemble (16 x 256x512, 16 x 512x1024, 16 x 384x1536, seeds 100..147):
    the autotuner's choice over every launch shape on `tune_steps`-step trials, then each
    launch shape (one launch per step, one persistent launch) at its best tile height,
    captured as one CUDA graph of `steps` steps from the initial state and timed on one
    replay."""
    lats = W.ensemble_48()
    Ls = []
    for lat in lats:
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        Ls.append(L)
    ens = lbm.Ensemble(Ls)
    tuned = ens.tune(steps=tune_steps)
    sites = sum(l.sites for l in lats)
    bps = 2 * Q * BYTES_PER_POP[prec]
    out = {"lattices": len(lats), "sites": sites, "steps": steps, "tuned": tuned,
           "tuner_trial_steps": tune_steps, "graph": "one CUDA graph replay of all steps"}
    for mode, key in ((0, "per_step_launches"), (1, "persistent_launch")):
        ens.config(mode=mode, tile_z=128)
        for L, lat in zip(Ls, lats):      # every timed run starts from the initial state
            L.init_from(lat)
        ens.step(2)                       # untimed warm-up (even: the lattices stay in their buffers)
        ens.sync()
        for L, lat in zip(Ls, lats):
            L.init_from(lat)
        ens.capture(steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.graph_launch()
        e1.record(stream)
        e1.synchronize()
        ens.sync()
        ms = e0.elapsed_time(e1)
        mass = Ls[0].global_sums()[0]
        out[key] = {"tile_z": 128, "ms_per_step": ms / steps, "mlups": sites * steps / (ms * 1e-3) / 1e6,
                    "gbs": bps * sites * steps / (ms * 1e-3) / 1e9, "finite": bool(np.isfinite(mass))}
    out["tuned_launch"] = "one persistent launch" if tuned["mode"] == 1 else "one launch per step"
    ens.close()
    for L in Ls:
        L.close()
    torch.cuda.empty_cache()
    return out


def bench_adjoint(torch):
    """Gradient workload: 256x512, 2000 steps, checkpoint every 100: forward and backward
    (recompute + adjoint) wall times and device memory, for the three backward stores of the
    float-float driver (recomputed moment records, with the recompute of earlier segments
    overlapping the adjoint of the current one on a second stream, four record sets (the
    default) or two, and without the overlap; moment records taped in the forward; segment
    states) and for an FP32-storage run."""
    from paper_1405_1253_b300 import adjoint
    lat = W.GRADIENT_256x512
    out = {"workload": "256x512, 2000 steps, checkpoint every 100, 16 modes per front (f64_ff)"}
    m = lat.modes()
    for key, store, prec, pipe, nset in (("moments", "moments", "f64_ff", True, None),
                                         ("moments_2sets", "moments", "f64_ff", True, 2),
                                         ("moments_serial", "moments", "f64_ff", False, None),
                                         ("tape", "tape", "f64_ff", False, None), ("states", "states", "f64_ff", False, None),
                                         ("f32", "states", "f32", False, None)):
        drv = adjoint.WidthGradient(lat, W.GRADIENT_STEPS, W.GRADIENT_CKPT, prec=prec, store=store, pipeline=pipe,
                                    record_sets=nset)
        drv.forward(m.amp_lo, m.amp_hi)      # warm
        drv.backward()
        drv.forward(m.amp_lo, m.amp_hi)
        g_lo, g_hi = drv.backward()
        st = drv.stats
        drv.close()
        mem = st.checkpoint_bytes + st.segment_bytes + 2 * st.state_bytes
        out[key] = {"forward_s": st.forward_s, "backward_s": st.backward_s,
                      "record_sets": len(getattr(drv, "moms_sets", [])) or None,
                      "recomputed_steps": st.recompute_steps,
                      "backward_over_forward": st.backward_s / st.forward_s,
                      "memory_bytes": mem, "forward_memory_bytes": 2 * st.state_bytes,
                      "memory_over_forward": mem / (2 * st.state_bytes),
                      "grad_norm": float(np.sqrt((g_lo ** 2).sum() + (g_hi ** 2).sum()))}
    # the tape's and the moment stores' forwards also write moment records: their backward
    # against the plain checkpointed forward (the state store's) too
    for key in ("tape", "moments", "moments_2sets", "moments_serial"):
        out[key]["backward_over_plain_forward"] = out[key]["backward_s"] / out["states"]["forward_s"]
    return out

def bench_slabs(torch, lbm, lat, steps, stream, prec="f64_ff"):
    """The x-slab decomposition of Sec. III.B on this device (halos exchanged by device
    copies each step): MLUPS for 1, 4 and 8 slabs with the exchange overlapped with the
    bulk update, and 8 slabs without overlap, against the single-domain step."""
    def timed(fn):
        fn(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
    L.init_from(lat)
    out = {"workload": f"{lat.Lx}x{lat.Lz}, {prec}, {steps} steps", "single_ms": timed(L.step)}
    for n, ov in ((1, True), (4, True), (8, True), (8, False)):
        S = lbm.Slabs(L, n)
        S.scatter()
        ms = timed(lambda k: S.step(k, ov))
        S.close()
        key = f"{n}_slabs" + ("" if ov else "_no_overlap")
        out[key] = {"ms": ms, "mlups": lat.sites / (ms * 1e-3) / 1e6,
                    "halo_bytes_per_step": 2 * n * 3 * lat.Lz * 37 * lbm.POP_BYTES[prec]}
    L.close()
    return out


def bench_push(torch, lbm, lat, steps, stream):
    """Pull form (lbm_step: misaligned reads, aligned writes) against the push form
    (lbm_step_push: aligned reads, misaligned writes), Sec. III.B."""
    out = {"workload": f"{lat.Lx}x{lat.Lz}, {steps} steps"}
    for prec in ("f64_ff", "f32"):
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        res = {}
        for name, fn in (("pull", L.step), ("push", L.step_push)):
            fn(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            res[name] = {"ms": ms, "mlups": lat.sites / (ms * 1e-3) / 1e6}
        res["pull_over_push"] = res["push"]["ms"] / res["pull"]["ms"]
        out[prec] = res
        L.close()
    return out


def bench_adjoint_kernel(torch, lbm, lat, steps, stream, peak, fp64_rate=None):
    """The adjoint step kernel alone on the 1024x2048 state, float-float, native FP64 and FP32:
    it reads f_t and lam_{t+1} and writes lam_t, 3 x 37 populations per site (888 B in FP64
    storage, 444 B in FP32)."""
    out = {"workload": f"{lat.Lx}x{lat.Lz}, FP64 storage, {steps} adjoint steps", "bytes_per_site": 888}
    for prec in ("f64_ff", "f64", "f32"):
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        f = L.current().clone()              # the state in the storage precision
        lam = [torch.rand_like(f), torch.empty_like(f)]
        for i in range(3):
            L.adjoint_step(f, lam[i & 1], lam[(i + 1) & 1])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            L.adjoint_step(f, lam[i & 1], lam[(i + 1) & 1])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bps = 3 * Q * BYTES_PER_POP[prec]                # 888 B/site (FP64 storage), 444 (FP32)
        gbs = bps * lat.sites / (ms * 1e-3) / 1e9
        out[prec] = {"ms": ms, "mlups": lat.sites / (ms * 1e-3) / 1e6, "gbs": gbs, "hbm_frac": gbs / peak,
                     "bytes_per_site": bps}
        if prec == "f64_ff":
            out[prec]["fp64"] = fp64_roof("k_adjoint_ff", lat.sites, ms, fp64_rate)
        if prec == "f64_ff":
            # the same adjoint with f_t given by its moment record: 32 + 296 + 296 = 624 B/site
            wa, wb = torch.empty_like(f), torch.empty_like(f)
            mom = [torch.empty(4 * lat.sites, dtype=torch.int64, device=f.device)]
            L.record_moments(f, wa, wb, mom)
            for i in range(3):
                L.adjoint_chain_moments(mom, lam[i & 1], lam[(i + 1) & 1])
            torch.cuda.synchronize()
            e0.record(stream)
            for i in range(steps):
                L.adjoint_chain_moments(mom, lam[i & 1], lam[(i + 1) & 1])
            e1.record(stream)
            e1.synchronize()
            msm = e0.elapsed_time(e1) / steps
            gbm = 624 * lat.sites / (msm * 1e-3) / 1e9
            out["f64_ff_moments"] = {"ms": msm, "mlups": lat.sites / (msm * 1e-3) / 1e6, "gbs": gbm,
                                     "hbm_frac": gbm / peak, "bytes_per_site": 624,
                                     "traffic": ncu_traffic("k_adjoint_ff_moments", lat.sites),
                                     "fp64": fp64_roof("k_adjoint_ff_moments", lat.sites, msm, fp64_rate)}
        L.close()
    out["f64_ff"]["traffic"] = ncu_traffic("k_adjoint_ff", lat.sites)
    return out


def bench_walls(torch, lbm, lat, steps, stream):
    """Thermal walls (lbm_set_walls: two launches per step) against the bounce-back step on
    the 1024x2048 state, float-float and FP32 storage."""
    out = {"workload": f"{lat.Lx}x{lat.Lz}, {steps} steps, walls at T_d / T_u"}
    for prec in ("f64_ff", "f32"):
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        res = {}
        for thermal in (False, True):
            L.set_walls(thermal, lat.T_d, lat.T_u)
            L.step(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.step(steps)
            e1.record(stream)
            e1.synchronize()
            res["thermal" if thermal else "bounce_back"] = lat.sites * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6
        out[prec] = {"bounce_back_mlups": res["bounce_back"], "thermal_mlups": res["thermal"],
                     "thermal_over_bounce_back": res["thermal"] / res["bounce_back"]}
        if prec == "f64_ff":                 # the adjoint step under each wall rule
            f = L.populations_device().clone()
            lam = [torch.rand_like(f), torch.empty_like(f)]
            for thermal in (False, True):
                L.set_walls(thermal, lat.T_d, lat.T_u)
                for i in range(3):
                    L.adjoint_step(f, lam[i & 1], lam[(i + 1) & 1])
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for i in range(20):
                    L.adjoint_step(f, lam[i & 1], lam[(i + 1) & 1])
                e1.record(stream)
                e1.synchronize()
                key = "adjoint_thermal_mlups" if thermal else "adjoint_bounce_back_mlups"
                out[prec][key] = lat.sites * 20 / (e0.elapsed_time(e1) * 1e-3) / 1e6
        L.close()
    return out


def fp32_error(torch, lbm, lat, steps, stream):
    """Relative L2 error of rho and T of the FP32-storage step (top level) and of the FP32
    deviation-storage step (f32_dev) against the FP64-accurate step after `steps` steps from
    the same initial state."""
    out = {}
    fields = {}
    for prec in ("f64_ff", "f32", "f32_dev"):
        L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
        L.init_from(lat)
        L.step(steps)
        rho, _, _, T = L.moments()
        fields[prec] = (rho, T, L.widths(lat.T_u, lat.T_m, lat.T_d))
        L.close()
    out["steps"] = steps
    r64, T64, w64 = fields["f64_ff"]
    for low in ("f32", "f32_dev"):
        r32, T32, w32 = fields[low]
        err = {"rho_rel_l2": float(np.linalg.norm(r32 - r64) / np.linalg.norm(r64)),
               "T_rel_l2": float(np.linalg.norm(T32 - T64) / np.linalg.norm(T64)),
               "width_rel_err": [float(abs(a - b) / abs(b)) for a, b in zip(w32, w64)]}
        if low == "f32":
            out.update(err)
        else:
            out["f32_dev"] = err
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1405_1253_b300 import lbm
    lat = W.THROUGHPUT_1024x2048
    sites = lat.sites
    prec = args.prec
    stream = torch.cuda.current_stream()
    L = lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=stream)
    L.init_from(lat)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    L.step(args.warmup)
    e1.record(stream)
    torch.cuda.synchronize()
    warm_ms_step = e0.elapsed_time(e1) / args.warmup
    # the FP64 pipe's rate on this GPU, the second roof of the FP64-storage step (outside the
    # timed region; two launches of about 2.6 ms)
    fp64_rate = lbm.probe_fp64_rate(512)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # The timed region (exactly K steps, a barrier and a device synchronisation on each side)
    # is repeated R times so that the clock sampler covers it: R is set from the warm-up's
    # step time (the same R on every rank) for about --clock-window seconds, at least 3; the
    # reported time is the median repeat (max over ranks).
    reps = repeats_for(warm_ms_step * args.steps, args.clock_window, ws)
    rep_ms = []
    with ClockSampler(local) as clk:
        clk.wait_first()
        for _ in range(reps):
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            L.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            rep_ms.append(e0.elapsed_time(e1))
    ms_total, ms_step, mlups = aggregate_ranks(statistics.median(rep_ms), args.steps, sites, ws, device="cuda")
    mass = L.global_sums()[0]

    # end to end through the C ABI with host buffers: every step copies its input state in
    # from pinned host memory, steps, and copies the result out (lbm_step_host, which runs
    # the copy out of one step concurrently with the copy in of the next)
    n = Q * sites
    e2e_mlups = None                      # lbm_step_host takes FP64 host buffers: FP64 storage only
    if BYTES_PER_POP[prec] == 8:
        h_in = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_out = torch.empty(n, dtype=torch.float64, pin_memory=True)
        h_in.copy_(L.populations_device().cpu())
        L.step_host([h_in], [h_out])      # warm-up (creates the copy streams)
        e2e_steps = 6
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.step_host([h_in] * e2e_steps, [h_out] * e2e_steps)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_mlups = ws * sites / e2e_s / 1e6
    L.close()

    variants = {}
    if not args.no_variants:
        for v in ("f64_ff", "f64", "f32", "f32_dev"):
            vsteps = 10 if v == "f64" else 20
            vms = time_variant(torch, lbm, lat, v, vsteps, 3, stream)
            vbytes = 2 * Q * BYTES_PER_POP[v] * sites
            variants[v] = {"mlups": sites / (vms * 1e-3) / 1e6, "ms_per_step": vms,
                           "gbs": vbytes / (vms * 1e-3) / 1e9, "arith": ARITH[v]}
            roof = fp64_roof(KERNEL[v], sites, vms, fp64_rate)
            if roof is not None:
                variants[v]["fp64"] = roof

    extras = {}
    if not args.no_extras and rank == 0:
        extras["fp32_error_1024x2048"] = fp32_error(torch, lbm, lat, 500, stream)
        es = torch.cuda.Stream()           # graph capture needs a non-default stream
        extras["ensemble_f64"] = bench_ensemble(torch, lbm, "f64_ff", W.ENSEMBLE_STEPS, es)
        extras["ensemble_f32"] = bench_ensemble(torch, lbm, "f32", W.ENSEMBLE_STEPS, es)
        extras["adjoint"] = bench_adjoint(torch)
        extras["adjoint_kernel"] = bench_adjoint_kernel(torch, lbm, lat, 20, stream,
                                                        float(measured_peaks()[0].get("hbm_gbs", 6400.0)), fp64_rate)
        extras["slabs"] = bench_slabs(torch, lbm, lat, 100, stream)
        extras["push_vs_pull"] = bench_push(torch, lbm, lat, 200, stream)
        extras["walls"] = bench_walls(torch, lbm, lat, 200, stream)
        extras["precision_4096x8192"] = bench_precision(torch, lbm, W.PRECISION_STEPS, stream)

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6400.0))
    alg_bytes = 2 * Q * BYTES_PER_POP[prec] * sites
    achieved = alg_bytes / (ms_step * 1e-3) / 1e9
    for v in variants.values():
        v["hbm_frac"] = v["gbs"] / peak
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        ncols, nsteps = 256, 30          # about 10 s of oracle work on a 16-core host
        cpu_mlups, cpu_s = time_oracle(lat, ncols, nsteps)
        cpu = {"value": cpu_mlups, "unit": "MLUPS", "cores": cores_used(), "kind": "oracle",
               "sample": f"{ncols}x{lat.Lz} column window of the {lat.Lx}x{lat.Lz} workload, {nsteps} steps ({cpu_s:.1f} s)"}
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ARITH[prec],
        "data": "synthetic (seeded three-layer Rayleigh-Taylor initial state)",
        "config": {"workload": "three-layer RT, D2Q37, 1024x2048, tau=0.7, g=5e-5, 64 modes",
                   "Lx": lat.Lx, "Lz": lat.Lz,
                   "storage": {"f32": "f32", "f32_dev": "f32 deviation from a per-row f64 reference"}.get(prec, "f64"),
                   "arith": ARITH[prec], "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "working set 1.24 GB per step > 126 MB L2 (no flush needed)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": ncu_traffic(KERNEL[prec], sites),
                     "bytes_per_site": 2 * Q * BYTES_PER_POP[prec],
                     "spec_peak": SPEC_HBM_GBS, "frac_of_spec": achieved / SPEC_HBM_GBS,
                     "target_frac": 0.70, "meets_target": bool(achieved / peak >= 0.70),
                     "kernel": KERNEL[prec],
                     "secondary": fp64_roof(KERNEL[prec], sites, ms_step, fp64_rate)},
        "e2e": ({"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                 "note": "lbm_step_host: per step host->device state, one step, device->host state (pinned; copies of consecutive steps overlapped)"}
                if e2e_mlups is not None else
                {"value": None, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                 "note": "lbm_step_host takes FP64 host buffers (FP64-storage contexts); not measured for this precision"}),
        "gpu_launches": args.steps,
        "timed_repeats": {"count": len(rep_ms), "ms_per_step_min": min(rep_ms) / args.steps,
                          "ms_per_step_median": statistics.median(rep_ms) / args.steps,
                          "ms_per_step_max": max(rep_ms) / args.steps,
                          "note": "each repeat is one timed region of exactly `steps` launches; value = median repeat"},
        "clocks": clk.summary(),
        "variants": variants,
        "mass_after": mass,
        "cpu_baseline": cpu,
        "paper_context": {"source": "the paper's Table I (FP64)", "note": "context, not the target",
                          "figures": PAPER_TABLE_I},
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["f64_ff", "f64", "f32", "f32_dev"], default="f64_ff")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ensemble, adjoint, slab, push, wall, precision and FP32-error sections")
    ap.add_argument("--clock-window", type=float, default=1.5,
                    help="seconds of repeated timed regions the clock record must cover")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

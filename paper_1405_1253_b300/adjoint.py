"""Gradient of the mixing-layer widths with respect to the interface-mode amplitudes.

The loss is L = L_u + L_d, the threshold widths of the two fronts (Sec. IV) at step N of
the three-layer run started from the perturbed initial state (Sec. I).  The forward pass
runs N fused steps, keeping every K-th state as a device checkpoint.  The backward pass
starts from lam_N = dL/df_N (width adjoint -> mean profile -> T -> f), then, segment by
segment from the last, recomputes the K states of the segment from its checkpoint into
device buffers (lbm_step_chain) and applies the adjoint step K times (lbm_adjoint_chain,
lam_t = P^T J_C^T lam_{t+1}); the
adjoint of the initial state finally gives dL/dA.  Every step runs in the CUDA library;
this module only orders the calls and owns the buffers (through PyTorch).

Memory: (N/K) checkpoints and 2 adjoint fields, each 37 Lx Lz doubles, and per segment either
(K - 1) states or K moment records of 4 Lx Lz int64 plus two states to step through (with the
moment records: `record_sets` sets of K records, by default four when the recompute of earlier
segments overlaps the adjoint of the current one on a second stream and one without; the
forward records the moments of its last `record_sets` segments into them directly, so the
backward recomputes only the segments before those).  The "tape" store instead records the
moments of all N steps during the forward pass (32 bytes per site and step, no checkpoints),
so the backward recomputes nothing.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm as _lbm
from .workloads import Lattice as LatticeDesc

Q = 37


@dataclass
class AdjointStats:
    forward_s: float = 0.0
    backward_s: float = 0.0
    recompute_steps: int = 0
    adjoint_steps: int = 0
    checkpoint_bytes: int = 0
    segment_bytes: int = 0
    state_bytes: int = 0
    widths: np.ndarray = field(default_factory=lambda: np.zeros(2))


class WidthGradient:
    """Forward/backward driver for one lattice description: prec "f64_ff" (float-float step
    and adjoint, the default), "f64" (native FP64) or "f32" (FP32 storage and arithmetic:
    the gradient of the FP32 run, to FP32 rounding).
    store "moments" (f64_ff only, its default): the backward recomputes each segment keeping
    only the per-site moments the adjoint needs (32 bytes per site and step); "states": it
    keeps the segment's states (296 bytes per site and step); "tape" (f64_ff only): the
    forward records the moments of every step (N x 32 bytes per site; ckpt only sets the
    length of each adjoint chain call) and the backward runs the adjoint steps alone.
    walls=(T_bottom, T_top): thermal walls (lbm_set_walls) in the forward and the adjoint
    (f64_ff, states).  pipeline (store "moments"): the recompute of earlier segments runs on a
    second stream while the adjoint chain of segment s runs; record_sets (store "moments"):
    the sets of K moment records, at least 2 with the pipeline (default 4) and 1 without
    (default 1); the recompute of segment r refills set r % record_sets after the adjoint of
    r + record_sets has read it, and the forward records its last record_sets segments itself.
    Every store and setting gives the same gradient bit for bit."""

    def __init__(self, lat: LatticeDesc, nsteps: int, ckpt: int, prec: str = "f64_ff", store: str = None,
                 walls=None, pipeline: bool = True, record_sets: int = None):
        import torch
        if nsteps < 1 or ckpt < 1 or nsteps % ckpt:
            raise ValueError("nsteps must be a positive multiple of ckpt")
        self.torch = torch
        self.lat = lat
        self.N = int(nsteps)
        self.K = int(ckpt)
        if prec not in ("f64", "f64_ff", "f32"):
            raise ValueError("prec is 'f64_ff', 'f64' or 'f32'")
        self.prec = prec
        self.store = store or ("moments" if prec == "f64_ff" and walls is None else "states")
        if self.store not in ("moments", "states", "tape") or (
                self.store != "states" and (prec != "f64_ff" or walls)):
            raise ValueError("store is 'states', or 'moments' / 'tape' with prec 'f64_ff' and bounce-back walls")
        self.pipeline = False
        self.n_taped = 0
        self.L = _lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec)
        if walls is not None:                      # thermal walls at (T_bottom, T_top)
            self.L.set_walls(True, *walls)
        n = Q * lat.Lx * lat.Lz
        dev = self.L.device
        dt = self.L.current().dtype              # checkpoints in the storage precision
        nck = 0 if self.store == "tape" else self.N // self.K
        self.ckpts = [torch.empty(n, dtype=dt, device=dev) for _ in range(nck)]
        if self.store == "tape":
            # moments of all N steps, and two states to step through
            self.moms = torch.empty((self.N, 4 * lat.Lx * lat.Lz), dtype=torch.int64, device=dev)
            self.work = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
            seg_bytes = self.moms.numel() * 8 + 2 * 8 * n
        elif self.store == "states":
            # states f_{sK+1} .. f_{sK+K-1} of a segment (f_{sK} is its checkpoint)
            self.seg = torch.empty((self.K - 1, n), dtype=dt, device=dev)
            seg_bytes = self.seg.element_size() * n * (self.K - 1)
        else:
            # moments of the K steps of a segment, and two states to step through; with the
            # pipeline, two sets of records: the recompute of segment s - 1 (a second context on
            # a second stream) fills one while the adjoint chain of segment s reads the other
            self.pipeline = bool(pipeline) and self.N // self.K > 1
            nset = record_sets if record_sets is not None else (4 if self.pipeline else 1)
            if nset < (2 if self.pipeline else 1):
                raise ValueError("record_sets must be at least 2 with the pipeline, 1 without")
            self.moms_sets = [torch.empty((self.K, 4 * lat.Lx * lat.Lz), dtype=torch.int64, device=dev)
                              for _ in range(nset)]
            self.moms = self.moms_sets[0]
            self.work = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
            seg_bytes = nset * self.moms.numel() * 8 + 2 * 8 * n
            # the forward records the moments of its last segments straight into the record
            # sets (one per set), so that the backward's first adjoint chains need no recompute
            self.n_taped = min(nset, self.N // self.K)
            if self.pipeline:
                self.rec_stream = torch.cuda.Stream(device=dev)
                self.Lrec = _lbm.Lattice(lat.Lx, lat.Lz, lat.tau, lat.grav, prec=prec, stream=self.rec_stream)
                seg_bytes += 2 * 8 * n          # the recompute context's own two buffers
        self.lam = [torch.empty(n, dtype=dt, device=dev) for _ in range(2)]
        es = self.lam[0].element_size()
        self.stats = AdjointStats(checkpoint_bytes=es * n * len(self.ckpts), segment_bytes=seg_bytes,
                                  state_bytes=es * n)
        self._amps = None

    def _init(self, amp_lo, amp_hi, ph_lo, ph_hi):
        lat = self.lat
        self.L.init_layers(lat.T_u, lat.T_m, lat.T_d, lat.z_lo, lat.z_hi, lat.rho_ref, lat.tanh_w,
                           amp_lo, ph_lo, amp_hi, ph_hi)

    def forward(self, amp_lo, amp_hi, ph_lo=None, ph_hi=None) -> float:
        """Run N steps from the initial state with these amplitudes (and phases; by default
        the description's); returns L_u + L_d."""
        torch = self.torch
        lat = self.lat
        m = lat.modes()
        amp_lo = np.asarray(amp_lo, dtype=np.float64)
        amp_hi = np.asarray(amp_hi, dtype=np.float64)
        ph_lo = np.asarray(m.ph_lo if ph_lo is None else ph_lo, dtype=np.float64)
        ph_hi = np.asarray(m.ph_hi if ph_hi is None else ph_hi, dtype=np.float64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self._init(amp_lo, amp_hi, ph_lo, ph_hi)
        if self.store == "tape":
            # the N steps, recording each one's moments; f_N ends in work[(N - 1) % 2]
            self.L.record_moments(self.L.current(), self.work[0], self.work[1], list(self.moms))
            self.L.current().copy_(self.work[(self.N - 1) % 2])
        else:
            S = self.N // self.K
            for s in range(S):
                if s >= S - self.n_taped:
                    # a segment the backward reads first: its K steps recording their moments
                    # into the record set the backward's adjoint chain of s reads (the same
                    # arithmetic as the plain step, so the same states bit for bit)
                    sets = self.moms_sets
                    self.L.record_moments(self.L.current(), self.work[0], self.work[1],
                                          list(sets[s % len(sets)]))
                    self.L.current().copy_(self.work[(self.K - 1) % 2])
                else:
                    self.ckpts[s].copy_(self.L.current())
                    self.L.step(self.K)
        widths, dL = self.L.widths(lat.T_u, lat.T_m, lat.T_d, with_grad=True)
        self.stats.forward_s = time.perf_counter() - t0
        self.stats.widths = widths
        self._amps = (amp_lo, amp_hi, ph_lo, ph_hi)
        self._dL = dL
        self._fN = self.L.current().clone()
        return float(widths.sum())

    def backward(self, grad_out: float = 1.0):
        """dL/damp_lo, dL/damp_hi for the last forward call (scaled by grad_out); the phase
        gradients dL/dphi_lo, dL/dphi_hi are left in self.grad_phases."""
        torch = self.torch
        lat = self.lat
        if self._amps is None:
            raise RuntimeError("backward before forward")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.stats.recompute_steps = self.stats.adjoint_steps = 0    # counts of this backward
        cur, nxt = self.lam
        self.L.loss_adjoint(self._fN, self._dL * float(grad_out), cur)
        segments = range(self.N // self.K - 1, -1, -1)
        if self.store == "moments" and self.pipeline:
            cur = self._backward_pipelined(cur, nxt)
            segments = ()
        for s in segments:
            if self.store == "tape":
                # the K recorded steps of segment s, adjoint steps only
                flip = self.L.adjoint_chain_moments([self.moms[s * self.K + j] for j in range(self.K)], cur, nxt)
            elif self.store == "states":
                # recompute f_{sK+1} .. f_{sK+K-1} from the checkpoint into the segment buffers
                # (one library call), then the K adjoint steps of the segment (one call)
                states = [self.ckpts[s]] + [self.seg[j] for j in range(self.K - 1)]
                self.L.step_chain(states)
                self.stats.recompute_steps += self.K - 1
                flip = self.L.adjoint_chain(states, cur, nxt)
            else:
                # recompute the K steps of the segment keeping only their moments (the last
                # segment's were recorded by the forward)
                sets = self.moms_sets
                moms = [sets[s % len(sets)][j] for j in range(self.K)]
                if s < self.N // self.K - self.n_taped:
                    self.L.record_moments(self.ckpts[s], self.work[0], self.work[1], moms)
                    self.stats.recompute_steps += self.K
                flip = self.L.adjoint_chain_moments(moms, cur, nxt)
            if flip == 1:
                cur, nxt = nxt, cur
            self.stats.adjoint_steps += self.K
        amp_lo, amp_hi, ph_lo, ph_hi = self._amps
        g_lo, g_hi, p_lo, p_hi = self.L.init_adjoint(cur, lat.T_u, lat.T_m, lat.T_d, lat.z_lo, lat.z_hi,
                                                     lat.rho_ref, lat.tanh_w, amp_lo, ph_lo, amp_hi, ph_hi,
                                                     phases=True)
        self.grad_phases = (p_lo, p_hi)
        self.stats.backward_s = time.perf_counter() - t0
        return g_lo, g_hi

    def _backward_pipelined(self, cur, nxt):
        """The moment-record backward with the recomputes of earlier segments (recording
        context, second stream) overlapping the adjoint chains (the context's stream), n record
        sets: the adjoint of s waits for the records of s (recorded by the forward for the last
        n segments); the recompute of r refills set r mod n, so it waits for the adjoint of
        r + n, the set's last reader, and is issued right after that adjoint is (a stream must
        not wait on an event before its record is enqueued).  Returns the tensor holding lam_0."""
        torch = self.torch
        S = self.N // self.K
        main = self.L.stream
        rec = self.rec_stream
        ev_rec = [torch.cuda.Event() for _ in range(S)]
        ev_adj = [torch.cuda.Event() for _ in range(S)]
        rec.wait_stream(main)                     # the checkpoints and lam_N are written on main

        def record(s):
            moms = self.moms_sets[s % nset]
            if s + nset < S:
                rec.wait_event(ev_adj[s + nset])  # its record set was read by the adjoint of s + nset
            self.Lrec.record_moments(self.ckpts[s], self.work[0], self.work[1], [moms[j] for j in range(self.K)])
            ev_rec[s].record(rec)
            self.stats.recompute_steps += self.K

        nset = len(self.moms_sets)
        first_rec = S - 1 - self.n_taped      # segments above it were recorded by the forward
        pending = [first_rec]                 # next segment to recompute (descending)

        def issue_records(limit):
            # every recompute down to segment `limit` whose set's last reader (the adjoint of
            # r + nset) has been issued, so that its event wait is ordered after that record
            while pending[0] >= 0 and pending[0] >= limit:
                record(pending[0])
                pending[0] -= 1

        issue_records(S - nset)
        for s in range(S - 1, -1, -1):
            if s <= first_rec:
                main.wait_event(ev_rec[s])
            moms = self.moms_sets[s % nset]
            flip = self.L.adjoint_chain_moments([moms[j] for j in range(self.K)], cur, nxt)
            ev_adj[s].record(main)
            if flip == 1:
                cur, nxt = nxt, cur
            self.stats.adjoint_steps += self.K
            issue_records(s - nset)
        return cur

    def close(self):
        self.L.close()
        if getattr(self, "Lrec", None) is not None:
            self.Lrec.close()


def _make_function():
    import torch

    class WidthLoss(torch.autograd.Function):
        """torch.autograd.Function: (amp_lo, amp_hi) -> L_u + L_d at step N."""

        @staticmethod
        def forward(ctx, amp_lo, amp_hi, driver: WidthGradient):
            val = driver.forward(amp_lo.detach().cpu().numpy(), amp_hi.detach().cpu().numpy())
            ctx.driver = driver
            ctx.dtype, ctx.device = amp_lo.dtype, amp_lo.device
            return torch.tensor(val, dtype=amp_lo.dtype, device=amp_lo.device)

        @staticmethod
        def backward(ctx, grad):
            g_lo, g_hi = ctx.driver.backward(float(grad))
            mk = lambda a: torch.as_tensor(a, dtype=ctx.dtype, device=ctx.device)
            return mk(g_lo), mk(g_hi), None

    return WidthLoss


_WidthLoss = None


def width_loss(amp_lo, amp_hi, driver: WidthGradient):
    """Differentiable L_u + L_d (torch tensors of mode amplitudes in, scalar tensor out)."""
    global _WidthLoss
    if _WidthLoss is None:
        _WidthLoss = _make_function()
    return _WidthLoss.apply(amp_lo, amp_hi, driver)

"""The 3DGS training step on the CUDA library: buffers, schedule, autograd.

`Frame` owns the device buffers of one batch of views for N Gaussians and runs
the hot path through the C ABI:

    project -> bin_sort -> [features -> MLP -> order] -> render_fwd -> L1
            -> render_bwd -> project_bwd -> Adam

`RasterizeGaussians` is the same forward/backward behind torch.autograd.
Every arithmetic step runs in libgs103.so; torch only provides device memory
and the stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .scenes import PARAM_FLOATS

# Per-group Adam learning rates: means, log-scales, quaternions, opacity
# logits, SH DC, SH rest (the 3DGS defaults).
DEFAULT_LR = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-15
MLP_W = 321


def _dev():
    if not torch.cuda.is_available():
        raise L.GsError("a CUDA device is required (no CPU fallback)")
    return torch.device("cuda")


def param_views(flat: torch.Tensor, N: int) -> dict:
    """Named views of a grouped 59 N buffer."""
    o, out = 0, {}
    for name, w in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
        out[name] = flat[o:o + w * N]
        o += w * N
    return out


def to_device_params(scene, device=None) -> torch.Tensor:
    """The scene's grouped parameter buffer on the device (59 N floats)."""
    return torch.from_numpy(scene.flat()).to(device or _dev())


@dataclass
class Schedule:
    """How render CTAs take tiles.  'raster': one CTA per tile, both passes.
    'count' (the plain split): persistent CTAs, tiles with the most
    instances first, both passes.  'learned': the forward in raster order
    (measured fastest: neighbouring tiles share Gaussians in L2), the reverse
    pass by persistent CTAs in the order of a cost MLP trained on the reverse
    pass's own tile times, longest predicted first, the tiles predicted to
    take more than a CTA's share split into strips; judged against the count
    order by measured duration."""
    mode: str = "raster"
    feature_cap: int = 128
    mlp_lr: float = 1e-3
    train_every: int = 4
    bwd_order: str = "forward"
    seed: int = 0
    # learned mode: the count order judges the learned one by measured
    # makespan (every judge_every-th pass of each kind runs the count order,
    # the pass half-way between runs the learned order, the others whichever
    # is faster on average) and is used until the learned order wins; False
    # uses the learned orders without judging
    judge: bool = True
    judge_every: int = 8


class PassJudge:
    """Chooses the tile order of one render pass between two by measured
    duration: a candidate (by default the learned cost model's order) and a
    fallback (by default the instance count's).  Every `every`-th pass runs
    the fallback, the pass half-way between runs the candidate, and the
    others the order with the lower mean duration (an exponential average
    over its measured passes; the fallback until both have been measured).
    Durations are CUDA events around the pass's kernel, read back without
    waiting."""

    def __init__(self, every: int = 8, weight: float = 0.25, arms=("learned", "count")):
        self.every = max(2, int(every))
        self.weight = weight
        self.cand, self.fallback = arms
        self.mean = {self.cand: None, self.fallback: None}
        self.passes = {self.cand: 0, self.fallback: 0}
        self.pending = []
        self.k = 0

    def winner(self) -> str:
        l, c = self.mean[self.cand], self.mean[self.fallback]
        return self.cand if l is not None and c is not None and l < c else self.fallback

    def pick(self) -> str:
        self.poll()
        r = self.k % self.every
        self.k += 1
        if r == 0:
            return self.fallback
        if r == self.every // 2:
            return self.cand
        return self.winner()

    def start(self, which: str):
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return which, e

    def stop(self, token) -> None:
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        self.pending.append((token[0], token[1], e))

    def poll(self) -> None:
        keep = []
        for which, a, b in self.pending:
            if not b.query():
                keep.append((which, a, b))
                continue
            ms = a.elapsed_time(b)
            m = self.mean[which]
            self.mean[which] = ms if m is None else m + self.weight * (ms - m)
            self.passes[which] += 1
        self.pending = keep

    def report(self) -> dict:
        self.poll()
        return {"in_use": self.winner(), "mean_ms": {k: (None if v is None else round(v, 4))
                                                      for k, v in self.mean.items()},
                "passes_timed": dict(self.passes)}


def _count_mlp_init(seed: int) -> np.ndarray:
    """FP32 weights of a cost MLP that starts out ordering tiles exactly by
    its feature 0 (a log count): hidden unit 0 passes it to the output, the
    other hidden units get random input weights but zero output weights, so
    they add nothing until training gives them a share (their output weights
    get gradient at once, their input weights from then on)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.zeros(MLP_W, np.float32)
    w[:256] = rng.normal(0, math.sqrt(2.0 / 8), 256)
    w[0:8] = 0.0
    w[0] = 1.0
    w[288] = 1.0
    w[320] = 10.0                      # log(ns) of a typical tile
    return w


class Frame:
    """Device buffers and calls for one batch of views of N Gaussians."""

    def __init__(self, cams, N: int, rgb_dtype: int = L.GS_F32, sh_dtype: int = L.GS_F32,
                 capacity: int | None = None, schedule: Schedule | None = None, device=None,
                 prefix: bool = False, defer_colour: bool = True):
        """prefix: bin with gs_bin_sort_prefix (exact list prefixes that blending
        never runs past) instead of the full lists of gs_bin_sort.
        defer_colour (with prefix): project without SH and colour only the
        records the kept lists reference (gs_colour_records), after binning
        and after a repair."""
        self.dev = device or _dev()
        self.prefix = prefix
        self.cams = list(cams)
        # (views of more than 16384 tiles get full lists, which reference every
        # visible record: nothing to defer)
        self.defer_colour = defer_colour and prefix and max(c.n_tiles for c in self.cams) <= 16384
        self.colour_src = None       # (means, sh) of the last projection whose colours are deferred
        self.colour_epoch = 0        # this step's mark of the records coloured
        self.V = len(self.cams)
        self.N = int(N)
        self.rgb_dtype = rgb_dtype
        self.sh_dtype = sh_dtype
        self.sched = schedule or Schedule()
        d = self.dev
        self.T = sum(c.n_tiles for c in self.cams)
        self.P = sum(c.W * c.H for c in self.cams)
        self.gcap = 0
        self._alloc_gaussians(self.N)
        self.err = torch.zeros(1, dtype=torch.int32, device=d)
        self.n_inst = torch.zeros(1, dtype=torch.int64, device=d)
        self.colour_count = torch.zeros(1, dtype=torch.int32, device=d)   # records the binning listed
        self.ranges = torch.empty(self.T * 2, dtype=torch.int32, device=d)
        self.tile_count = torch.zeros(self.T, dtype=torch.int32, device=d)
        self.img = torch.empty(3 * self.P, dtype=torch.float32, device=d)
        self.T_final = torch.empty(self.P, dtype=torch.float32, device=d)
        self.n_proc = torch.empty(self.P, dtype=torch.int32, device=d)
        self.tile_nproc = torch.full((self.T,), -1, dtype=torch.int32, device=d)   # -1: no history
        self.flag_tiles = torch.zeros(self.T, dtype=torch.int32, device=d)
        self.flag_count = torch.zeros(1, dtype=torch.int32, device=d)
        self.limit_history = True          # cut prefixes at 2x the last step's processed count
        self.tile_ns = torch.zeros(self.T, dtype=torch.int64, device=d)
        self.dimg = torch.empty(3 * self.P, dtype=torch.float32, device=d)
        self.loss = torch.zeros(1, dtype=torch.float32, device=d)
        self.capacity = 0
        self.inst_per_gaussian = 0.0
        self.vals = None
        self.keys = None
        self.ws = None
        if capacity is not None:
            self.reserve(capacity)
        # scheduler state
        self.queue = torch.zeros(1, dtype=torch.int32, device=d)
        self.split = torch.zeros(1, dtype=torch.int32, device=d)   # heavy tiles the reverse pass splits
        self.feats = torch.zeros(self.T * 8, dtype=torch.float32, device=d)
        self.cost = torch.zeros(self.T, dtype=torch.float32, device=d)
        self.order_f = torch.arange(self.T, dtype=torch.int32, device=d)
        self.order_b = torch.arange(self.T, dtype=torch.int32, device=d)
        self.order_ws = torch.empty(L.gs_sched_order_workspace(self.T) // 4 + 64,
                                    dtype=torch.float32, device=d)
        # learned mode: the cost MLP of the reverse pass predicts a tile's
        # reverse-pass time from what the forward left (gs_bwd_tile_features);
        # it starts as the order by processed count and trains on the reverse
        # pass's own tile times.  (A forward cost model, gs_tile_features,
        # exists in the library; the forward runs in raster order.)
        self.mlp = {}
        for k, seed in (("bwd", self.sched.seed + 1),):
            w32 = torch.from_numpy(_count_mlp_init(seed)).to(d)
            self.mlp[k] = dict(w32=w32, w16=w32.to(torch.float16),
                               m=torch.zeros(MLP_W, dtype=torch.float32, device=d),
                               v=torch.zeros(MLP_W, dtype=torch.float32, device=d),
                               g=torch.zeros(MLP_W, dtype=torch.float32, device=d),
                               loss=torch.zeros(1, dtype=torch.float32, device=d))
        self.mlp_t = 0
        self.pred = torch.zeros(self.T, dtype=torch.float32, device=d)
        self.feats_b = torch.zeros(self.T * 8, dtype=torch.float32, device=d)
        self.pred_b = torch.zeros(self.T, dtype=torch.float32, device=d)
        self.tile_ns_b = torch.zeros(self.T, dtype=torch.int64, device=d)
        # which order each pass uses: forced ("learned" / "count") or judged
        self.force_order = "learned" if self.sched.mode == "learned" and not self.sched.judge else None
        self.judge_b = PassJudge(self.sched.judge_every)
        self.pick_b = "count"
        # the forward of the learned schedule: raster order (one CTA per tile),
        # judged against the order of the previous step's processed counts,
        # computed at the start of the judged time
        self.judge_f = PassJudge(self.sched.judge_every, arms=("processed", "raster"))
        self.fwd_prep = None         # (pick, None): the forward's arm for this step
        self.cost_f = torch.zeros(self.T, dtype=torch.float32, device=d)
        self.step_count = 0
        # the error word, read back each step without waiting (pinned copy +
        # event): an instance-capacity overflow raises, never passes silently
        self.err_host = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.err_event = None
        # a second stream for work off the critical path of a training step
        # (zeroing the 2D gradients during the binning, the reverse pass's
        # order during the L1, the cost MLP's training during the fused
        # backward), joined back by events
        self.side = None
        self.ev_zeroed = None        # the 2D gradients zeroed on the side stream
        self.bwd_prep = None         # (timing, schedule, event): the reverse pass's order, prepared
        self.ev_mlp = None           # the cost MLP's training step queued on the side stream

    # -- buffers -----------------------------------------------------------
    def _alloc_gaussians(self, N: int) -> None:
        """Per-Gaussian buffers for up to N Gaussians in every view (non-empty
        even for N = 0); the kernels index them by the current N."""
        d = self.dev
        self.gcap = max(1, int(N))
        VN = self.V * self.gcap
        nb = L.SPLAT_BYTES[self.rgb_dtype]
        self.splats = torch.empty(VN * nb // 4, dtype=torch.float32, device=d)
        self.depth = torch.empty(VN, dtype=torch.float32, device=d)
        self.rect = torch.empty(VN * 4, dtype=torch.int16, device=d)
        self.touched = torch.empty(VN, dtype=torch.int32, device=d)
        self.radius = torch.empty(VN, dtype=torch.int32, device=d)
        self.grad2d = torch.empty(VN * 12, dtype=torch.float32, device=d)
        self.grad2d_zero = False     # whether the 2D-gradient records are known to be all zero
        if self.defer_colour:
            self.colour_mark = torch.zeros(VN, dtype=torch.int32, device=d)
            self.colour_list = torch.empty(VN, dtype=torch.int32, device=d)
        self.dparams = torch.empty(PARAM_FLOATS * self.gcap, dtype=torch.float32, device=d)

    def resize(self, N: int) -> None:
        """A new Gaussian count (after clone and prune).  Per-Gaussian buffers
        and the instance capacity (which grows in proportion to the count)
        are enlarged with 25% slack when they must grow and never shrunk; the
        binning workspace is checked against the new count.  Per-tile history
        (last processed counts, scheduler state) is kept: the prefix repair
        covers lists that grew past it."""
        N = int(N)
        if N == self.N:
            return
        if N > self.gcap:
            self._alloc_gaussians(N + N // 4)
        self.N = N
        self.grad2d_zero = False
        if self.vals is None:
            return
        need = int(self.inst_per_gaussian * N) + 65536
        if need > self.capacity:
            self.reserve(min(int(need * 1.25), 0xF0000000), with_keys=self.keys is not None)
        self._size_ws()

    def reserve(self, capacity: int, with_keys: bool = False) -> None:
        capacity = int(max(capacity, 1))
        if capacity <= self.capacity and (not with_keys or self.keys is not None):
            return
        self.capacity = max(capacity, self.capacity)
        self.vals = None                  # release before allocating the larger buffers
        self.keys = None
        self.ws = None
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=self.dev)
        self.keys = torch.empty(self.capacity, dtype=torch.int64, device=self.dev) if with_keys else None
        self._size_ws()

    def _size_ws(self) -> None:
        """Binning workspace for the current count and capacity (reallocated
        only when it must grow)."""
        if self.prefix:
            nbytes = L.gs_bin_sort_prefix_workspace(self.cams, self.N, self.capacity)
        else:
            nbytes = L.gs_bin_sort_workspace(self.cams, self.N, self.capacity)
        if self.ws is None or self.ws.numel() * 4 < nbytes + 256:
            self.ws = None
            self.ws = torch.empty(nbytes // 4 + 64, dtype=torch.float32, device=self.dev)

    # -- forward -----------------------------------------------------------
    def project(self, params: dict) -> None:
        defer = self.defer_colour
        self.colour_src = (params["means"], params["sh"]) if defer else None
        L.gs_project(self.cams, self.N, params["means"], params["log_scales"], params["quats"],
                     params["opacity_logits"], None if defer else params["sh"], self.sh_dtype, self.splats,
                     self.rgb_dtype, self.depth, self.rect, self.touched, self.radius, self.err)

    def colour_kept(self) -> None:
        """The deferred colours of the records the kept lists reference (after
        bin_sort with colour=False)."""
        if self.colour_src is None:
            return
        means, sh = self.colour_src
        L.gs_colour_records(self.cams, self.N, means, sh, self.sh_dtype, self.colour_list, self.colour_count,
                            self.splats, self.rgb_dtype)

    def _colour_repaired(self) -> None:
        """The deferred colours of the records only the repaired lists reference."""
        if self.colour_src is None:
            return
        means, sh = self.colour_src
        L.gs_colour_repaired(self.cams, self.N, means, sh, self.sh_dtype, self.vals, self.capacity,
                             self.flag_tiles, self.flag_count, self.ranges, self.colour_mark, self.colour_epoch,
                             self.splats, self.rgb_dtype)

    def _bin(self, capacity: int, keys) -> None:
        if self.prefix:
            lim = self.tile_nproc if self.limit_history else None
            col = self.colour_src is not None and capacity > 0
            if col:
                self.colour_epoch += 1
            L.gs_bin_sort_prefix(self.cams, self.N, self.depth, self.rect, self.touched, self.splats,
                                 self.rgb_dtype, lim, capacity, self.vals, self.ranges, self.tile_count,
                                 keys, self.n_inst, self.ws, self.err,
                                 colour_list=self.colour_list if col else None,
                                 colour_count=self.colour_count if col else None,
                                 colour_mark=self.colour_mark if col else None, colour_epoch=self.colour_epoch)
        else:
            L.gs_bin_sort(self.cams, self.N, self.depth, self.rect, self.touched, capacity, self.vals,
                          self.ranges, keys, self.n_inst, self.ws, self.err)

    def _watch_errors(self, issue: bool) -> None:
        """Check the error word read back after the previous step's render,
        and (issue=True) start the read-back of this step's.  A capacity
        overflow there means that step rendered cut lists: raise rather than
        train on them."""
        if self.err_event is not None and self.err_event.query():
            bits = int(self.err_host.item())
            self.err_event = None
            if bits & L.GS_EW_CAPACITY:
                raise L.GsError(f"instance capacity {self.capacity} was exceeded (error word {bits:#x}): "
                                "the lists of that step were cut; reserve() a larger capacity")
        if issue and self.err_event is None:
            self.err_host.copy_(self.err, non_blocking=True)
            self.err_event = torch.cuda.Event()
            self.err_event.record()

    def bin_sort(self, want_keys: bool = False, colour: bool = True) -> None:
        """Bin and sort; colour: then the deferred colours of the kept records
        (else the caller calls colour_kept())."""
        self._watch_errors(issue=False)
        if self.vals is None:
            # first call: size the instance buffers from the exact count
            self.reserve(1)
            self._bin(0, None)
            need = int(self.n_inst.item())
            if self.prefix:          # room for repairs: the full lists
                need = max(need, int(self.tile_count.sum().item()))
            self.inst_per_gaussian = need / max(1, self.N)     # scales the capacity when the count changes
            self.reserve(int(need * 1.25) + 65536, with_keys=want_keys)
            self.err.bitwise_and_(~L.GS_EW_CAPACITY)      # the sizing pass overflowed on purpose
        elif want_keys and self.keys is None:
            self.reserve(self.capacity, with_keys=True)
        self._bin(self.capacity, self.keys if want_keys else None)
        if colour:
            self.colour_kept()

    @property
    def use_learned(self) -> bool:
        """Whether the reverse pass uses the learned order (forced, or
        winning its judge)."""
        if self.force_order is not None:
            return self.force_order == "learned"
        return self.judge_b.winner() == "learned"

    @use_learned.setter
    def use_learned(self, on: bool) -> None:
        self.force_order = "learned" if on else "count"

    def _pick(self, judge: PassJudge) -> str:
        return self.force_order if self.force_order is not None else judge.pick()

    def _count_order(self, out: torch.Tensor) -> None:
        L.gs_range_cost(self.ranges, self.T, self.cost)
        L.gs_sched_order(self.cost, self.T, out, self.order_ws)

    def _sched_fwd(self, pick=None):
        """The forward's schedule: None (raster) for the raster schedule, the
        instance-count order for the plain one; for the learned one raster,
        or, when its judge picked it, the order of the processed counts the
        previous forward left (computed here, inside the judged time)."""
        if self.sched.mode == "learned":
            if pick != "processed":
                return None
            L.gs_int_cost(self.tile_nproc, self.T, self.cost_f)
            L.gs_sched_order(self.cost_f, self.T, self.order_f, self.order_ws)
            return {"mode": L.GS_SCHED_ORDER, "order": self.order_f, "queue": self.queue}
        if self.sched.mode != "count":
            return None
        self._count_order(self.order_f)
        return {"mode": L.GS_SCHED_ORDER, "order": self.order_f, "queue": self.queue}

    def _sched_bwd(self, timing: bool = False):
        """The reverse pass's order.  The plain schedule reuses the forward's
        order (bwd_order 'forward') or orders tiles by the entries the
        forward processed ('processed'); the learned schedule orders them by
        the reverse-pass MLP's prediction (and splits the tiles it predicts
        heavy) or, when its judge says so, by instance count.  timing:
        measure the reverse pass's tile times (self.tile_ns_b)."""
        if self.sched.mode == "raster":
            return None
        if self.ev_mlp is not None:          # the cost MLP's training reads the buffers refilled below
            torch.cuda.current_stream().wait_event(self.ev_mlp)
            self.ev_mlp = None
        base = {"queue": self.queue, "split": self.split, "mode": L.GS_SCHED_ORDER}
        if timing:
            L.gs_zero(self.tile_ns_b)
            base["tile_ns"] = self.tile_ns_b
        if self.sched.mode == "learned":
            self.pick_b = self._pick(self.judge_b)
            if self.pick_b == "learned" or timing:
                L.gs_bwd_tile_features(self.cams, self.ranges, self.tile_nproc, self.n_proc, self.tile_ns,
                                       self.feats_b, self.mlp["bwd"]["w16"], self.pred_b)
            if self.pick_b == "learned":
                L.gs_sched_order(self.pred_b, self.T, self.order_b, self.order_ws)
                return dict(base, order=self.order_b, split_cost=self.pred_b)
            self._count_order(self.order_b)
            return dict(base, order=self.order_b)
        self.pick_b = "count"
        if self.sched.bwd_order == "forward":
            return dict(base, order=self.order_f)
        L.gs_int_cost(self.tile_nproc, self.T, self.cost)
        L.gs_sched_order(self.cost, self.T, self.order_b, self.order_ws)
        return dict(base, order=self.order_b)

    # -- side stream ---------------------------------------------------------
    def _fork(self):
        """The side stream, ordered after everything queued so far on the
        current stream."""
        if self.side is None:
            self.side = torch.cuda.Stream(device=self.dev)
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream())
        self.side.wait_event(ev)
        return self.side

    @staticmethod
    def _recorded(stream):
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    def zero_grad2d_async(self) -> None:
        """Zero the 2D gradients on the side stream (after every reader queued
        so far); render_bwd waits for it instead of zeroing itself.  Nothing
        to do when the last consumer left them all zero (the fused one-view
        backward + Adam does)."""
        if self.grad2d_zero:
            self.ev_zeroed = None
            return
        s = self._fork()
        with torch.cuda.stream(s):
            L.gs_zero(self.grad2d[:self.V * self.N * 12])
        self.ev_zeroed = self._recorded(s)

    def prepare_bwd_async(self, timing: bool = False) -> None:
        """The reverse pass's order (features, cost MLP, order) on the side
        stream, after the forward queued so far and overlapping what the
        current stream does next (the L1); render_bwd with the same timing
        waits for it and uses it."""
        s = self._fork()
        with torch.cuda.stream(s):
            sched = self._sched_bwd(timing=timing)
        self.bwd_prep = (timing, sched, self._recorded(s))

    def prepare_fwd_async(self) -> None:
        """The learned schedule's forward order for this step: its judge picks
        raster or the previous step's processed-count order.  The order is
        computed when the forward starts, inside the time the judge measures,
        so that its cost counts against it (computed on the side stream
        during the binning, it slowed the binning by as much as it saved)."""
        if self.sched.mode != "learned" or self.force_order is not None:
            self.fwd_prep = None
            return
        self.fwd_prep = (self.judge_f.pick(), None)

    def train_scheduler_async(self) -> None:
        """train_scheduler on the side stream, overlapping what the current
        stream does next; the next reverse-pass order waits for it."""
        s = self._fork()
        with torch.cuda.stream(s):
            self.train_scheduler()
        self.ev_mlp = self._recorded(s)

    def render(self, timing: bool = False, mark=None) -> None:
        pick = self.fwd_prep[0] if self.fwd_prep is not None else None
        self.fwd_prep = None
        tok = self.judge_f.start(pick) if pick is not None else None     # the order's cost included
        s = self._sched_fwd(pick)
        if mark:
            mark("render_fwd")
        tns = self.tile_ns if timing else None
        if not self.prefix:
            L.gs_render_fwd(self.cams, self.ranges, self.vals, self.splats, self.rgb_dtype, s, self.img,
                            self.T_final, self.n_proc, self.tile_nproc, tns, self.err)
            if tok:
                self.judge_f.stop(tok)
            return
        # kept prefixes: check that no pixel ran past one, rebuild and re-render any that did
        L.gs_zero(self.flag_count)
        L.gs_render_fwd(self.cams, self.ranges, self.vals, self.splats, self.rgb_dtype, s, self.img,
                        self.T_final, self.n_proc, self.tile_nproc, tns, self.err,
                        tile_count=self.tile_count, flag_tiles=self.flag_tiles, flag_count=self.flag_count)
        if tok:
            self.judge_f.stop(tok)
        L.gs_bin_sort_prefix_repair(self.cams, self.N, self.rect, self.touched, self.flag_tiles,
                                    self.flag_count, self.capacity, self.vals, self.ranges, self.n_inst,
                                    self.ws, self.err)
        self._colour_repaired()
        rep = {"mode": L.GS_SCHED_ORDER, "order": self.flag_tiles, "queue": self.queue,
               "n_order": self.flag_count}
        L.gs_render_fwd(self.cams, self.ranges, self.vals, self.splats, self.rgb_dtype, rep, self.img,
                        self.T_final, self.n_proc, self.tile_nproc, tns, self.err)
        self._watch_errors(issue=True)

    def render_merged(self) -> torch.Tensor:
        """Forward render with similarity-based sampling and merging of the
        current tile lists (Sec. IV-C1; lossy, forward only): gs_colour_merge
        keeps one representative per (tile, colour bucket), then
        gs_render_fwd blends the merged lists into self.img (T_final and
        n_proc are overwritten; the per-tile history is not)."""
        cap = self.vals.numel()
        if getattr(self, "merge_cap", 0) < cap:
            self.m_ranges = torch.empty(self.T * 2, dtype=torch.int32, device=self.dev)
            self.m_vals = torch.empty(cap, dtype=torch.int32, device=self.dev)
            self.m_splats = torch.empty(cap * L.SPLAT_BYTES[L.GS_F32] // 4, dtype=torch.float32, device=self.dev)
            self.m_tile_nproc = torch.empty(self.T, dtype=torch.int32, device=self.dev)
            self.merge_cap = cap
        L.gs_colour_merge(self.T, self.ranges, self.vals, self.splats, self.rgb_dtype, self.m_ranges, self.m_vals,
                          self.m_splats)
        L.gs_render_fwd(self.cams, self.m_ranges, self.m_vals, self.m_splats, L.GS_F32, None, self.img,
                        self.T_final, self.n_proc, self.m_tile_nproc, None, self.err)
        return self.img

    def forward(self, params: dict, timing: bool = False) -> torch.Tensor:
        self.project(params)
        self.bin_sort()
        self.render(timing=timing)
        return self.img

    # -- backward ----------------------------------------------------------
    def render_bwd(self, dimg: torch.Tensor, timing: bool = False, mark=None) -> None:
        """The reverse pass into self.grad2d (zeroed first) in the schedule's
        order; timing: also measure its per-tile times (self.tile_ns_b)."""
        cur = torch.cuda.current_stream()
        if self.ev_zeroed is not None:
            cur.wait_event(self.ev_zeroed)
            self.ev_zeroed = None
        elif not self.grad2d_zero:
            L.gs_zero(self.grad2d[:self.V * self.N * 12])
        self.grad2d_zero = False                 # the reverse pass adds into the records
        judged = self.sched.mode == "learned" and self.force_order is None
        if self.bwd_prep is not None and self.bwd_prep[0] == timing:
            # the judged time includes the wait for the order the side stream
            # prepared (the learned order's features and MLP cost more than
            # the count order's ranking)
            tok = self.judge_b.start(self.pick_b) if judged else None
            s = self.bwd_prep[1]
            cur.wait_event(self.bwd_prep[2])
        else:
            s = self._sched_bwd(timing=timing)
            tok = self.judge_b.start(self.pick_b) if judged else None
        self.bwd_prep = None
        if mark:
            mark("render_bwd")
        L.gs_render_bwd(self.cams, self.ranges, self.vals, self.splats, self.rgb_dtype, s, dimg,
                        self.T_final, self.n_proc, self.tile_nproc, self.grad2d, self.err)
        if tok:
            self.judge_b.stop(tok)

    def backward(self, params: dict, dimg: torch.Tensor, mark=None) -> torch.Tensor:
        self.render_bwd(dimg, mark=mark)
        if mark:
            mark("project_bwd")
        L.gs_project_bwd(self.cams, self.N, params["means"], params["log_scales"], params["quats"],
                         params["opacity_logits"], params["sh"], self.sh_dtype, self.touched,
                         self.grad2d, self.dparams)
        return self.dparams

    def l1(self, target: torch.Tensor) -> torch.Tensor:
        if target.numel() != 3 * self.P or target.dtype != torch.float32 or not target.is_cuda:
            raise ValueError(f"L1 target must be a float32 CUDA tensor of 3 x {self.P} values "
                             f"(every view's pixels), got {tuple(target.shape)} {target.dtype}")
        L.gs_l1_loss(3 * self.P, self.img, target, self.loss, self.dimg)
        return self.loss

    # -- scheduler training ------------------------------------------------
    def train_scheduler(self) -> None:
        """One training step of the reverse pass's cost MLP on the tile times
        of the last timed reverse pass (self.tile_ns_b) and the features
        computed for it."""
        if self.sched.mode != "learned":
            return
        self.mlp_t += 1
        m = self.mlp["bwd"]
        if self.mlp_t == 1:
            self._fit_line(m)
        L.gs_mlp_train_step(m["w32"], m["w16"], m["m"], m["v"], self.mlp_t, self.sched.mlp_lr, self.feats_b,
                            self.tile_ns_b, None, self.T, m["g"], m["loss"])

    def _fit_line(self, m: dict) -> None:
        """Once, before the first training step: set the MLP's output to the
        least-squares line of log(reverse-pass tile time) on its feature 0
        (log1p of the processed count), fitted on the tile times just
        measured (one read-back).  The MLP then starts as the processed-count
        order at the right scale, and training refines it instead of first
        spending its steps on the offset."""
        f0 = self.feats_b.view(-1, 8)[:, 0].cpu().numpy().astype(np.float64)
        ns = self.tile_ns_b.cpu().numpy().astype(np.float64)
        live = ns > 0
        if live.sum() < 2 or np.ptp(f0[live]) <= 0:
            return
        a, b = np.polyfit(f0[live], np.log(ns[live]), 1)
        if not (a > 0 and np.isfinite(a) and np.isfinite(b)):
            return
        w = m["w32"].cpu().numpy()
        w[288] = a                     # hidden unit 0 passes feature 0 with weight 1
        w[320] = b
        m["w32"].copy_(torch.from_numpy(w))
        m["w16"].copy_(torch.from_numpy(w.astype(np.float16)))

    def schedule_report(self) -> dict:
        """The orders in use and the measured pass durations behind them."""
        if self.sched.mode != "learned":
            return {"forward": self.sched.mode, "backward": self.sched.mode}
        if self.force_order is not None:
            return {"forward": "raster", "backward": self.force_order, "judged": False}
        return {"forward": self.judge_f.report(), "backward": self.judge_b.report(), "judged": True}

    def check_errors(self) -> int:
        return int(self.err.item())

    # -- views ---------------------------------------------------------------
    def image(self, v: int = 0) -> torch.Tensor:
        base = sum(c.W * c.H for c in self.cams[:v])
        c = self.cams[v]
        return self.img[3 * base:3 * (base + c.W * c.H)].view(3, c.H, c.W)

    def pixel_map(self, buf: torch.Tensor, v: int = 0) -> torch.Tensor:
        base = sum(c.W * c.H for c in self.cams[:v])
        c = self.cams[v]
        return buf[base:base + c.W * c.H].view(c.H, c.W)


class Trainer:
    """Full training step: forward, L1 against targets, backward, Adam."""

    def __init__(self, cams, params_flat: torch.Tensor, N: int, targets: torch.Tensor,
                 rgb_dtype: int = L.GS_F32, sh_storage: int = L.GS_F32,
                 schedule: Schedule | None = None, lr=DEFAULT_LR, prefix: bool = True,
                 defer_colour: bool = True):
        """defer_colour: colour only the records the kept lists reference (see
        Frame); off where repairs are frequent, since a repaired full list's
        records are coloured one by one."""
        self.N = N
        self.p = params_flat
        self.m = torch.zeros_like(params_flat)
        self.v = torch.zeros_like(params_flat)
        self.lr = lr
        self.t = 0
        self.sh_storage = sh_storage
        self.views = param_views(self.p, N)
        if sh_storage != L.GS_F32:
            dt = torch.bfloat16 if sh_storage == L.GS_BF16 else torch.float16
            self.sh_shadow = self.views["sh"].to(dt)
        else:
            self.sh_shadow = None
        self.frame = Frame(cams, N, rgb_dtype=rgb_dtype, sh_dtype=sh_storage, schedule=schedule,
                           device=params_flat.device, prefix=prefix, defer_colour=defer_colour)
        if targets.numel() != 3 * self.frame.P:
            raise ValueError(f"targets must hold 3 x {self.frame.P} values (every view's pixels, "
                             f"view after view), got {targets.numel()}")
        self.targets = targets
        self.grad_norm = None             # screen-space gradient statistic, when tracked

    def track_screen_grad(self, on: bool = True) -> None:
        """Accumulate, every step, each Gaussian's screen-space gradient norm
        summed over views (the statistic densify() clones by)."""
        self.grad_norm = torch.zeros(max(1, self.N), dtype=torch.float32, device=self.p.device) if on else None

    def densify(self, clone_frac: float = 0.02, min_opacity: float = 0.005) -> int:
        """One clone-and-prune step between training steps (adaptive density
        control of 3DGS training in its plain form, Sec. II-A): drop the
        Gaussians with opacity below min_opacity, clone the
        floor(clone_frac N) kept ones with the largest accumulated
        screen-space gradient (trimmed or padded to a multiple of 4; see
        gs_densify), clones starting with zero Adam moments.  Parameters,
        moments, the 16-bit SH shadow and the frame's buffers move to the new
        count, which is read back (4 bytes) and returned; the statistic
        restarts from zero."""
        n_clone = int(clone_frac * self.N)
        thr = float(np.float32(math.log(min_opacity / (1.0 - min_opacity))))
        cap = self.N + n_clone + 3
        dev = self.p.device
        p2 = torch.empty(PARAM_FLOATS * cap, dtype=torch.float32, device=dev)
        m2 = torch.empty_like(p2)
        v2 = torch.empty_like(p2)
        sh2 = None
        if self.sh_shadow is not None:
            sh2 = torch.empty(48 * cap, dtype=self.sh_shadow.dtype, device=dev)
        gn = self.grad_norm if self.grad_norm is not None else torch.zeros(max(1, self.N), device=dev)
        ws = torch.empty(L.gs_densify_workspace(self.N) // 4 + 64, dtype=torch.float32, device=dev)
        n_out = torch.zeros(1, dtype=torch.int32, device=dev)
        f = self.frame
        L.gs_densify(self.N, self.p, self.m, self.v, gn, thr, n_clone, cap, p2, m2, v2, sh2, self.sh_storage,
                     n_out, ws, f.err)
        n2 = int(n_out.item())
        if f.check_errors():
            raise L.GsError(f"gs_densify reported error bits {f.check_errors():#x}")
        if f.vals is not None and self.N > 0:
            # instances per Gaussian of the latest binning (full lists), which
            # resize() scales the instance capacity by
            need = int(f.tile_count.sum().item()) if f.prefix else int(f.n_inst.item())
            f.inst_per_gaussian = need / self.N
        self.N = n2
        self.p = p2[:PARAM_FLOATS * n2]
        self.m = m2[:PARAM_FLOATS * n2]
        self.v = v2[:PARAM_FLOATS * n2]
        self.views = param_views(self.p, n2)
        if sh2 is not None:
            self.sh_shadow = sh2[:48 * n2]
        f.resize(n2)
        if self.grad_norm is not None:
            self.track_screen_grad(True)
        return n2

    def params_for_kernels(self) -> dict:
        d = dict(self.views)
        if self.sh_shadow is not None:
            d["sh"] = self.sh_shadow
        return d

    def iteration(self, targets: torch.Tensor | None = None, mark=None) -> torch.Tensor:
        """One fwd+bwd iteration: the step without Adam.  Projection, binning,
        schedule, forward, L1, reverse pass, projection backward to the 59
        parameter gradients (in frame.dparams), and the cost models' training
        step every train_every-th iteration."""
        return self.step(mark=mark, targets=targets, adam=False)

    def step(self, mark=None, targets: torch.Tensor | None = None, adam: bool = True,
             targets_ready=None) -> torch.Tensor:
        """One training step (adam=False: without the parameter update, see
        iteration()).  `mark(name)`, if given, is called before each stage
        (and with "end" after the last) so a caller can time stages.
        targets_ready: a CUDA event the L1 waits for (e.g. the end of the
        targets' copy from the host on another stream, which then overlaps
        the projection, binning and forward)."""
        mk = mark or (lambda name: None)
        f = self.frame
        pk = self.params_for_kernels()
        timing = f.sched.mode == "learned"
        train_now = timing and (f.step_count % max(1, f.sched.train_every) == 0)
        f.prepare_fwd_async()                  # the forward's order, if judged, overlaps the projection
        mk("project")
        f.project(pk)
        f.zero_grad2d_async()                  # overlaps the binning (latency-bound, SM slots to spare)
        mk("bin_sort")
        f.bin_sort(colour=False)
        mk("colour")
        f.colour_kept()
        mk("sched_fwd")
        f.render(timing=timing, mark=mark)
        f.prepare_bwd_async(timing=train_now)  # overlaps the L1
        mk("l1")
        if targets_ready is not None:
            torch.cuda.current_stream().wait_event(targets_ready)
        f.l1(self.targets if targets is None else targets)
        mk("sched_bwd")
        f.render_bwd(f.dimg, timing=train_now, mark=mark)
        if train_now:
            f.train_scheduler_async()          # overlaps the fused backward
        if self.grad_norm is not None:
            mk("grad_stat")
            L.gs_grad2d_norm(len(f.cams), self.N, f.grad2d, self.grad_norm)
        pk_sh = self.sh_shadow if self.sh_shadow is not None else pk["sh"]
        if not adam:
            mk("project_bwd")
            L.gs_project_bwd(f.cams, self.N, pk["means"], pk["log_scales"], pk["quats"], pk["opacity_logits"],
                             pk_sh, self.sh_storage, f.touched, f.grad2d, f.dparams)
        elif len(f.cams) == 1:
            # one view: the projection backward and Adam in one streaming pass
            # (the per-Gaussian gradients never go to memory)
            self.t += 1
            mk("project_bwd_adam")
            L.gs_project_bwd_adam(f.cams, self.N, self.p, self.sh_shadow, self.sh_storage, f.touched, f.grad2d,
                                  self.m, self.v, self.lr, ADAM_B1, ADAM_B2, ADAM_EPS, self.t,
                                  self.sh_shadow, self.sh_storage)
            f.grad2d_zero = True                 # the call leaves the records all zero
        else:
            # several views: gradients summed over views, then Adam
            self.t += 1
            mk("project_bwd")
            L.gs_project_bwd(f.cams, self.N, pk["means"], pk["log_scales"], pk["quats"], pk["opacity_logits"],
                             pk_sh, self.sh_storage, f.touched, f.grad2d, f.dparams)
            mk("adam")
            L.gs_adam_step(self.N, self.p, f.dparams, self.m, self.v, self.lr, ADAM_B1, ADAM_B2, ADAM_EPS,
                           self.t, self.sh_shadow, self.sh_storage)
        mk("end")
        f.step_count += 1
        return f.loss


class RasterizeGaussians(torch.autograd.Function):
    """image = render(means, log_scales, quats, opacity_logits, sh) for one
    view; backward through the hand-written reverse-mode kernels."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cam, rgb_dtype=L.GS_F32):
        N = means.shape[0]
        fr = Frame([cam], N, rgb_dtype=rgb_dtype, sh_dtype=_sh_dtype(sh), device=means.device)
        params = {"means": means.contiguous(), "log_scales": log_scales.contiguous(),
                  "quats": quats.contiguous(), "opacity_logits": opacity_logits.contiguous(),
                  "sh": sh.contiguous()}
        fr.forward(params)
        ctx.frame = fr
        ctx.params = params
        ctx.sh_float = sh.dtype
        return fr.image(0).clone()

    @staticmethod
    def backward(ctx, grad_img):
        fr = ctx.frame
        g = fr.backward(ctx.params, grad_img.contiguous().view(-1))
        N = fr.N
        v = param_views(g, N)
        return (v["means"].view(N, 3).clone(), v["log_scales"].view(N, 3).clone(),
                v["quats"].view(N, 4).clone(), v["opacity_logits"].view(N).clone(),
                v["sh"].view(N, 16, 3).to(ctx.sh_float), None, None)


def _sh_dtype(sh: torch.Tensor) -> int:
    if sh.dtype == torch.float32:
        return L.GS_F32
    if sh.dtype == torch.bfloat16:
        return L.GS_BF16
    if sh.dtype == torch.float16:
        return L.GS_F16
    raise L.GsError(f"unsupported SH dtype {sh.dtype}")

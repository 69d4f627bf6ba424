#!/usr/bin/env python3
"""Throughput of the 3DGS training hot path on GB300.

One step = one pass of the whole hot path over one view: projection + SH
colour, tile binning and sort, the schedule (tile features, MLP prediction,
work order), forward blending, L1 loss, backward blending, projection
backward, Adam, and one training step of the tile-cost MLP.

Workload: 3M Gaussians, 80% in 20 tight clusters (sigma 0.02) and 20%
uniform in [-1,1]^3, one 1600x1060 view, L1 against a seeded image.  The
headline `value` is iterations/s of the learned-schedule path with SH and
colours stored in BF16; the plain FP32 count-ordered path is measured on the
same box and reported beside it.

Prints one JSON line.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd splat iters/s @3M Gaussians 1600x1060, learned vs plain schedule; %HBM"
WORKLOAD = "skewed-3M-1600x1060"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}

# DRAM bytes (read + write) per Gaussian of the dominant call, from one ncu
# capture of the full-size workload in the configuration the bench times
# (one view: FP32 SH, no 16-bit shadow; the summary of that capture is kept
# with the profiles).  Valid only while the kernel sources hash as they did
# when captured.
MEASURED_TRAFFIC = {
    "project_bwd_adam": {
        "bytes_per_gaussian": (0.558744576 + 0.338226944 + 1.872152320 + 1.666972416) * 1e9 / 3e6,
        "sources": {
            "paper_2510_14564_gb300/csrc/project.cu":
                "8821ff4c7b336f1479fe6dab051ac7ff5b4c229375965d7f86c937917166570a",
            "paper_2510_14564_gb300/csrc/gs_common.cuh":
                "48ec94c1bce3261c8aa6f96a82c366ec0c9b5ffa9490f3f62cec3ebaa685e270",
        },
    },
}


def measured_traffic(stage: str, N: int):
    """Captured DRAM traffic of `stage` scaled to N Gaussians, or None if
    there is no capture or a kernel source changed since it was taken."""
    import hashlib
    rec = MEASURED_TRAFFIC.get(stage)
    if rec is None:
        return None
    for rel, digest in rec["sources"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return int(rec["bytes_per_gaussian"] * N)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        try:
            rows = open(self.path).read().strip().splitlines()
        except OSError:
            rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            c = [x.strip() for x in r.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx = float(c[2])
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# replicas (one process per GPU): time = the slowest rank's, value = the
# steps all ranks ran over that time
# ---------------------------------------------------------------------------
def max_over_ranks(ms: float, world: int, device) -> float:
    """The largest of the ranks' times (every rank gets it)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps: int, ms_max: float, world: int) -> float:
    """Steps per second of the whole job: every rank ran `steps` steps, the
    job took the slowest rank's time."""
    return world * steps / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def algorithmic_bytes(N, P, I, I_proc, half: bool, V: int = 1, n_grad: int = 0,
                      sh_half: bool | None = None, n_col: int | None = None) -> dict:
    """Minimum bytes each stage must move (per step) for N Gaussians seen
    from V views with P pixels in all, n_grad of them with a 2D gradient;
    half: 16-bit colour records, sh_half: 16-bit SH storage (default: half);
    n_col: the records whose colour is deferred to the colour stage (None:
    the projection colours every record)."""
    if sh_half is None:
        sh_half = half
    rec = 34 if half else 40            # id + xy + conic + opacity + rgb per processed instance
    sh_read = 140 if sh_half else 236
    sh_b = 96 if sh_half else 192
    out = {
        "project": V * N * ((44 if n_col is not None else sh_read) + (46 if half else 52)),
        "bin_sort": V * N * 8 + I * (12 + 24 + 8),
        "render_fwd": I_proc * rec + P * 20,
        "l1": P * 36,
        "render_bwd": I_proc * rec + P * 20 + V * N * 36,
        "project_bwd": N * (sh_read + 32 + 236) + V * N * 36,
        "adam": N * (1652 + (96 if sh_half else 0)),
        # fused, one view, two launches.  Geometry: 11 params, touched, the 2D
        # gradient record, m and v of the 11; writes p, m, v of the 11.  SH:
        # the SH-gradient factors (24 bytes of the record), p, m and v of the
        # 48 SH entries read and written (+ the 16-bit shadow).  A Gaussian
        # with a 2D gradient (n_grad of them) also has its SH read by the
        # geometry kernel and its record written twice: the factors over it
        # (48 bytes), then zeros (24); the others' gradients are zero.
        "project_bwd_adam": N * ((44 + 4 + 48 + 88 + 132) + (24 + 576 + 576 + (96 if sh_half else 0)))
                            + n_grad * ((96 if sh_half else 192) + 48 + 24),
    }
    if n_col is not None:
        # the listed records: index, mean and SH read, colour written
        out["colour"] = n_col * (4 + 12 + sh_b + (8 if half else 12))
    return out


# Warp instructions the reverse pass issues per (pixel, Gaussian) pair its
# pixels walk, from one ncu capture of the full-size workload
# (smsp__inst_executed.sum of k_render_bwd over the sum of the per-pixel
# processed counts).  Valid only while the kernel sources hash as captured.
RENDER_BWD_INSTR = {
    "warp_instr_per_pair": 339131212 / 306789136,
    "sources": {
        "paper_2510_14564_gb300/csrc/render.cu": "db548d8484e4c08ba09f4f09652b36166792a331993a4a6b5523a6acf7395b17",
        "paper_2510_14564_gb300/csrc/gs_common.cuh": "48ec94c1bce3261c8aa6f96a82c366ec0c9b5ffa9490f3f62cec3ebaa685e270",
    },
}


def issue_roofline(pairs: int, ms: float | None, sm_count: int, clock_hz: float) -> dict | None:
    """The reverse pass against its issue roofline: the time its measured
    warp instructions per pair would take at the peak issue rate (4 warp
    instructions per SM per cycle, i.e. 128 thread instructions), over the
    measured time."""
    import hashlib
    w = RENDER_BWD_INSTR.get("warp_instr_per_pair")
    if not ms or not w:
        return None
    for path, digest in RENDER_BWD_INSTR["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != digest:
                return None
    instr = w * pairs
    t_min = instr / (sm_count * 4 * clock_hz)
    return {"bound": "issue", "pairs": pairs, "warp_instr_per_pair": w,
            "achieved": round(instr / (ms / 1e3) / 1e12, 4), "peak": round(sm_count * 4 * clock_hz / 1e12, 4),
            "unit": "T warp-instr/s", "frac": round(t_min / (ms / 1e3), 4),
            "issue_roofline_ms": round(t_min * 1e3, 4), "measured_ms": round(ms, 4)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import pipeline as P
    from paper_2510_14564_gb300 import scenes as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    L.lib()

    scene, cams = S.make_workload(args.workload, seed=0)
    cam = cams[0]
    N = scene.n
    # one target image per view, concatenated (the L1 runs over every view's pixels)
    tgt_host = torch.from_numpy(np.concatenate([S.random_image(c.W, c.H, seed=1 + v).ravel()
                                                for v, c in enumerate(cams)])).pin_memory()
    tgt = tgt_host.cuda()
    tgt_bufs = [torch.empty_like(tgt), torch.empty_like(tgt)]      # the e2e steps' targets, in turn
    cs = torch.cuda.Stream()                                        # their host-to-device copies
    flat0 = torch.from_numpy(scene.flat())

    # Learning rates scaled by --lr-scale: every step runs the full Adam update
    # (its work does not depend on the rates), while the scene -- and with it
    # the workload -- stays the configured one over the hundreds of steps the
    # bench runs (at full rates, L1 against a random target grows the
    # Gaussians step after step).
    lr = tuple(x * args.lr_scale for x in P.DEFAULT_LR)

    # SH storage of the learned path: a 16-bit shadow halves the projection's
    # SH read of every (view, Gaussian) but costs a write of it per step; with
    # one view the fused backward + Adam reads SH only for the Gaussians with a
    # gradient, so FP32 SH (no shadow) is the faster step there, while several
    # views read SH once per view and in the backward, and the shadow pays.
    learned_sh = L.GS_BF16 if len(cams) > 1 else L.GS_F32

    def make(mode, half):
        dt = L.GS_BF16 if half else L.GS_F32
        tr = P.Trainer(cams, flat0.cuda(), N, tgt, rgb_dtype=dt, sh_storage=learned_sh if half else L.GS_F32,
                       schedule=P.Schedule(mode=mode), lr=lr)
        return tr

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(tr, steps, stage_times=None, e2e=False, profile=False, adam=True):
        st = torch.cuda.current_stream()
        marks = []

        def mark(name):
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            marks.append((name, e))

        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        barrier()
        torch.cuda.synchronize()
        l0 = L.gs_launch_count()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        if profile:                     # a profiler started with --profile-from-start off sees only this
            torch.cuda.profiler.start()
        t0.record(st)
        if e2e:
            # each step's targets come from pinned host memory on a copy
            # stream (two device buffers in turn), overlapping the step's
            # projection, binning and forward; the L1 waits for its copy
            cs.wait_event(t0)
            freed = [None, None]
        for k in range(steps):
            ready = None
            if e2e:
                buf = tgt_bufs[k % 2]
                if freed[k % 2] is not None:
                    cs.wait_event(freed[k % 2])
                with torch.cuda.stream(cs):
                    buf.copy_(tgt_host, non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(cs)
            tr.step(mark=mark if stage_times is not None else None, adam=adam,
                    targets=buf if e2e else None, targets_ready=ready)
            if e2e:
                freed[k % 2] = torch.cuda.Event()
                freed[k % 2].record(st)
                loss_host.copy_(tr.frame.loss, non_blocking=True)
        t1.record(st)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        launches = L.gs_launch_count() - l0
        barrier()
        ms = max_over_ranks(t0.elapsed_time(t1), world, "cuda")
        if stage_times is not None:
            for (n0, e0), (_, e1) in zip(marks[:-1], marks[1:]):
                if n0 != "end":
                    stage_times.setdefault(n0, []).append(e0.elapsed_time(e1))
        return ms, launches

    # plain FP32 path, tile order by instance count: the training step, then
    # the fwd+bwd iteration (no Adam).  Its steps follow the learned path's
    # sequence (calibration + warm-up, timed steps, the end-to-end steps,
    # the iterations), so that at real learning rates, where the scene
    # changes from step to step, both paths are timed on the same steps of
    # the same training run.
    plain = make("count", False)
    for _ in range(args.calib + args.warmup):
        plain.step()
    plain_stages = {}
    plain_ms, _ = timed(plain, args.steps, stage_times=plain_stages)
    plain_ips = replica_throughput(args.steps, plain_ms, 1)
    for _ in range(args.steps):             # where the learned path runs its end-to-end steps
        plain.step()
    for _ in range(3):
        plain.iteration()
    plain_it_ms, _ = timed(plain, args.steps, adam=False)
    plain_it_ips = replica_throughput(args.steps, plain_it_ms, 1)
    assert plain.frame.check_errors() == 0, "kernel error word set (plain path)"
    del plain
    torch.cuda.empty_cache()

    # learned schedule, BF16 storage
    tr = make("learned", True)
    # calibration: the tile-cost MLPs learn from the renderer's own timings
    for _ in range(args.calib):
        tr.step()
    for _ in range(args.warmup):
        tr.step()
    stages = {}
    with Clocks(local) as clk:
        ms, launches = timed(tr, args.steps, stage_times=stages, profile=True)
    clocks = clk.summary()
    ips = replica_throughput(args.steps, ms, 1)
    e2e_ms, _ = timed(tr, args.steps, e2e=True)
    e2e_ips = replica_throughput(args.steps, e2e_ms, 1)
    # the fwd+bwd iteration alone (projection .. projection backward + L1, no Adam)
    for _ in range(3):
        tr.iteration()
    it_stages = {}
    it_ms, _ = timed(tr, args.steps, adam=False)
    timed(tr, args.steps, stage_times=it_stages, adam=False)
    it_ips = replica_throughput(args.steps, it_ms, 1)
    assert tr.frame.check_errors() == 0, "kernel error word set (learned path)"
    # Gaussians the reverse pass gave a 2D gradient (the iteration's projection
    # backward leaves the records as the reverse pass wrote them)
    n_grad = int((tr.frame.grad2d[:len(cams) * N * 12].view(-1, 12)[:, :9] != 0).any(1).sum().item())
    # records whose colour the colour stage computed (the lists' records)
    n_col = int(tr.frame.colour_count.sum().item()) if tr.frame.defer_colour else None

    f = tr.frame
    # tiles whose kept prefix ran short and were repaired, per step (read back
    # step by step after the timed regions)
    flagged = []
    for _ in range(20):
        tr.step()
        flagged.append(int(f.flag_count.item()))
    sched_diag = schedule_diagnostics(f, L, torch)
    I = int(f.n_inst.item())
    I_full = int(f.tile_count.sum().item())
    I_proc = int(f.tile_nproc.sum().item())
    pairs = int(f.n_proc.sum().item())           # (pixel, Gaussian) pairs the blend loops walk
    Pix = sum(c.W * c.H for c in cams)
    ab = algorithmic_bytes(N, Pix, I, I_proc, True, len(cams), n_grad, learned_sh != L.GS_F32, n_col)
    stage_ms = {k: statistics.mean(v) for k, v in stages.items()}
    it_stage_ms = {k: statistics.mean(v) for k, v in it_stages.items()}
    kernel_stages = {k: v for k, v in stage_ms.items() if k in ab}
    dom = max(kernel_stages, key=kernel_stages.get)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = ab[dom] / (stage_ms[dom] / 1e3) / 1e9
    step_bytes = sum(v for k, v in ab.items() if k in stage_ms)
    whole = step_bytes / (ms / args.steps / 1e3) / 1e9
    it_bytes = sum(v for k, v in ab.items() if k in it_stage_ms)
    it_gbs = it_bytes / (it_ms / args.steps / 1e3) / 1e9
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clock_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    # the pairs are read after the timed region: valid for the timed steps
    # only while the scene stays the configured one (small learning rates)
    issue = issue_roofline(pairs, stage_ms.get("render_bwd"), sm_count, clock_hz) if args.lr_scale <= 1e-2 else None

    out = {
        "metric": METRIC, "value": round(ips * world, 3), "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded skewed-density scene, random-init parameters)",
        "config": {"workload": args.workload, "gaussians": N,
                   "view": [cam.W, cam.H] if len(cams) == 1 else [[c.W, c.H] for c in cams],
                   "step": "training step: every hot-path row incl. Adam and the cost-MLP training",
                   "schedule": f.schedule_report(),
                   "storage": ("bf16" if learned_sh == L.GS_BF16 else "fp32") + " SH + bf16 colour records, "
                              "fp32 blending and gradients",
                   "plain_fp32_count_iters_per_s": round(plain_ips * world, 3),
                   "learned_vs_plain": round(ips / plain_ips, 4),
                   "fwd_bwd_iteration": {
                       "what": "the step without Adam: project, bin, schedule, forward, L1, reverse pass, "
                               "projection backward, cost-MLP training",
                       "iters_per_s": round(it_ips * world, 3),
                       "plain_fp32_count_iters_per_s": round(plain_it_ips * world, 3),
                       "learned_vs_plain": round(it_ips / plain_it_ips, 4),
                       "algorithmic_bytes": int(it_bytes), "achieved_gbs": round(it_gbs, 1),
                       "hbm_frac": round(it_gbs / hbm, 4),
                       "stage_ms": {k: round(v, 4) for k, v in it_stage_ms.items()}},
                   "instances_full_lists": I_full, "instances_kept": I, "processed_instances": I_proc,
                   "pixel_pairs_processed": pairs, "gaussians_with_2d_gradient": n_grad,
                   "records_coloured": n_col,
                   "flagged_tiles_per_step": {"mean": round(statistics.mean(flagged), 2), "max": max(flagged)},
                   "l2": "inputs larger than L2 (0.4-0.7 GB of parameters, 1.5+ GB of instances)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "mlp_calibration_steps": args.calib, "adam_lr_scale": args.lr_scale,
                   "schedules": sched_diag},
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_ms_plain_fp32": {k: round(statistics.mean(v), 4) for k, v in plain_stages.items()},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": measured_traffic(dom, N), "algorithmic_bytes": int(ab[dom]),
                     "peak_source": peak_kind,
                     "whole_step_hbm_frac": round(whole / hbm, 4)},
        "issue_roofline_render_bwd": issue,
        "e2e": {"value": round(e2e_ips * world, 3), "unit": "iters/s",
                "h2d_bytes_per_step": int(tgt.numel() * 4), "d2h_bytes_per_step": 4},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene, cam)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_dynamic(args):
    """Dynamic training: every step is a training step (forward, L1, backward,
    Adam over all views) followed by one clone-and-prune (clone the 2% of
    Gaussians with the largest accumulated screen-space gradient, drop those
    with opacity below 0.005), so the Gaussian count changes from step to
    step and every buffer follows it.  Reports steps/s over the timed steps,
    the count trajectory, per-stage times and the clone-and-prune's HBM
    rate (parameters, both moments and the 16-bit shadow read and written
    once)."""
    import torch

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import pipeline as P
    from paper_2510_14564_gb300 import scenes as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.lib()
    w = S.WORKLOADS[args.workload]
    scene, cams = S.make_workload(args.workload, seed=0)
    N0 = scene.n
    tgt_host = torch.from_numpy(np.concatenate([S.random_image(c.W, c.H, seed=1 + v).ravel()
                                                for v, c in enumerate(cams)])).pin_memory()
    tgt = tgt_host.cuda()
    lr = tuple(x * args.lr_scale for x in P.DEFAULT_LR)
    # colours computed at projection: the clone rule piles Gaussians into the
    # same tiles, some 400 tiles a step outgrow their prefix, and colouring
    # the records of their rebuilt full lists one by one cost the forward
    # 1.2 ms a step (19.09 against 19.50 steps/s)
    tr = P.Trainer(cams, torch.from_numpy(scene.flat()).cuda(), N0, tgt, rgb_dtype=L.GS_BF16,
                   sh_storage=L.GS_BF16, schedule=P.Schedule(mode="learned"), lr=lr, defer_colour=False)
    del scene
    tr.track_screen_grad()
    frac, min_op = w["dynamic"]["clone_frac"], w["dynamic"]["min_opacity"]
    for _ in range(args.calib):
        tr.step()
    for _ in range(args.warmup):
        tr.step()
        tr.densify(frac, min_op)
    st = torch.cuda.current_stream()
    marks, counts, densify_ms = [], [tr.N], []

    def mark(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        marks.append((name, e))

    torch.cuda.synchronize()
    l0 = L.gs_launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        torch.cuda.profiler.start()     # a profiler started with --profile-from-start off sees only this
        t0.record(st)
        for _ in range(args.steps):
            tr.step(mark=mark)
            d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            d0.record(st)
            n_before = tr.N
            tr.densify(frac, min_op)
            d1.record(st)
            densify_ms.append((d0, d1, n_before, tr.N))
            counts.append(tr.N)
        t1.record(st)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    launches = L.gs_launch_count() - l0
    assert tr.frame.check_errors() == 0, "kernel error word set (dynamic training)"
    ms = t0.elapsed_time(t1)
    stages = {}
    for (n0, e0), (_, e1) in zip(marks[:-1], marks[1:]):
        if n0 != "end":
            stages.setdefault(n0, []).append(e0.elapsed_time(e1))
    dms = [a.elapsed_time(b) for a, b, _, _ in densify_ms]
    # clone-and-prune traffic: params, m, v read (N) and written (N'), the
    # 16-bit shadow written, the gradient statistic and sort keys read
    dbytes = [(3 * 59 * 4) * (n + n2) + 96 * n2 + 4 * n for _, _, n, n2 in densify_ms]
    dach = statistics.mean(b / (t / 1e3) / 1e9 for b, t in zip(dbytes, dms))
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ips = args.steps / (ms / 1e3)
    out = {
        "metric": "dynamic training steps/s (training step + clone/prune) @6M Gaussians, 4 views 1920x1080",
        "value": round(ips, 3), "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded skewed-density scene, random-init parameters)",
        "config": {"workload": args.workload, "gaussians_start": N0, "gaussians_timed_first": counts[0],
                   "gaussians_timed_last": counts[-1], "gaussians_mean": round(statistics.mean(counts)),
                   "clone_frac": frac, "min_opacity": min_op, "views": [[c.W, c.H] for c in cams],
                   "schedule": tr.frame.schedule_report(),
                   "storage": "bf16 SH + bf16 colour, fp32 blending and gradients",
                   "adam_lr_scale": args.lr_scale, "mlp_calibration_steps": args.calib,
                   "l2": "inputs larger than L2", "graphs": "none (eager launches; the count is read back)"},
        "stage_ms": {**{k: round(statistics.mean(v), 4) for k, v in stages.items()},
                     "densify": round(statistics.mean(dms), 4)},
        "roofline": {"kernel": "densify", "bound": "hbm", "achieved": round(dach, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(dach / hbm, 4), "traffic": None,
                     "algorithmic_bytes": int(statistics.mean(dbytes)), "peak_source": peak_kind},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def run_colour_ablation(args):
    """Colour-layout ablation of the forward pass (the reordering-based
    memory access of Sec. V): the same lists rendered with the colour planar
    or interleaved, read in the blend loop or batch-loaded into shared
    memory, beside the production kernel (colour inside the staged splat
    record).  FP32 records; kept prefixes from the guaranteed bound of a
    first step (nothing flagged).  Each render is timed alone with CUDA
    events after an L2 flush; the images are checked equal bit for bit."""
    import torch

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import pipeline as P
    from paper_2510_14564_gb300 import scenes as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.lib()
    scene, cams = S.make_workload(args.workload, seed=0)
    N = scene.n
    params = P.to_device_params(scene)
    fr = P.Frame(cams, N, rgb_dtype=L.GS_F32, prefix=True)
    fr.project(P.param_views(params, N))
    fr.bin_sort()
    fr.render()
    torch.cuda.synchronize()
    assert fr.check_errors() == 0 and int(fr.flag_count.item()) == 0
    VN = fr.V * N
    planar = torch.empty(3 * VN, dtype=torch.float32, device="cuda")
    inter = torch.empty(3 * VN, dtype=torch.float32, device="cuda")
    L.gs_colour_arrays(VN, fr.splats, planar, inter)
    ref = fr.img.clone()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")     # 256 MB > L2
    img = torch.empty_like(fr.img)
    T = torch.empty_like(fr.T_final)
    npx = torch.empty_like(fr.n_proc)
    tn = torch.empty_like(fr.tile_nproc)

    def production():
        L.gs_render_fwd(fr.cams, fr.ranges, fr.vals, fr.splats, L.GS_F32, None, img, T, npx, tn, None, fr.err)

    runs = {"production_record": production}
    for name, layout in L.COLOUR_LAYOUTS.items():
        col = planar if "planar" in name else inter
        runs[name] = (lambda layout=layout, col=col: L.gs_render_fwd_colour(
            fr.cams, N, fr.ranges, fr.vals, fr.splats, layout, col, img, T, npx))
    st = torch.cuda.current_stream()
    times, equal = {}, {}
    for name, fn in runs.items():
        for _ in range(3):
            fn()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        times[name] = statistics.median(ms)
        equal[name] = bool(torch.equal(img, ref))
    torch.cuda.profiler.start()         # one launch of each, for a profiler started with --profile-from-start off
    for fn in runs.values():
        fn()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    base = times["planar_global"]
    out = {
        "metric": "forward-pass ms by colour layout (planar/interleaved x blend-loop/staged)",
        "unit": "ms", "higher_is_better": False, "steps": args.steps, "dtype": "f32",
        "data": "synthetic (seeded skewed-density scene, random-init parameters)",
        "config": {"workload": args.workload, "gaussians": N, "views": [[c.W, c.H] for c in cams],
                   "instances_kept": int(fr.n_inst.item()), "schedule": "raster, one CTA per tile",
                   "l2": "flushed before every timed render (256 MB write)"},
        "render_ms": {k: round(v, 4) for k, v in times.items()},
        "speedup_vs_planar_global": {k: round(base / v, 3) for k, v in times.items()},
        "images_equal_to_production": equal,
        "gpu_launches_per_render": 1,
    }
    print(json.dumps(out), flush=True)


def run_density_control(args):
    """One round of workload-sensitive density control (Sec. III-C) on the
    benchmark scene: local densities within r, thresholds, k-nearest
    dispersion, spawned and merged Gaussians written into buffers of the new
    count.  Reports ms per round and for the statistics alone (CUDA events),
    the classes' sizes and the thresholds."""
    import torch

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import scenes as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.lib()
    scene, _ = S.make_workload(args.workload, seed=0)
    N = scene.n
    r, k, alpha_d, delta = args.density_r, 3, 1.5, 0.2 * args.density_r
    p = torch.from_numpy(scene.flat()).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    z, u = (torch.from_numpy(a.ravel()).cuda() for a in S.density_draws(N))
    cap = 2 * N + 3
    p2 = torch.empty(59 * cap, device="cuda")
    m2, v2 = torch.empty_like(p2), torch.empty_like(p2)
    sh = torch.empty(48 * cap, dtype=torch.bfloat16, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    thr = torch.zeros(3, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.gs_density_workspace(N) // 4 + 64, dtype=torch.float32, device="cuda")
    rho = torch.empty(N, dtype=torch.int32, device="cuda")
    nn = torch.empty_like(rho)
    dbar = torch.empty(N, device="cuda")
    dnn = torch.empty_like(dbar)

    def control():
        L.gs_density_control(N, p, m, v, z, u, r, k, 1.0, 1.0, alpha_d, delta, 1.0, cap, p2, m2, v2, sh,
                             L.GS_BF16, n_out, thr, ws, err)

    def stats():
        L.gs_density_stats(N, p, r, k, rho, dbar, nn, dnn, (1.0, 1.0, 1.0), thr, ws)

    st = torch.cuda.current_stream()
    res = {}
    for name, fn in (("round", control), ("stats", stats)):
        for _ in range(args.warmup):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(args.steps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / args.steps
    assert int(err.item()) == 0
    lo, hi, dm = (float(x) for x in thr.cpu())
    rh = rho.cpu().numpy()
    out = {
        "metric": "density-control round ms (densities, thresholds, kNN dispersion, spawn and merge)",
        "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "data": "synthetic (seeded skewed-density scene; seeded normal and uniform draws)",
        "config": {"workload": args.workload, "gaussians": N, "r": r, "k": k, "alpha": 1.0, "beta": 1.0,
                   "gamma": 1.0, "alpha_d": alpha_d, "delta": delta},
        "round_ms": round(res["round"], 3), "stats_ms": round(res["stats"], 3),
        "gaussians_out": int(n_out.item()), "rho_low": lo, "rho_high": hi, "d_merge": dm,
        "low": int((rh < lo).sum()), "high": int((rh > hi).sum()), "rho_mean": float(rh.mean()),
        "rho_max": int(rh.max()),
    }
    print(json.dumps(out), flush=True)


def run_colour_buckets(args):
    """Colour hashing of the tile lists (Sec. IV-C1) on the benchmark view:
    the full lists and the kept prefixes of a training step (16-bit records),
    each hashed into the 4096 buckets.  Reports ms (CUDA events), entries per
    second, the mean number of distinct buckets per non-empty tile and the
    share of entries whose tile holds another entry of the same bucket."""
    import torch

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import pipeline as P
    from paper_2510_14564_gb300 import scenes as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.lib()
    scene, cams = S.make_workload(args.workload, seed=0)
    N = scene.n
    views = P.param_views(P.to_device_params(scene), N)
    st = torch.cuda.current_stream()
    res = {}
    for name, prefix in (("full_lists", False), ("kept_prefixes", True)):
        fr = P.Frame(cams, N, rgb_dtype=L.GS_BF16, prefix=prefix)
        fr.project(views)
        fr.bin_sort()
        if prefix:                     # a step's history: prefixes cut at twice the processed counts
            fr.render()
            fr.bin_sort()
        count = torch.zeros(4096, dtype=torch.int64, device="cuda")
        sums = torch.zeros(4 * 4096, dtype=torch.float64, device="cuda")
        distinct = torch.zeros(fr.T, dtype=torch.int32, device="cuda")
        run = lambda: L.gs_colour_buckets(fr.T, fr.ranges, fr.vals, fr.splats, L.GS_BF16, count, sums, distinct)
        for _ in range(args.warmup):
            run()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(args.steps):
            run()
        b.record(st)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        lens = (fr.ranges.view(-1, 2)[:, 1] - fr.ranges.view(-1, 2)[:, 0]).double()
        d = distinct.double()
        entries = float(lens.sum())
        res[name] = {"ms": round(ms, 4), "entries": int(entries),
                     "entries_per_s": round(entries / (ms / 1e3), 1),
                     "mean_distinct_buckets_per_tile": round(float(d[lens > 0].mean()), 2),
                     "share_in_shared_bucket": round(1.0 - float(d.sum()) / max(entries, 1.0), 4)}
        del fr
        torch.cuda.empty_cache()
    out = {"metric": "colour hashing of tile lists (4096 buckets), ms per pass", "unit": "ms",
           "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
           "data": "synthetic (seeded skewed-density scene, random-init parameters)",
           "config": {"workload": args.workload, "gaussians": N, "records": "bf16 colour"},
           "passes": res}
    print(json.dumps(out), flush=True)


def run_colour_merge(args):
    """Similarity-based sampling and merging (Sec. IV-C1) on the benchmark
    view, BF16 records: the exact forward pass against the merge plus the
    render of the merged lists, for the full lists and for the kept prefixes
    of a training step.  Reports ms (CUDA events, median of --steps, L2
    flushed before each), the entries kept and the merged image's distance to
    the exact one (the mode is lossy)."""
    import torch

    from paper_2510_14564_gb300 import _lib as L
    from paper_2510_14564_gb300 import pipeline as P
    from paper_2510_14564_gb300 import scenes as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.lib()
    scene, cams = S.make_workload(args.workload, seed=0)
    N = scene.n
    params = P.to_device_params(scene)
    views = dict(P.param_views(params, N))
    views["sh"] = views["sh"].to(torch.bfloat16)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2

    def timed(fn):
        ts = []
        for k in range(args.warmup + args.steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res = {}
    for name, prefix in (("full_lists", False), ("kept_prefixes", True)):
        fr = P.Frame(cams, N, rgb_dtype=L.GS_BF16, sh_dtype=L.GS_BF16, prefix=prefix)
        fr.project(views)
        fr.bin_sort()
        if prefix:                     # a step's history: prefixes cut at twice the processed counts
            fr.render()
            fr.bin_sort()
        tile_nproc = torch.empty(fr.T, dtype=torch.int32, device="cuda")    # leaves the history alone
        exact = lambda: L.gs_render_fwd(fr.cams, fr.ranges, fr.vals, fr.splats, fr.rgb_dtype, None, fr.img,
                                        fr.T_final, fr.n_proc, tile_nproc, None, fr.err)
        ms_exact = timed(exact)
        img_exact = fr.img.clone()
        ms_merged = timed(fr.render_merged)
        mr = fr.m_ranges.view(-1, 2).long()
        lens = fr.ranges.view(-1, 2).long()
        kept = int((mr[:, 1] - mr[:, 0]).sum())
        entries = int((lens[:, 1] - lens[:, 0]).sum())
        d = (fr.img - img_exact).double()
        mse = float((d * d).mean())
        assert fr.check_errors() == 0
        res[name] = {"entries": entries, "representatives": kept, "kept_share": round(kept / max(1, entries), 4),
                     "ms_exact_render": round(ms_exact, 4), "ms_merge_plus_render": round(ms_merged, 4),
                     "speedup": round(ms_exact / ms_merged, 3),
                     "image_vs_exact": {"max_abs": round(float(d.abs().max()), 5),
                                        "mean_abs": round(float(d.abs().mean()), 6),
                                        "psnr_db": round(10 * np.log10(1.0 / max(mse, 1e-30)), 2)}}
        del fr
        torch.cuda.empty_cache()
    out = {"metric": "similarity-based sampling and merging: merged vs exact forward render, ms", "unit": "ms",
           "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
           "data": "synthetic (seeded skewed-density scene, random-init parameters)",
           "config": {"workload": args.workload, "gaussians": N, "records": "bf16 colour",
                      "l2": "flushed before each timed pass"},
           "passes": res}
    print(json.dumps(out), flush=True)


def schedule_diagnostics(f, L, torch, reps=5) -> dict:
    """Render makespans (best of `reps`, ms) of the forward pass in raster
    and count order, and of the reverse pass in raster, count,
    processed-count and learned order (orders computed beforehand; the
    learned one splits the tiles its MLP predicts heavy, the others by
    processed count); the cost of computing each order; per-tile time
    spread of the forward."""
    def best(fn):
        out = 1e9
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            out = min(out, a.elapsed_time(b))
        return round(out, 4)

    keep = f.force_order
    t_count = best(lambda: f._count_order(f.order_f))
    o_count = f.order_f.clone()
    f.force_order = "learned"
    t_learned = best(lambda: f._sched_bwd())
    o_learned = f.order_b.clone()
    pred = f.pred_b.clone()
    f.force_order = keep
    L.gs_int_cost(f.tile_nproc, f.T, f.cost)
    L.gs_sched_order(f.cost, f.T, f.order_b, f.order_ws)
    o_proc = f.order_b.clone()

    def sch(o):
        return None if o is None else {"mode": L.GS_SCHED_ORDER, "order": o, "queue": f.queue}

    def fwd(o):
        L.gs_render_fwd(f.cams, f.ranges, f.vals, f.splats, f.rgb_dtype, sch(o), f.img, f.T_final, f.n_proc,
                        f.tile_nproc, None, f.err)

    def bwd(o, cost=None):
        s = sch(o)
        if s is not None:
            s["split"] = f.split
            s["split_cost"] = cost
        L.gs_render_bwd(f.cams, f.ranges, f.vals, f.splats, f.rgb_dtype, s, f.dimg, f.T_final, f.n_proc,
                        f.tile_nproc, f.grad2d, f.err)

    out = {"fwd_ms": {"raster": best(lambda: fwd(None)), "count": best(lambda: fwd(o_count))},
           "bwd_ms": {"raster": best(lambda: bwd(None)), "count": best(lambda: bwd(o_count)),
                      "by_processed": best(lambda: bwd(o_proc)), "learned": best(lambda: bwd(o_learned, pred))},
           "order_cost_ms": {"count": t_count, "learned_bwd": t_learned}}
    L.gs_render_fwd(f.cams, f.ranges, f.vals, f.splats, f.rgb_dtype, None, f.img, f.T_final,
                    f.n_proc, f.tile_nproc, f.tile_ns, f.err)
    torch.cuda.synchronize()
    ns = f.tile_ns.double()
    out["tile_us"] = {"mean": round(float(ns.mean()) / 1e3, 3), "max": round(float(ns.max()) / 1e3, 3),
                      "p99": round(float(ns.quantile(0.99)) / 1e3, 3)}
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def cpu_baseline(scene, cam) -> dict:
    """The oracle on the host cores, one bounded step of about 20 s."""
    from oracle import oracle as O
    O.build()
    step = OracleStep(scene, cam, steps_total=1, budget_s=20.0)
    full = step()
    return {"value": round(1.0 / full, 6), "unit": "iters/s", "cores": O.get_threads(), "kind": "oracle",
            "sample": step.describe()}


class OracleStep:
    """One bounded step of the oracle on the benchmark workload, sized so
    that `steps_total` steps take about `budget_s` seconds: the per-Gaussian
    stages (key path, projection, projection backward) on a seeded subset of
    the Gaussians, the per-pixel stages (render, L1, backward render) on
    seeded random segments of tile rows; each part's time is extrapolated to
    the whole view (by the Gaussian count and by the tile count; the segments
    are a uniform sample, and each call's fixed cost, which a whole-view run
    pays once, is charged to every segment)."""

    def __init__(self, scene, cam, steps_total: int, budget_s: float = 120.0):
        from oracle import oracle as O
        self.O, self.scene, self.cam = O, scene, cam
        t0 = time.perf_counter()
        self.kp = O.keypath(cam, scene)                       # full key path and projection, untimed:
        self.pr = O.project(cam, scene, self.kp)              # the tile renders need every Gaussian
        rng = np.random.default_rng(7)
        per_step = max(0.05, budget_s / max(1, steps_total))
        probe = scene.subset(np.sort(rng.choice(scene.n, min(scene.n, 50_000), replace=False)))
        tg = self._gauss_part(probe)
        self.n_sub = int(min(scene.n, max(10_000, 0.5 * per_step * probe.n / tg)))
        # row segments: whole rows when a row fits half the step, else quarter rows
        tx = cam.tiles_x
        probe_seg = [(cam.tiles_y // 2, 0, tx)]
        t_row = self._pixel_part(probe_seg)
        self.seg = tx if t_row <= 0.5 * per_step else max(1, tx // 4)
        per_seg = t_row * self.seg / tx
        nseg = int(np.clip(0.5 * per_step / per_seg, 1, 64))
        segs = [(ty, x0, min(tx, x0 + self.seg)) for ty in range(cam.tiles_y) for x0 in range(0, tx, self.seg)]
        pick = rng.choice(len(segs), min(nseg, len(segs)), replace=False)
        self.segs = [segs[k] for k in pick]
        self.seg_tiles = sum(b - a for _, a, b in self.segs)
        self.sub = scene.subset(np.sort(rng.choice(scene.n, self.n_sub, replace=False)))
        self.setup_s = time.perf_counter() - t0

    def _gauss_part(self, sc):
        O, cam = self.O, self.cam
        t0 = time.perf_counter()
        kp = O.keypath(cam, sc)
        O.project(cam, sc, kp)
        O.project_bwd(cam, sc, kp, np.full((sc.n, 9), 1e-3))
        return time.perf_counter() - t0

    def _pixel_part(self, segs):
        O, cam = self.O, self.cam
        t0 = time.perf_counter()
        for ty, a, b in segs:
            x0, y0, x1, y1 = 16 * a, 16 * ty, min(16 * b, cam.W), min(16 * ty + 16, cam.H)
            r = O.render(cam, self.kp, self.pr, window=(x0, y0, x1, y1))
            crop = np.ascontiguousarray(r["img"][:, y0:y1, x0:x1])
            _, dc = O.l1(crop, np.zeros_like(crop))
            dimg = np.zeros_like(r["img"])
            dimg[:, y0:y1, x0:x1] = dc
            O.render_bwd(cam, self.kp, self.pr, dimg, window=(x0, y0, x1, y1))
        return time.perf_counter() - t0

    def __call__(self) -> float:
        """Seconds of one whole-view oracle iteration (extrapolated)."""
        tg = self._gauss_part(self.sub) * (self.scene.n / self.n_sub)
        tp = self._pixel_part(self.segs) * (self.cam.n_tiles / self.seg_tiles)
        return tg + tp

    def describe(self) -> str:
        return (f"per-Gaussian stages on a seeded subset of {self.n_sub} of {self.scene.n} Gaussians; "
                f"per-pixel stages on {len(self.segs)} seeded random tile-row segments ({self.seg_tiles} of "
                f"{self.cam.n_tiles} tiles); each extrapolated to the whole view by Gaussian and tile count")


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2510_14564_gb300 import scenes as S
    O.build()
    scene, cams = S.make_workload(args.workload, seed=0)
    cam = cams[0]
    step = OracleStep(scene, cam, args.steps + args.warmup)
    for _ in range(args.warmup):
        step()
    fulls = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fulls.append(step())
    wall = time.perf_counter() - t0
    full = statistics.mean(fulls)
    v = 1.0 / full
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "iters/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(full * 1e3, 2), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample_wall_s": round(wall, 2)},
           "cpu_baseline": {"kind": "oracle", "cores": O.get_threads(), "value": round(v, 6),
                            "sample": step.describe()},
           "e2e": {"value": round(v, 6), "unit": "iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _workloads() -> dict:
    from paper_2510_14564_gb300 import scenes as S
    return S.WORKLOADS


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 300; 20 for a dynamic-training workload, whose count grows)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--calib", type=int, default=40, help="untimed MLP calibration steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--colour-ablation", action="store_true",
                    help="time the forward pass under four colour layouts (prints its own JSON line)")
    ap.add_argument("--colour-buckets", action="store_true",
                    help="time the colour hashing of the tile lists (prints its own JSON line)")
    ap.add_argument("--colour-merge", action="store_true",
                    help="time the merged-bucket render against the exact one (prints its own JSON line)")
    ap.add_argument("--density-control", action="store_true",
                    help="time one round of workload-sensitive density control (prints its own JSON line)")
    ap.add_argument("--density-r", type=float, default=0.005, help="neighbour radius of the density control")
    ap.add_argument("--lr-scale", type=float, default=1e-3,
                    help="scale of the Adam learning rates (keeps the scene fixed over the run)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.colour_buckets:
        args.steps = 10 if args.steps is None else args.steps
        run_colour_buckets(args)
    elif args.colour_merge:
        args.steps = 20 if args.steps is None else args.steps
        run_colour_merge(args)
    elif args.density_control:
        args.steps = 10 if args.steps is None else args.steps
        run_density_control(args)
    elif args.colour_ablation:
        args.steps = 20 if args.steps is None else args.steps
        run_colour_ablation(args)
    elif args.impl == "reference":
        args.steps = 300 if args.steps is None else args.steps
        run_reference(args)
    elif "dynamic" in _workloads().get(args.workload, {}):
        args.steps = 20 if args.steps is None else args.steps
        w = _workloads()[args.workload]
        grown = w["n"] * (1 + w["dynamic"]["clone_frac"]) ** (args.warmup + args.steps)
        if grown > 32e6:
            ap.error(f"{args.warmup + args.steps} clone-and-prune steps could grow the count to "
                     f"{grown / 1e6:.0f}M Gaussians; at most 32M are allowed")
        run_dynamic(args)
    else:
        args.steps = 300 if args.steps is None else args.steps
        run_ours(args)


if __name__ == "__main__":
    main()

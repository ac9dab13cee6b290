"""Benchmark of the batched MPT hot path on GB300.

One step = the whole path over one batch: candidate enumeration, the
Gauss-Newton solve of every candidate (FP32 iterations + FP64 refinement),
validation with visibility and compaction, and the adjoint of every valid
path (unit weight on its length).  Workload: the 12-box urban block (97
objects: 48 walls, 48 vertical edges, ground), 1 TX at 30 m, 32x32 RX at
1.5 m, every reflection/diffraction sequence of order <= 2: 9,634,816
candidate solves per step, synthetic seeded scene.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is device-resident throughput
(scene and endpoints already in HBM) with the solve's schedule picked by
mpt_autotune for this workload before the warm-up (--no-tune: library
defaults); `e2e` is the same metric through the C ABI starting from host
arrays: the scene resident (uploaded once, like a model's weights), every
step's TX/RX endpoints copied host->device and its valid paths (count,
candidate ids, points, lengths) and TX gradient read device->host inside the
timed region, steps pipelined over two contexts and streams.  The default
1000 steps keep the timed region above a second.  `workloads` times the other
workloads as their own steps, outside the timed region: the street canyon
(plain FP64 method and FP32 + refinement), the mixed-order city (library
defaults and autotuned, eager and as a CUDA graph), the curved scene, the
64x64-RX block (forward alone and forward + adjoint) and the image method
beside the minimiser on the urban block's reflection-only candidates.
Under torchrun each rank solves its own batch (weak scaling, no data-path
collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPT candidate solves/sec at <=1e-6 m vs FP64 oracle; % of FP32 FMA peak"
UNIT = "solves/s"
WORKLOAD = "urban_block_12box_97obj_1tx_32x32rx_order2"
L2_FLUSH_BYTES = 256 << 20
SM_MAX_MHZ_NOMINAL = 2070.0
FP32_LANES_PER_SM = 128


def max_over_ranks(x: float, dev=None) -> float:
    """Max of a per-rank scalar over the process group: the whole job takes
    as long as its slowest rank.  gloo reduces CPU tensors, NCCL device ones."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    d = torch.device("cpu") if dist.get_backend() == "gloo" or dev is None else dev
    t = torch.tensor([float(x)], dtype=torch.float64, device=d)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2301_06399_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_tag: str):
    """DRAM bytes per launch recorded from an ncu capture of this source
    revision (profiles/*.md lines `traffic_bytes_per_launch[tag]: N sha`)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    sha = csrc_hash()
    for f in sorted(os.listdir(d)):
        if not f.endswith(".md"):
            continue
        for ln in open(os.path.join(d, f)):
            key = f"traffic_bytes_per_launch[{kernel_tag}]:"
            if ln.startswith(key):
                parts = ln[len(key):].split()
                if len(parts) >= 2 and parts[1] == sha:
                    return float(parts[0])
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


def build_scene(rank: int, rx_side: int = 32):
    from paper_2301_06399_gb300 import scenes

    sc = scenes.urban_block(rx_side)
    # each rank solves its own batch: the TX height differs per rank
    sc.tx = sc.tx.copy()
    sc.tx[:, 2] += 0.5 * rank
    return sc, scenes.CONFIG_SPECS["urban_block"]


def flop_table(mpt, sc):
    """Algorithmic FP32 FLOPs per (evaluation, factorisation) for every kind
    pattern of orders 1 and 2, from the library's counting model."""
    tab = {}
    kinds = sorted(set(int(k) for k in sc.obj_kind))
    for a in kinds:
        tab[(a,)] = mpt.flop_model([a])
        for b in kinds:
            tab[(a, b)] = mpt.flop_model([a, b])
    return tab


def algorithmic_flops(mpt, sc, cands, sols, n, only_order=None):
    """Sum over candidates (of one path order when only_order is set) of
    evals * F_eval + iters * F_iter (pattern-wise)."""
    rec = cands.rec[:n]
    kinds_t = torch.as_tensor(sc.obj_kind, dtype=torch.int64, device=rec.device)
    r = rec.to(torch.int64) & 0xFFFFFFFF
    order = r[:, 3] & 0xFF
    id0 = r[:, 1] & 0xFFFF
    id1 = (r[:, 1] >> 16) & 0xFFFF
    k0 = kinds_t[id0.clamp(max=kinds_t.numel() - 1)]
    k1 = torch.where(order >= 2, kinds_t[id1.clamp(max=kinds_t.numel() - 1)], torch.full_like(k0, -1))
    code = (order * 25 + (k0 + 1) * 5 + (k1 + 1)).to(torch.int64)
    ev = sols.evals[:n].to(torch.float64)
    it = sols.iters[:n].to(torch.float64)
    nbins = 3 * 25
    sum_ev = torch.bincount(code, weights=ev, minlength=nbins).cpu().numpy()
    sum_it = torch.bincount(code, weights=it, minlength=nbins).cpu().numpy()
    tab = flop_table(mpt, sc)
    total = 0.0
    for code_v in np.nonzero(sum_ev + sum_it)[0]:
        o, rest = divmod(int(code_v), 25)
        if only_order is not None and o != only_order:
            continue
        a, b = divmod(rest, 5)
        key = (a - 1,) if o == 1 else (a - 1, b - 1)
        f_iter, f_eval, _ = tab[key]
        total += sum_ev[code_v] * f_eval + sum_it[code_v] * f_iter
    return total


def solve_launches(mpt, sch, n_orders=4) -> int:
    """Kernels one FP32+refinement mpt_solve launches under schedule sch:
    endpoint copy, the exclusion pass (beams, bit table, candidate pass) with
    per-order launches, the solvers, and per order the visibility prescreen
    if on, the refinement and its fallback."""
    mixed = bool(sch.mixed_orders)
    prescreen = sch.prescreen != 2
    exclusion = 0 if (mixed or sch.exclude == 2) else 3
    return 1 + exclusion + (1 if mixed else n_orders) + n_orders * (3 if prescreen else 2)


def timed(stream, fn, reps, flush=None):
    """Median device time (ms) of fn() over reps calls, CUDA events on stream,
    an L2 flush outside the events before each call."""
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        stream.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def workload_legs(mpt, ctx, dev, stream, flush, reps):
    """The other workloads, each timed as its own step (outside the main timed
    region): candidates/s, valid paths/s and the schedule used."""
    from paper_2301_06399_gb300 import scenes

    legs = {}

    def trace_leg(sc, spec, max_order, precision=mpt.FP32_FP64REFINE, sch=None, grad_pts=False, graph=False):
        ds = mpt.DeviceScene(ctx, sc)
        n = mpt.candidate_count(ds, max_order, spec)
        cands = mpt.alloc_candidates(n, dev)
        sols = mpt.alloc_solutions(n, dev)
        paths = mpt.alloc_paths(1 << 22, dev)
        g_len = torch.ones(paths.capacity, dtype=torch.float64, device=dev)
        g_pts = torch.full((12, paths.capacity), 0.1, dtype=torch.float64, device=dev) if grad_pts else None

        def fwd():
            mpt.enumerate_candidates(ds, max_order, spec, out=cands, stream=stream)
            mpt.solve(ds, cands, precision, sch, out=sols, stream=stream)
            mpt.validate(ds, cands, sols, out=paths, stream=stream)

        def fwd_bwd():
            fwd()
            mpt.grad(ds, cands, paths, g_len, g_pts, stream=stream)

        fwd()
        stream.synchronize()
        out = {"candidates": n, "valid_paths_per_step": paths.n()}
        t = timed(stream, fwd, reps, flush)
        out.update({"ms_per_step": t, "solves_per_sec": n / (t * 1e-3), "valid_paths_per_sec": paths.n() / (t * 1e-3)})
        if grad_pts:
            tb = timed(stream, fwd_bwd, reps, flush)
            out.update({"forward_backward_ms": tb, "forward_only_ms": t})
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                fwd()
            g.replay()
            stream.synchronize()
            out["cuda_graph_ms"] = timed(stream, g.replay, reps, flush)
            del g
        del cands, sols, paths, g_len, g_pts, ds
        torch.cuda.empty_cache()
        return out

    # street canyon: the plain FP64 method of its config, and FP32 + refinement
    sc = scenes.street_canyon()
    legs["street_canyon_fp64_plain"] = trace_leg(sc, scenes.CONFIG_SPECS["street_canyon"], 2, mpt.FP64_PLAIN)
    legs["street_canyon_fp32_refine"] = trace_leg(sc, scenes.CONFIG_SPECS["street_canyon"], 2)
    # mixed orders 1-4: library defaults, then the autotuned schedule (eager and graph)
    sc = scenes.mixed_order_city()
    spec = scenes.CONFIG_SPECS["mixed_order"]
    legs["mixed_orders_default"] = trace_leg(sc, spec, 4, graph=True)
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 4, spec, stream=stream)
    best, best_ms = mpt.autotune(ds, cands, stream=stream)
    del cands, ds
    torch.cuda.empty_cache()
    legs["mixed_orders_tuned"] = trace_leg(sc, spec, 4, sch=best, graph=True)
    legs["mixed_orders_tuned"]["schedule"] = mpt.schedule_dict(best)
    # curved geometry, 4,096 pairs, 8 starts for curved sequences
    legs["curved_4096pairs"] = trace_leg(scenes.curved_scene(), scenes.CONFIG_SPECS["curved"], 3)
    # differentiable block, 64x64 RX: forward alone and forward + adjoint
    legs["differentiable_64x64rx"] = trace_leg(scenes.urban_block(64), scenes.CONFIG_SPECS["differentiable"], 2,
                                               grad_pts=True)
    # image method beside the minimiser on the urban block's reflection-only candidates
    ub = scenes.urban_block(32)
    keep = np.nonzero(ub.obj_kind == scenes.PLANE)[0]
    planes = scenes.Scene("urban_block_planes", ub.scale, ub.obj_kind[keep], ub.obj_param[keep], ub.occ_kind,
                          ub.occ_param, ub.tx, ub.rx, ub.pair_mode, ub.meta).contiguous()
    spec2 = scenes.SequenceSpec(quota=(-1, -1, 0, 0))
    ds = mpt.DeviceScene(ctx, planes)
    cands = mpt.enumerate_candidates(ds, 2, spec2, stream=stream)
    sols = mpt.alloc_solutions(cands.capacity, dev)
    paths = mpt.alloc_paths(1 << 20, dev)
    im = {"candidates": cands.capacity}
    im["image_method_ms"] = timed(stream, lambda: mpt.image_method(ds, cands, out=sols, stream=stream), reps, flush)
    mpt.validate(ds, cands, sols, out=paths, stream=stream)
    stream.synchronize()
    im["image_method_valid"] = paths.n()
    im["minimiser_ms"] = timed(stream, lambda: mpt.solve(ds, cands, mpt.FP32_FP64REFINE, out=sols, stream=stream),
                               reps, flush)
    mpt.validate(ds, cands, sols, out=paths, stream=stream)
    stream.synchronize()
    im["minimiser_valid"] = paths.n()
    im["minimiser_over_image_method"] = im["minimiser_ms"] / im["image_method_ms"]
    legs["image_method_vs_minimiser_urban_block_planes"] = im
    del cands, sols, paths, ds
    torch.cuda.empty_cache()
    return legs


def run_ours(args):
    ws, rank, local = dist_env()
    import torch.distributed as dist

    if ws > 1:
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_2301_06399_gb300 import mpt

    sc, spec = build_scene(rank, args.rx_side)
    ctx = mpt.Context(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ds = mpt.DeviceScene(ctx, sc)
        n_cand = mpt.candidate_count(ds, 2, spec)
        cands = mpt.alloc_candidates(n_cand, dev)
        sols = mpt.alloc_solutions(n_cand, dev)
        path_cap = 1 << 20
        paths = mpt.alloc_paths(path_cap, dev)
        g_len = torch.ones(path_cap, dtype=torch.float64, device=dev)
        g_tx = torch.zeros_like(ds.tx)
        g_rx = torch.zeros_like(ds.rx)
        g_obj = torch.zeros(sc.n_obj, dtype=torch.float64, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        # the schedule of the solve: mpt_autotune's choice for this workload
        mpt.enumerate_candidates(ds, 2, spec, out=cands, stream=stream)
        if args.no_tune:
            sched = mpt.schedule_struct()
        else:
            sched, _ = mpt.autotune(ds, cands, out=sols, stream=stream)

        def step(precision=mpt.FP32_FP64REFINE, ev=None):
            mpt.enumerate_candidates(ds, 2, spec, out=cands, stream=stream)
            if ev is not None:
                ev[0].record(stream)
            mpt.solve(ds, cands, precision, sched, out=sols, stream=stream)
            if ev is not None:
                ev[1].record(stream)
            mpt.validate(ds, cands, sols, out=paths, stream=stream)
            mpt.grad(ds, cands, paths, g_len, g_tx=g_tx, g_rx=g_rx, g_obj=g_obj, stream=stream)
        for _ in range(args.warmup):
            step()
        stream.synchronize()
        n_valid = paths.n()
        n_excluded = int(((sols.status[:n_cand] & 0x0F) == mpt.PATH_EXCLUDED).sum().item())
        flops = algorithmic_flops(mpt, sc, cands, sols, n_cand)
        # enumerate (2) + solve (endpoint copy, solver launches, per order the
        # visibility prescreen if on, refinement and its fallback) + validate
        # (list, test, scan, scatter, fill) + adjoint (one launch per order)
        launches_per_step = 2 + solve_launches(mpt, sched) + 5 + 4

        # ---- device-resident timing
        ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        ev_solve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    for _ in range(args.steps)]
        clocks = ClockSampler(local)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        time.sleep(0.3)
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # L2 flush between steps, outside the step events
            ev_step[i][0].record(stream)
            step(ev=ev_solve[i])
            ev_step[i][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
        if ws > 1:
            dist.barrier()
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in ev_step]
        solve_ms = [a.elapsed_time(b) for a, b in ev_solve]
        total_ms = float(sum(step_ms))
        total_ms = max_over_ranks(total_ms, dev)
        ms_per_step = total_ms / args.steps
        value = n_cand * ws / (ms_per_step * 1e-3)

        # ---- the same step captured once as a CUDA graph (the auxiliary
        # streams of the per-order chains join the capture through their
        # fork/join events) and replayed: no host launch work per step
        graph_leg = None
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                step()
            g.replay()
            stream.synchronize()
            n_valid_graph = paths.n()
            graph_ms = []
            for i in range(max(3, min(args.steps, 20))):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.replay()
                b.record(stream)
                stream.synchronize()
                graph_ms.append(a.elapsed_time(b))
            graph_leg = {"ms_per_step": float(np.median(graph_ms)),
                         "value": n_cand * ws / (float(np.median(graph_ms)) * 1e-3), "unit": UNIT,
                         "valid_paths_per_step": n_valid_graph}
            del g
        except Exception as exc:  # reported, never silently replaced
            graph_leg = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        stream.synchronize()

        # ---- plain FP64 GPU method (same algorithm, FP64 throughout)
        fp64_ms = []
        for i in range(max(1, min(args.steps, 3))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(precision=mpt.FP64_PLAIN)
            b.record(stream)
            stream.synchronize()
            fp64_ms.append(a.elapsed_time(b))
        n_valid_fp64 = paths.n()

        # ---- received field of the valid paths (Sec. V; 1 GHz, PEC
        # reflections, unit diffraction coefficient), on the last step's paths
        fld = torch.zeros((ds.n_pairs, 2), dtype=torch.float64, device=dev)
        field_ms = []
        for i in range(max(3, min(args.steps, 10))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mpt.field(ds, cands, paths, 2 * np.pi / 0.3, 1.0, -1.0, 1.0, out=fld, stream=stream)
            b.record(stream)
            stream.synchronize()
            field_ms.append(a.elapsed_time(b))
        field_leg = {"ms": float(np.median(field_ms)), "paths": paths.n(),
                     "paths_per_sec": paths.n() / (float(np.median(field_ms)) * 1e-3)}

        # ---- the pipeline on the visibility-pruned graph of Algorithm 1
        # (mpt_visibility as the enumeration's adjacency mask; the masked
        # enumeration synchronises once to size its table)
        vis_ms, pr_ms = [], []
        pr_cands = mpt.alloc_candidates(cands.capacity, dev)
        for i in range(max(3, min(args.steps, 10))):
            flush.zero_()
            a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            V = mpt.visibility(ds, stream=stream)
            b.record(stream)
            mpt.enumerate_candidates(ds, 2, spec, adj=V, out=pr_cands, stream=stream)
            mpt.solve(ds, pr_cands, mpt.FP32_FP64REFINE, sched, out=sols, stream=stream)
            mpt.validate(ds, pr_cands, sols, out=paths, stream=stream)
            mpt.grad(ds, pr_cands, paths, g_len, g_tx=g_tx, g_rx=g_rx, g_obj=g_obj, stream=stream)
            c2.record(stream)
            stream.synchronize()
            vis_ms.append(a.elapsed_time(b))
            pr_ms.append(a.elapsed_time(c2))
        pruned = {"candidates": int(pr_cands.count.item()), "visibility_ms": float(np.median(vis_ms)),
                  "ms_per_step": float(np.median(pr_ms)), "valid_paths_per_step": paths.n()}
        pruned["valid_paths_per_sec"] = pruned["valid_paths_per_step"] * ws / (pruned["ms_per_step"] * 1e-3)

        # ---- the FP32 minimiser alone (MPT_FP32: endpoint copy + k_gn per
        # order, no prescreen or refinement), for the roofline of the
        # dominant kernel
        mini_ms = []
        for i in range(max(3, min(args.steps, 10))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mpt.solve(ds, cands, mpt.FP32, sched, out=sols, stream=stream)
            b.record(stream)
            stream.synchronize()
            mini_ms.append(a.elapsed_time(b))
        mini_flops = algorithmic_flops(mpt, sc, cands, sols, n_cand)
        # the same with every candidate iterated (no half-space exclusion):
        # the minimiser's efficiency over the whole candidate set
        sched_all = mpt.Schedule.from_buffer_copy(sched)
        sched_all.exclude = 2
        all_ms = []
        for i in range(max(3, min(args.steps, 10))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mpt.solve(ds, cands, mpt.FP32, sched_all, out=sols, stream=stream)
            b.record(stream)
            stream.synchronize()
            all_ms.append(a.elapsed_time(b))
        all_flops = algorithmic_flops(mpt, sc, cands, sols, n_cand)
        # ---- the dominant kernel alone, live: the order-2 solver's launch
        # inside full steps, timed by the library with CUDA events on the
        # stream it runs on (mpt_ctx_time_solver), L2 flushed before each step
        ctx.time_solver(True)
        kgn_ms = []
        for i in range(max(5, min(args.steps, 40))):
            flush.zero_()
            step()
            stream.synchronize()
            kgn_ms.append(ctx.solver_ms(2))
        ctx.time_solver(False)
        kgn2_flops = algorithmic_flops(mpt, sc, cands, sols, n_cand, only_order=2)
        kgn2_ms = float(np.mean(kgn_ms))
        # restore the FP32 state for the e2e leg
        step()
        stream.synchronize()

        # ---- end to end through the C ABI from host arrays.  The scene stays
        # resident (uploaded once, like a model's weights); every step copies
        # its TX/RX endpoints from pinned host memory and reads back its valid
        # paths (count, candidate ids, points, lengths) and the TX gradient.
        # Steps alternate between two contexts, each on its own stream, so
        # that one step's count read and result copies overlap the next
        # step's kernels.  The working set (candidates and solutions, ~0.9 GB)
        # exceeds the L2, so no flush runs between these steps.
        tx_h = torch.as_tensor(sc.tx).pin_memory()
        rx_h = torch.as_tensor(sc.rx).pin_memory()
        h2d_bytes = tx_h.numel() * 8 + rx_h.numel() * 8

        class Slot:
            pass

        slots = []
        for k in range(2):
            sl = Slot()
            sl.ctx = ctx if k == 0 else mpt.Context(local)
            sl.st = stream if k == 0 else torch.cuda.Stream(device=dev)
            with torch.cuda.stream(sl.st):
                sl.ds = ds if k == 0 else mpt.DeviceScene(sl.ctx, sc)
                sl.cands = cands if k == 0 else mpt.alloc_candidates(n_cand, dev)
                sl.sols = sols if k == 0 else mpt.alloc_solutions(n_cand, dev)
                sl.paths = paths if k == 0 else mpt.alloc_paths(path_cap, dev)
                sl.g_len = g_len if k == 0 else torch.ones(path_cap, dtype=torch.float64, device=dev)
                sl.g_tx = g_tx if k == 0 else torch.zeros_like(sl.ds.tx)
                sl.g_rx = g_rx if k == 0 else torch.zeros_like(sl.ds.rx)
                sl.g_obj = g_obj if k == 0 else torch.zeros(sc.n_obj, dtype=torch.float64, device=dev)
            sl.count_h = torch.zeros(1, dtype=torch.int64).pin_memory()
            sl.out_cand = torch.empty(path_cap, dtype=torch.int64).pin_memory()
            sl.out_X = torch.empty(12 * path_cap, dtype=torch.float64).pin_memory()
            sl.out_len = torch.empty(path_cap, dtype=torch.float64).pin_memory()
            sl.out_gtx = torch.empty_like(g_tx, device="cpu").pin_memory()
            sl.ev_count = torch.cuda.Event()
            slots.append(sl)
        stream.synchronize()

        def e2e_launch(sl):
            with torch.cuda.stream(sl.st):
                sl.ds.tx.copy_(tx_h, non_blocking=True)  # host -> device inputs
                sl.ds.rx.copy_(rx_h, non_blocking=True)
                mpt.enumerate_candidates(sl.ds, 2, spec, out=sl.cands, stream=sl.st)
                mpt.solve(sl.ds, sl.cands, mpt.FP32_FP64REFINE, sched, out=sl.sols, stream=sl.st)
                mpt.validate(sl.ds, sl.cands, sl.sols, out=sl.paths, stream=sl.st)
                sl.g_tx.zero_()
                mpt.grad(sl.ds, sl.cands, sl.paths, sl.g_len, g_tx=sl.g_tx, g_rx=sl.g_rx, g_obj=sl.g_obj,
                         stream=sl.st)
                sl.count_h.copy_(sl.paths.count.view(1), non_blocking=True)  # device -> host count
                sl.ev_count.record(sl.st)

        def e2e_read_back(sl):
            sl.ev_count.synchronize()
            nv = min(int(sl.count_h[0]), path_cap)
            with torch.cuda.stream(sl.st):
                sl.out_cand[:nv].copy_(sl.paths.cand[:nv], non_blocking=True)
                # the 12 coordinate rows gathered on the device, then one copy
                sl.out_X[:12 * nv].copy_(sl.paths.X[:, :nv].contiguous().view(-1), non_blocking=True)
                sl.out_len[:nv].copy_(sl.paths.length[:nv], non_blocking=True)
                sl.out_gtx.copy_(sl.g_tx, non_blocking=True)
            return 8 + nv * (8 + 12 * 8 + 8) + sl.out_gtx.numel() * 8

        n_e2e = max(3, min(args.steps, 200))
        e2e_launch(slots[0])  # warm-up of the second context's scratch as well
        e2e_launch(slots[1])
        e2e_read_back(slots[0])
        e2e_read_back(slots[1])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_launch(slots[0])
        d2h_list = []
        for i in range(n_e2e):
            if i + 1 < n_e2e:
                e2e_launch(slots[(i + 1) % 2])
            d2h_list.append(e2e_read_back(slots[i % 2]))
        for sl in slots:
            sl.st.synchronize()
        e2e_total_ms = (time.perf_counter() - t0) * 1e3
        d2h_bytes = int(np.median(d2h_list))
        e2e_ms = [e2e_total_ms / n_e2e]
        e2e_steps = n_e2e
        del slots
        e2e_ms_step = float(np.median(e2e_ms))
        e2e_ms_step = max_over_ranks(e2e_ms_step, dev)
        legs = None
        if not args.no_legs and rank == 0:
            del pr_cands
            torch.cuda.empty_cache()
            legs = workload_legs(mpt, ctx, dev, stream, flush, max(3, min(args.steps, 10)))

    solve_avg_ms = float(np.mean(solve_ms))
    achieved = flops / (solve_avg_ms * 1e-3) / 1e12
    n_sm = ctx.sm_count
    peak_max = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+ff48 (fp64 storage)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.rx_side == 32 else f"{WORKLOAD} (rx grid {args.rx_side}x{args.rx_side})",
                   "candidates_per_gpu": n_cand, "max_order": 2,
                   "precision": "fp32 iterations; float-float refinement of prescreened candidates (fp64 results); fp64 fallback solve of ill-conditioned ones; fp64 acceptance decisions near the margins",
                   "schedule": mpt.schedule_dict(sched) | {"source": "defaults" if args.no_tune else "mpt_autotune"},
                   "step": "enumerate + solve + validate/compact + adjoint",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write), outside the step events",
                   "parallelism": f"weak: one process per GPU, {ws} GPU(s)"},
        "valid_paths_per_step": n_valid,
        "valid_paths_per_sec": n_valid * ws / (ms_per_step * 1e-3),
        "excluded_per_step": n_excluded,
        "iterated_per_step": n_cand - n_excluded,
        "roofline": {"kernel": "k_gn<2> (the order-2 FP32 solver, the dominant kernel; launch timed live with "
                               "CUDA events inside full steps)", "bound": "alu",
                     "achieved": kgn2_flops / (kgn2_ms * 1e-3) / 1e12, "peak": peak_max, "unit": "TFLOP/s",
                     "frac": kgn2_flops / (kgn2_ms * 1e-3) / 1e12 / peak_max,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 x {SM_MAX_MHZ_NOMINAL:.0f} MHz (derived)",
                     "kernel_ms": kgn2_ms, "fp32_flops_per_launch": kgn2_flops,
                     "traffic": profile_traffic("k_gn2") if args.rx_side == 32 else None,
                     "solve_call": {"kernels": "mpt_solve: exclusion pass, k_gn orders 1-4, visibility prescreen, "
                                               "refinement", "ms": solve_avg_ms, "fp32_flops": flops,
                                    "frac": achieved / peak_max,
                                    "traffic": profile_traffic("mpt_solve") if args.rx_side == 32 else None},
                     "fp32_minimiser": {"kernel": "MPT_FP32 solve call: exclusion pass and k_gn orders 1-4 (no prescreen "
                                                  "or refinement)",
                                        "ms": float(np.median(mini_ms)), "fp32_flops": mini_flops,
                                        "achieved": mini_flops / (float(np.median(mini_ms)) * 1e-3) / 1e12,
                                        "frac": mini_flops / (float(np.median(mini_ms)) * 1e-3) / 1e12 / peak_max,
                                        "every_candidate_iterated": {
                                            "ms": float(np.median(all_ms)), "fp32_flops": all_flops,
                                            "frac": all_flops / (float(np.median(all_ms)) * 1e-3) / 1e12 / peak_max}}},
        "cuda_graph": graph_leg,
        "pruned_graph": pruned,
        "field": field_leg,
        "fp64_plain": {"ms_per_step": float(np.median(fp64_ms)),
                       "value": n_cand * ws / (float(np.median(fp64_ms)) * 1e-3), "unit": UNIT,
                       "valid_paths_per_step": n_valid_fp64},
        "e2e": {"value": n_cand * ws / (e2e_ms_step * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms_step,
                "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes), "steps": e2e_steps,
                "timing": "host wall clock over all steps, max over ranks",
                "pipeline": "scene resident; per step TX/RX host->device, paths and TX gradient device->host; "
                            "two contexts on two streams, one step's read-back beside the next step's kernels"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk | ({"sm_cycles_per_step": ms_per_step * 1e3 * clk["sm_mhz"]} if clk.get("sm_mhz") else {}),
        "workloads": legs,
        "wall_s_timed_region": t_wall,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_child(args.cpu_seconds, args.rx_side)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(sc, spec, seconds: float) -> dict:
    """The FP64 oracle, as it stands, on the host cores: whole sequences
    (x every RX) drawn at random from the workload until ~`seconds` pass."""
    import oracle

    table = oracle.enumerate_sequences(sc, 2, spec)
    rng = np.random.default_rng(7)
    order = rng.permutation(len(table))
    n_pairs = sc.n_pairs
    done = 0
    t0 = time.perf_counter()
    used = 0
    for e in order:
        b = int(e) * n_pairs
        oracle.candidate_range(sc, table, b, b + n_pairs)
        done += n_pairs
        used += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": oracle.threads(0), "kind": "oracle",
            "sample": f"{used} random sequences x {n_pairs} RX = {done} candidates of the workload "
                      f"(solve + validate), {dt:.1f} s"}


def cpu_baseline_child(seconds: float, rx_side: int) -> dict:
    """cpu_baseline in a fresh process, so that the oracle's threads share the
    host cores with nothing this process leaves running."""
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only", "--cpu-seconds",
                              str(seconds), "--rx-side", str(rx_side)], capture_output=True, text=True, check=True,
                             timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported in the line, never replaced by a number
        return {"error": f"{type(exc).__name__}: {exc}"[:300], "kind": "oracle"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    from paper_2301_06399_gb300 import scenes

    oracle.build()
    sc, spec = build_scene(0)
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_pairs = sc.n_pairs
    rng = np.random.default_rng(11)
    per_step = max(1, int(args.ref_entries))
    times = []
    done_total = 0
    for i in range(args.warmup + args.steps):
        ents = rng.choice(len(table), per_step, replace=False)
        t0 = time.perf_counter()
        for e in ents:
            b = int(e) * n_pairs
            oracle.candidate_range(sc, table, b, b + n_pairs)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            done_total += per_step * n_pairs
    total = sum(times)
    value = done_total / total
    cores = oracle.threads(0)
    sample = f"{per_step} random sequences x {n_pairs} RX per step (solve + validate)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "candidates_per_step": per_step * n_pairs,
                   "note": "FP64 CPU oracle (Gauss-Newton with backtracking, dual-number Jacobians) on the host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the per-workload legs")
    ap.add_argument("--no-tune", action="store_true", help="library default schedule instead of mpt_autotune")
    ap.add_argument("--ref-entries", type=int, default=64)
    ap.add_argument("--rx-side", type=int, default=32, help="RX grid side (32 = the benchmark workload)")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_baseline_only:
        import oracle

        oracle.build()
        sc, spec = build_scene(0, args.rx_side)
        print(json.dumps(cpu_baseline(sc, spec, args.cpu_seconds)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

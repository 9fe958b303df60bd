"""Benchmark of the light-field SGM depth path on GB300.

One step = the whole method on one 9x9 x 512x512 light field already resident in HBM:
initial disparity (census, per-arm cost, integer SGM, WTA, fusion, hole filling,
windows), bounded cost volume, bounded 8-path SGM, WTA + sub-pixel.  The headline
metric is the time of the cost volume + SGM stages per light field (the paper's final
map stage, Sec. III-E); the full-step time is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload bench|plenoptic|tiny|epfl|middlebury] [--channels 1|3]

Beside it: the training pattern (forward + hand-written backward, soft-argmin) and the
serving pattern (64 mixed light fields as one CUDA-graph launch against sequential launches).

N > 1 is launched with torchrun: every rank runs its own light field (independent
replicas, no collective on the data path), the step time is the max over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a row band of the
same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per 9x9x512^2 light field (cost+SGM)"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128      # 4 sub-partitions x 32 lanes issue one 32-bit lane op each per clock
L2_NOTE = "GPU arm: L2 flushed (256 MB write) before every step; CPU arm: not applicable"
PENALTY_NOTE = "P1 = 0.05 mean cost, P2 = 0.5 mean cost (coarse: per arm, integer)"


# DRAM bytes (read + write) per launch from one ncu capture of the bench workload, with the
# SHA-256 prefix of the kernel's source at capture time; a changed source reports null.
NCU_TRAFFIC = {
    "fine_cost": {"bytes": 324262400, "workload": "bench", "channels": 1,
                  "source": "paper_1907_13449_gb300/csrc/k_fine_cost.cu",
                  "sha256_16": "50737e8b0a1d0d04"},
}


def ncu_traffic(kernel, workload_name="bench", channels=1):
    import hashlib
    e = NCU_TRAFFIC.get(kernel)
    if not e or e["workload"] != workload_name or e["channels"] != channels:
        return None
    try:
        with open(os.path.join(ROOT, e["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return e["bytes"] if h == e["sha256_16"] else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name, lf_index, channels=1):
    import lfsynth
    if channels == 1:
        return lfsynth.WORKLOADS[name](lf_index)
    return lfsynth.WORKLOADS[name](lf_index, params=lfsynth.PARAMS[name](channels=channels))


def workload_label(p):
    colour = " RGB" if p.channels == 3 else ""
    return (f"{p.name}: {p.U}x{p.V} views of {p.H}x{p.W}{colour} f32, census {p.census_w}x{p.census_w}, "
            f"coarse {p.coarse_labels} labels on [{p.dmin:g},{p.dmax:g}], fine window 2x{p.fine_radius}+1 "
            f"of {p.fine_labels} labels, {p.paths}-path SGM, parabolic sub-pixel")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline models
def hbm_bytes_cost_sgm(p, nnz_active):
    """Algorithmic bytes of the cost volume + SGM stages: each reads its inputs once and
    writes its outputs once (views; window map lo/cnt/off 16 B per pixel per stage;
    cost written and read once; aggregated cost written once)."""
    N = p.H * p.W
    views = p.U * p.V * p.channels * N * 4
    cost = 4 * nnz_active
    return {"cost_volume": views + 16 * N + cost, "sgm_aggregate": 16 * N + cost + cost}


def alu_ops_per_cell_view(p):
    """Algorithmic 32-bit lane operations per (active cell, non-reference view) of the cost volume:
    per channel a bilinear sample at 4 ops (one horizontal and one vertical lerp of 2 ops each, the
    other row's horizontal lerp being shared with the adjacent row), the difference, and its
    absolute-value accumulation -- 6 ops, the upper end of the 4-6 instructions per sample of the
    algorithmic count -- or for colour the squared accumulation of each channel's difference plus
    one square root and one add per view.  The census term is left out: Hamming distances are
    piecewise constant in the label, so only the distinct nearest offsets of a window need a
    popcount (a few per pixel and view, under a tenth of the l2 work)."""
    return 6 * p.channels + (2 if p.channels > 1 else 0)


def alu_ops_cost(p, nnz_active):
    return nnz_active * (p.U * p.V - 1) * alu_ops_per_cell_view(p)


ROW_KW = 36      # default label span of the row cost kernel's ranges (36 or 44, lfsgm_set_tuning)


def row_kernel_cells(lo, cnt, H, W, kw=ROW_KW):
    """Cells the row cost kernel computes (the rest go to the list kernel): per run of 32 pixels
    of a row it takes the kw-label range [g0, g0 + kw) that holds the most windows of at most 32
    labels (ties: the lowest start, candidates in lane order) and computes the windows inside it --
    the kernel's own selection, replayed on the host from the window map."""
    import numpy as np
    lo = lo.reshape(H, W).astype(np.int64)
    cnt = cnt.reshape(H, W).astype(np.int64)
    Wt = (W + 31) // 32 * 32
    l = np.zeros((H, Wt), np.int64)
    n = np.zeros((H, Wt), np.int64)
    l[:, :W], n[:, :W] = lo, cnt
    l, n = l.reshape(-1, 32), n.reshape(-1, 32)
    nar = (n >= 1) & (n <= 32)
    best = np.full(l.shape[0], -1)
    g0 = np.zeros(l.shape[0], np.int64)
    for c in range(32):
        cl = l[:, c]
        fit = (nar & (l >= cl[:, None]) & (l + n <= cl[:, None] + kw)).sum(1)
        take = nar[:, c] & ((fit > best) | ((fit == best) & (cl < g0)))
        best = np.where(take, fit, best)
        g0 = np.where(take, cl, g0)
    fits = nar & (l >= g0[:, None]) & (l + n <= g0[:, None] + kw) & (best[:, None] > 0)
    return int((n * fits).sum())


def max_over_ranks(vals, ws, device):
    """Element-wise max of per-rank timings (the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def ms_per_lf(stage_ms, steps, ws):
    """Whole-job ms per light field: ws replicas each ran `steps` light fields in stage_ms."""
    return stage_ms / (steps * ws)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1907_13449_gb300 as lf

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = lf.load()
    views_np, gt, p = workload(args.workload, rank, args.channels)
    views = torch.from_numpy(views_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    L = lf.LightFieldDepth(p, stream=stream, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # the library's autotuner picks the speed knobs for this shape (untimed)
    row_kw, list_ctas = lf.lfsgm_autotune(L.h, views) if args.autotune else (36, 0)
    if args.sgm_warps is not None:
        lf.lfsgm_set_sgm_warps(L.h, args.sgm_warps)
    if args.sgm_split is not None:
        lf.lfsgm_set_sgm_split(L.h, args.sgm_split)
    knob_note = ("speed knobs picked by lfsgm_autotune on this light field before the timed region"
                 if args.autotune else "the library's default speed knobs (no autotuning)")
    if args.sgm_warps is not None or args.sgm_split is not None:
        knob_note += "; SGM knobs fixed on the command line"
    sgm_warps = lf.lfsgm_get_tuning(L.h)[2]
    sgm_split = lf.lfsgm_get_sgm_split(L.h)

    def step(events=None):
        L.initial(views)
        if events:
            events[0].record(stream)
        L.cost_volume(views)
        L.aggregate(-1.0, -1.0)
        if events:
            events[1].record(stream)
        L.wta()

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    nnz = int(L.off[-1].item())
    cnt = L.cnt.cpu().numpy()
    active = int(cnt.sum())
    row_cells = row_kernel_cells(L.lo.cpu().numpy(), cnt, p.H, p.W, row_kw)

    lf.lfsgm_set_profiling(L.h, True)
    lf.lfsgm_kernel_times(L.h)          # drop anything recorded so far
    launches0 = lf.lfsgm_launch_count(L.h)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    stage_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            step_ev[i][0].record(stream)
            step(stage_ev[i])
            step_ev[i][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = lf.lfsgm_launch_count(L.h) - launches0
    ktimes = lf.lfsgm_kernel_times(L.h, cap=100000)
    lf.lfsgm_set_profiling(L.h, False)
    step_ms = sum(a.elapsed_time(b) for a, b in step_ev)
    stage_each = sorted(a.elapsed_time(b) for a, b in stage_ev)
    stage_ms = sum(stage_each)
    step_ms, stage_ms = max_over_ranks([step_ms, stage_ms], ws, dev)

    # per-kernel aggregates over the timed region
    per = {}
    for name, ms in ktimes:
        a = per.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += ms
    kernels = {k: {"launches": v[0], "ms_total": round(v[1], 4), "ms_avg": round(v[1] / v[0], 5)}
               for k, v in sorted(per.items(), key=lambda kv: -kv[1][1])}

    # the paper's 16 SGM directions (Sec. IV-C) on the same light field: cost + SGM per step
    import dataclasses
    L16 = lf.LightFieldDepth(dataclasses.replace(p, paths=16), stream=stream, device=dev)
    L16.initial(views)
    for _ in range(2):
        L16.cost_volume(views)
        L16.aggregate(-1.0, -1.0)
    e16 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a, b in e16:
        flush.zero_()
        a.record(stream)
        L16.cost_volume(views)
        L16.aggregate(-1.0, -1.0)
        b.record(stream)
    torch.cuda.synchronize()
    paths16_ms = statistics.median(a.elapsed_time(b) for a, b in e16)
    L16.close()

    # the paper's post-processing median (Sec. III-F), timed on its own
    med = torch.empty_like(L.disp)
    for _ in range(3):
        lf.lfsgm_median_filter(L.h, L.disp, med)
    me0, me1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    me0.record(stream)
    for _ in range(20):
        lf.lfsgm_median_filter(L.h, L.disp, med)
    me1.record(stream)
    torch.cuda.synchronize()
    median_ms = me0.elapsed_time(me1) / 20

    # end to end through the host-buffer entry point (pinned host memory)
    vh = torch.from_numpy(views_np).pin_memory()
    dh = torch.empty(p.H * p.W, dtype=torch.float32).pin_memory()
    lh = torch.empty(p.H * p.W, dtype=torch.int32).pin_memory()
    for _ in range(max(1, args.warmup)):
        lf.lfsgm_depth_host(L.h, vh, dh, lh)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lf.lfsgm_depth_host(L.h, vh, dh, lh)
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.mean(e2e)
    # accuracy of the disparity map against the scene's ground truth (Sec. IV-B measures)
    from paper_1907_13449_gb300 import quality
    margin = int(np.ceil(max(p.U - 1 - p.uc, p.uc, p.V - 1 - p.vc, p.vc) * max(abs(p.dmin), abs(p.dmax)))) \
        + p.census_w // 2
    qual = {"all_pixels": quality.report(dh.numpy(), gt, e2e_ms * 1e-3),
            "interior": quality.report(dh.numpy(), gt, e2e_ms * 1e-3, margin=margin),
            "note": "BadPix(0.07) in %, MSE x 100, M = (100 - BadPix) / e2e runtime (Eq. 14); synthetic "
                    "ground truth of the rendered scene; interior = pixels farther than max shift + census "
                    "half-width from the border"}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    peaks = load_peaks()
    clocks = clk.summary()
    K = args.steps
    value = ms_per_lf(stage_ms, K, ws)          # whole-job ms per light field (cost+SGM)
    # dominant kernel of the cost+SGM stages and its roofline
    hot = ["fine_cost", "fine_cost_wide", "fine_sgm", "census_all", "cost_partial_sums", "zero_agg", "sgm_split"]
    if "fine_cost" not in kernels:
        row_cells = 0                     # no row-kernel plan for this shape: every window in the list
    dom = max((k for k in kernels if k in hot), key=lambda k: kernels[k]["ms_total"])
    mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    by = hbm_bytes_cost_sgm(p, active)
    hbm_total = by["cost_volume"] + by["sgm_aggregate"]
    hbm_model_frac = round(hbm_total / (peaks["hbm_gbs"] * 1e9) * 1e3 / value, 4)
    if dom in ("fine_cost", "fine_cost_wide"):
        # the row kernel computes row_cells of the active cells, the list kernel the rest
        ops = alu_ops_cost(p, row_cells if dom == "fine_cost" else active - row_cells)
        peak_ops = n_sm * FP32_LANES_PER_SM * mhz * 1e6
        ach = ops / (kernels[dom]["ms_avg"] * 1e-3)
        roof = {"kernel": dom, "bound": "alu", "achieved": round(ach / 1e12, 3),
                "peak": round(peak_ops / 1e12, 3), "unit": "T 32-bit lane-ops/s",
                "cells": row_cells if dom == "fine_cost" else active - row_cells,
                "lane_ops_per_cell_view": alu_ops_per_cell_view(p),
                "frac": round(ach / peak_ops, 4), "traffic": ncu_traffic(dom, args.workload, p.channels),
                "algorithmic_bytes": by["cost_volume"],
                "sms": n_sm, "sm_mhz": mhz,
                "peak_basis": f"{n_sm} SMs (cudaDevAttrMultiProcessorCount) x {FP32_LANES_PER_SM} FP32 lanes x "
                              f"{mhz:.0f} MHz (median SM clock sampled during the timed region)",
                "hbm_frac_of_cost_sgm": hbm_model_frac}
    else:
        b = by["sgm_aggregate"] if dom == "fine_sgm" else by["cost_volume"]
        ach = b / (kernels[dom]["ms_avg"] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": ncu_traffic(dom, args.workload, p.channels)}
    hbm_model = {"bytes_per_lf": hbm_total, "roofline_ms": round(hbm_total / (peaks["hbm_gbs"] * 1e9) * 1e3, 4),
                 "frac": hbm_model_frac,
                 "peak_gbs": peaks["hbm_gbs"], "peak_source": peaks["_source"]}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(step_ms / K, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(p), "l2": L2_NOTE, "penalties": PENALTY_NOTE,
                   "parallelism": f"replicas x{ws}"},
        "gcell_per_s": round(active / (value * 1e-3) / 1e9, 2),
        "tuning": {"row_kw": row_kw, "list_ctas_per_sm": list_ctas, "sgm_warps": sgm_warps, "sgm_split": sgm_split,
                   "note": knob_note},
        "value_stats": {"median": round(statistics.median(stage_each), 4), "min": round(stage_each[0], 4),
                        "p99": round(stage_each[min(len(stage_each) - 1, int(0.99 * len(stage_each)))], 4),
                        "unit": "ms, cost+SGM per step on this rank"},
        "active_cells": active, "nnz_padded": nnz,
        "full_forward_ms_per_lf": round(step_ms / (K * ws), 4),
        "quality": qual,
        "paths16": {"cost_sgm_ms": round(paths16_ms, 4), "note": "the same light field with the paper's 16 SGM "
                    "directions (Sec. IV-C); the workload's configs use 8"},
        "post_filter": {"median3_ms": round(median_ms, 4), "note": "3x3 median of the disparity map, "
                        "Sec. III-F; not part of the timed step (off in the workload, as in its configs)"},
        "kernels": kernels,
        "roofline": roof,
        "hbm_model": hbm_model,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(views_np.nbytes),
                "d2h_bytes_per_step": int(dh.numel() * 4 + lh.numel() * 4),
                "scope": "per light field through lfsgm_depth_host: host->device views, the whole method "
                         "(initial pass, cost volume, SGM, WTA + sub-pixel), device->host disparity + label"},
    }
    if args.backward:
        out["backward"] = run_backward(args, dev, views, p)
    if args.batch_lfs > 0:
        out["batch"] = run_batch(args, dev)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, views_np, p, rows=args.cpu_rows)
    if ws > 1:
        dist.destroy_process_group()
    return out


def run_backward(args, dev, views, p):
    """Training pattern: forward (cost volume, SGM with fixed penalties recording its branches,
    soft-argmin) and the hand-written backward on that record (grad wrt cost, P1, P2 and views) on
    the same light field; beside it the inference forward with the backward that recomputes the
    SGM.  L2 flushed before every step."""
    import dataclasses

    import torch

    import paper_1907_13449_gb300 as lf
    q = dataclasses.replace(p, subpixel=2)
    L = lf.LightFieldDepth(q, device=dev)
    stream = L.stream
    L.initial(views)
    L.cost_volume(views)
    torch.cuda.synchronize()
    nnz = int(L.off[-1].item())
    active = int(L.cnt.sum().item())
    mean = float(L.cost[:nnz].double().sum().item()) / active     # padding slots hold 0
    P1, P2 = q.p1_frac * mean, q.p2_frac * mean
    gdisp = torch.randn(L.N, generator=torch.Generator(device=dev).manual_seed(5), device=dev)
    gcost = torch.empty_like(L.cost)
    gviews = torch.empty_like(views)
    gp = torch.zeros(2, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def fwd():
        L.cost_volume(views)
        lf.lfsgm_sgm_aggregate_record(L.h, L.cost, L.lo, L.cnt, L.off, P1, P2, L.agg)
        lf.lfsgm_wta_subpixel(L.h, L.agg, L.lo, L.cnt, L.off, None, L.disp)

    def bwd():
        lf.lfsgm_backward_recorded(L.h, views, L.cost, L.agg, L.lo, L.cnt, L.off, P1, P2, gdisp, gcost, gp[0:1],
                                   gp[1:2], gviews)

    def fwd_plain():
        L.cost_volume(views)
        L.aggregate(P1, P2)
        lf.lfsgm_wta_subpixel(L.h, L.agg, L.lo, L.cnt, L.off, None, L.disp)

    def bwd_plain():
        lf.lfsgm_backward(L.h, views, L.cost, L.lo, L.cnt, L.off, P1, P2, gdisp, gcost, gp[0:1], gp[1:2], gviews)

    K = max(3, args.steps // 4)

    def timed(f1, f2):
        for _ in range(args.warmup):
            flush.zero_()
            f1()
            f2()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            ev[i][0].record(stream)
            f1()
            ev[i][1].record(stream)
            f2()
            ev[i][2].record(stream)
        torch.cuda.synchronize()
        return (statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
                statistics.mean(e[1].elapsed_time(e[2]) for e in ev))

    f0, b0 = timed(fwd_plain, bwd_plain)
    f, b = timed(fwd, bwd)
    # per-kernel split of forward + backward (separate, untimed pass with the library's events)
    lf.lfsgm_set_profiling(L.h, True)
    lf.lfsgm_kernel_times(L.h)
    for _ in range(3):
        fwd()
        bwd()
    torch.cuda.synchronize()
    per = {}
    for name, ms in lf.lfsgm_kernel_times(L.h, cap=100000):
        per[name] = per.get(name, 0.0) + ms / 3
    lf.lfsgm_set_profiling(L.h, False)
    ok = bool(torch.isfinite(gviews).all().item() and torch.isfinite(gp).all().item())
    L.close()
    return {"config": "9x9x512x512, 31-label windows, soft-argmin tau 0.1, fixed P1/P2 = 0.05/0.5 mean cost",
            "forward_ms": round(f, 4), "backward_ms": round(b, 4), "steps": K,
            "backward_over_forward": round(b / f, 3), "train_step_ms": round(f + b, 4),
            "scope": "forward = cost volume + SGM recording its branches (lfsgm_sgm_aggregate_record) + "
                     "soft-argmin; backward = lfsgm_backward_recorded",
            "recompute": {"forward_ms": round(f0, 4), "backward_ms": round(b0, 4), "train_step_ms": round(f0 + b0, 4),
                          "scope": "forward = cost volume + lfsgm_sgm_aggregate + soft-argmin; backward = "
                                   "lfsgm_backward (runs the SGM again with its record)"},
            "grads_finite": ok,
            "kernels_ms": {k: round(v, 4) for k, v in sorted(per.items(), key=lambda kv: -kv[1])},
            "grads": "cost volume, P1, P2, views (l2 term through the bilinear weights)"}


def run_batch(args, dev):
    """Serving pattern: the mixed batch (4 shape classes, census 5/7, coarse labels 16..128)
    as one CUDA-graph launch, against the same light fields launched one after another."""
    import numpy as np
    import torch

    import lfsynth
    import paper_1907_13449_gb300 as lf
    n = args.batch_lfs
    t0 = time.perf_counter()
    lfs = [lfsynth.batch_lf(i, device=dev) for i in range(n)]
    gen_s = time.perf_counter() - t0
    params = [p for _, p in lfs]
    views = [v for v, _ in lfs]
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    B = lf.LightFieldBatch(params, views, branches=args.batch_branches, stream=stream)
    tune_s = time.perf_counter() - t0
    kw, lc, sw, sp = B.knobs()
    knobs = {}
    for i, p in enumerate(params):
        knobs.setdefault(lfsynth.BATCH_CLASSES[i % 4]["name"], set()).add((int(kw[i]), int(lc[i]), int(sw[i]), int(sp[i])))
    knobs = {k: sorted(v) for k, v in knobs.items()}
    for _ in range(2):
        B.run()
    torch.cuda.synchronize()
    R = max(3, args.steps // 10)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(R)]
    done, flight = [], []
    for i in range(R):
        ev[i][0].record(stream)
        B.run()
        ev[i][1].record(stream)
        s, e, k = B.times()
        done.append(e)
        flight.append(e - s)
    batch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    done = np.concatenate(done)
    flight = np.concatenate(flight)
    disp_b = [d.clone() for d in B.disp]
    nodes = B.kernel_nodes
    B.close()

    # sequential single-light-field launches on one stream (buffers allocated beforehand)
    hs = [lf.lfsgm_create(p, stream) for p in params]
    outs = [torch.empty(p.H * p.W, dtype=torch.float32, device=dev) for p in params]
    for h, v, o in zip(hs, views, outs):
        lf.lfsgm_depth(h, v, o, None)
    torch.cuda.synchronize()
    seq_total, seq_each, seq_done = [], [], []
    for _ in range(R):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        evs[0].record(stream)
        for i, (h, v, o) in enumerate(zip(hs, views, outs)):
            lf.lfsgm_depth(h, v, o, None)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        each = [evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
        seq_each += each
        seq_done += list(np.cumsum(each))
        seq_total.append(evs[0].elapsed_time(evs[n]))
    for h in hs:
        lf.lfsgm_destroy(h)
    # the batch and the sequential launches agree where the decision is clear
    diff = max(float(torch.quantile(torch.abs(a - b), 0.999).item()) for a, b in zip(disp_b, outs))
    seq_ms = statistics.mean(seq_total)
    pct = lambda a, q: round(float(np.percentile(a, q)), 3)
    return {"lfs": n, "classes": [c["name"] for c in lfsynth.BATCH_CLASSES],
            "branches": int(k), "graph_kernel_nodes": int(nodes), "runs": R,
            "knobs": {"per_class_row_kw_list_ctas_sgm_warps_split": knobs},
            "lf_per_s": round(n / (batch_ms * 1e-3), 1), "ms_per_batch": round(batch_ms, 3),
            "p50_ms": pct(done, 50), "p99_ms": pct(done, 99),
            "latency": "completion time of each light field after the batch starts (all submitted at once)",
            "in_flight_p50_ms": pct(flight, 50), "in_flight_p99_ms": pct(flight, 99),
            "sequential": {"lf_per_s": round(n / (seq_ms * 1e-3), 1), "ms_total": round(seq_ms, 3),
                           "p50_ms": pct(seq_done, 50), "p99_ms": pct(seq_done, 99),
                           "per_lf_p50_ms": pct(seq_each, 50), "per_lf_p99_ms": pct(seq_each, 99)},
            "speedup_vs_sequential": round(seq_ms / batch_ms, 3),
            "disp_diff_p999_px": diff,
            "inputs": f"{sum(v.numel() for v in views) * 4 / 1e9:.2f} GB of views (larger than L2), "
                      f"rendered on the GPU in {gen_s:.1f} s; autotune + capture {tune_s:.1f} s"}


class OracleBand:
    """The oracle (FP64, OpenMP over rows) timed on the cost volume + SGM of a band of image
    rows of the light field; windows come from the oracle's own initial pass on the band
    (untimed, computed once per band height)."""

    def __init__(self, views_np, p):
        self.views_np, self.p, self.cache = views_np, p, {}

    def prepare(self, rows):
        import numpy as np

        import oracle
        if rows not in self.cache:
            p = self.p
            band = np.ascontiguousarray(self.views_np[..., :rows, :])     # [V][U]([C])[rows][W]
            q = type(p)(**{**p.__dict__, "H": rows})
            cfg = oracle.make_cfg(q)
            init = oracle.initial_disparity(cfg, band, None, q.p1_frac, q.p2_frac)
            self.cache[rows] = (band, q, cfg, init)
        return self.cache[rows]

    def run(self, rows):
        """Seconds of one timed pass over `rows` rows."""
        import oracle
        band, q, cfg, init = self.prepare(rows)
        t0 = time.perf_counter()
        off, cost = oracle.cost_volume(cfg, band, init["lo"], init["cnt"], init["census"])
        mean = float(cost.mean())
        oracle.sgm_bounded(q.H, q.W, init["lo"], init["cnt"], off, cost, q.p1_frac * mean, q.p2_frac * mean)
        return time.perf_counter() - t0


def cpu_baseline(args, views_np, p, rows, min_s=10.0, max_reps=20):
    """The oracle on `rows` rows of the same light field, repeated until at least `min_s`
    seconds of timed CPU work; ms per whole light field = mean pass time x H / rows."""
    import oracle
    ob = OracleBand(views_np, p)
    rows = max(1, min(rows, p.H))
    times = []
    while sum(times) < min_s and len(times) < max_reps:
        times.append(ob.run(rows))
    per = statistics.mean(times)
    cores = oracle.threads()
    # one thread (the paper's own set-up) on a smaller band
    rows1 = max(1, min(64, p.H))
    oracle.set_threads(1)
    try:
        t1 = ob.run(rows1)
    finally:
        oracle.set_threads(cores)
    return {"value": round(per * 1e3 * p.H / rows, 1), "unit": "ms", "cores": cores,
            "kind": "oracle",
            "sample": f"cost volume + SGM of rows 0..{rows - 1} of the light field (windows from the "
                      f"oracle's own initial pass, untimed), {len(times)} passes, {sum(times):.1f} s, "
                      f"scaled by {p.H}/{rows}",
            "single_thread": {"value": round(t1 * 1e3 * p.H / rows1, 1), "unit": "ms", "cores": 1,
                              "sample": f"rows 0..{rows1 - 1}, one pass, {t1:.1f} s, scaled by {p.H}/{rows1}"}}


def run_reference(args, ws, rank):
    """Reference arm: the oracle itself, each step a band of rows sized so that the whole
    --steps/--warmup run stays within about two minutes; value = ms per whole light field."""
    if rank != 0:
        return None
    import oracle
    views_np, gt, p = workload(args.workload, 0, args.channels)
    ob = OracleBand(views_np, p)
    cal_rows = min(32, p.H)
    t_cal = ob.run(cal_rows)
    per_row = t_cal / cal_rows
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows = int(max(8, min(p.H, budget / max(per_row, 1e-9))))
    rows = min(rows, p.H)
    for _ in range(args.warmup):
        ob.run(rows)
    samples = [ob.run(rows) for _ in range(args.steps)]
    v = statistics.mean(samples) * 1e3 * p.H / rows
    cb = {"value": round(v, 1), "unit": "ms", "cores": oracle.threads(), "kind": "oracle",
          "sample": f"each step: cost volume + SGM of rows 0..{rows - 1} (windows from the oracle's own "
                    f"initial pass, untimed), scaled by {p.H}/{rows}"}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(samples) * 1e3, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_label(p), "l2": L2_NOTE, "penalties": PENALTY_NOTE,
                                            "parallelism": "host cores"},
            "cpu_baseline": cb, "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bench", choices=["bench", "plenoptic", "tiny", "epfl", "middlebury"])
    ap.add_argument("--cpu-rows", type=int, default=512, help="image rows of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-lfs", type=int, default=64, help="light fields in the mixed batch (0: skip)")
    ap.add_argument("--batch-branches", type=int, default=0, help="concurrent branches (0: autotune)")
    ap.add_argument("--no-backward", dest="backward", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="default speed knobs instead of lfsgm_autotune (fixed kernel choice for profiling)")
    ap.add_argument("--sgm-warps", type=int, default=None, choices=[2, 4, 8],
                    help="fix the fine SGM's warps per CTA (after the autotuner, if it runs)")
    ap.add_argument("--sgm-split", type=int, default=None,
                    help="fix the fine SGM's split threshold (0: off; after the autotuner, if it runs)")
    ap.add_argument("--channels", type=int, default=1, choices=[1, 3],
                    help="colour channels of the rendered light field (3: RGB, Sec. III-B/C)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark: spin-images/s and culled point-pairs/s on one GB300, DLS vs STATIC.

Workload: the 100,000-point clustered heightfield (density varying 20:1 over
[0,1]^2, 32 Gaussian bumps), images for all points, W=32, B=0.01, support
angle 60 deg.  A step is one pass of the whole path with the inputs already
resident in HBM: mesh creation (normalise, bounding box), grid build
(counting sort), and the persistent spin kernel under one loop schedule.  Each
schedule (STATIC, SS, GSS, FAC) is timed for K steps after W warm-up steps;
the L2 cache is flushed (a 512 MB write) before every timed step.  `value` is
the best dynamic schedule.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU (no
data exchange: images are independent), timing is max over ranks and value
is the images of all ranks / that time ("weak" scaling).  ``--impl
reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (the only other place this script runs the oracle is the
cpu_baseline leg).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "spin-images/s & culled point-pairs/s on 1 GB300, DLS vs STATIC; p50/p99 latency"
UNIT = "spin-images/s"
SCHEDULES = ("STATIC", "SS", "GSS", "FAC")


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate_max_ms(local_ms, world):
    """Max of a per-rank time over all ranks (the slowest rank bounds the job)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, steps, world, max_ms):
    """Whole-job rate: the units every rank processed over the max-over-ranks time."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def _workload():
    from paper_1811_00901_gb300 import workloads as wl
    return wl.nonuniform_heightfield()


def _config(c, extra=None):
    d = {"workload": c["name"], "points": int(c["points"].shape[0]), "images": int(c["m"]), "W": int(c["W"]),
         "bin_size": float(c["bin_size"]), "support_angle_deg": 60.0,
         "density": "clustered heightfield, 20:1", "l2": "flushed (512 MB write) before each timed step",
         "inputs": "resident in HBM (device pointers)"}
    if extra:
        d.update(extra)
    return d


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "", 1).isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# roofline helpers
# --------------------------------------------------------------------------

def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def _group_cost_cov(examined_per_image):
    """sigma / mu of the per-group cost.  A group's cost follows its candidate
    stream, whose length every image of the group reports as its examined
    count, so the spread over images is the spread over groups."""
    e = np.asarray(examined_per_image, dtype=np.float64)
    return float(e.std() / max(e.mean(), 1e-30))


def sms_count(torch, dev):
    return torch.cuda.get_device_properties(dev).multi_processor_count


def _quartiles(xs):
    q = np.percentile(np.asarray(xs, dtype=np.float64), [25, 50, 75])
    return [float(v) for v in q]


def _peak_clocks(peaks, clk):
    """SM clocks to quote the ALU peak at: the maximum, the median seen during
    the timed region, and the median under a long power-capped load."""
    fs = [float(peaks.get("sm_max_mhz", 2070.0))]
    if clk and clk.get("sm_mhz"):
        fs.append(float(clk["sm_mhz"]))
    cul = peaks.get("clocks_under_load") or {}
    if cul.get("sm_mhz_median"):
        fs.append(float(cul["sm_mhz_median"]))
    return sorted(set(fs), reverse=True)


def _kernel_source_hash():
    h = hashlib.sha256()
    for name in ("spin_kernel.cu", "device_common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1811_00901_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _ncu_traffic(workload):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "spin_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("kernel_source_hash") != _kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# Algorithmic ALU work, per unit (lane-operations; an FMA counts once):
#   per culled pair (the candidate set, fl32 |X-P|^2 <= Rc2): difference d =
#   X - P (3), normal dot n.n_X (3), angle compare (1)                  -> 7
#   per angle-passing pair: beta = n.d (3), orthogonal part r = d - beta n
#   (3), alpha^2 = |r|^2 (3), u (1), row test (1), alpha = sqrt (1),
#   fixed-point column V (1), column test (1), fixed-point row U (1)   -> 15
#   per contributing pair: fraction split (2), product weight (2), the other
#   weights (3), row and column of the address (4), four shared-memory int32
#   atomics (4), count (1)                                              -> 16
# A coarser per-unit estimate (8 per culled pair, ~30 per angle-passing pair,
# 4 read-modify-writes + ~6 integer ops per in-support pair) gives a second
# figure, roofline["coarse_counts"].
OPS_PER_CULLED = 7
OPS_PER_ANGLE = 15
OPS_PER_SUPPORT = 16
COARSE_OPS = (8, 30, 10)


def alu_ops(n_culled, n_angle, n_support, counts=(OPS_PER_CULLED, OPS_PER_ANGLE, OPS_PER_SUPPORT)):
    return counts[0] * n_culled + counts[1] * n_angle + counts[2] * n_support


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args):
    import torch

    import paper_1811_00901_gb300 as spin
    from paper_1811_00901_gb300 import _build

    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    c = _workload()
    n, m, W, B, cs = c["points"].shape[0], c["m"], c["W"], float(c["bin_size"]), float(c["cos_s"])
    tp = torch.from_numpy(c["points"]).to(dev)
    tn = torch.from_numpy(c["normals"]).to(dev)
    out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def one_step(sched):
        mesh = spin.si_mesh_create(tp, tn, n, stream)
        spin.si_generate(mesh, None, m, W, B, cs, sched, out, stream)
        return mesh

    # ---- counts for the pair metrics (probe run, untimed)
    sched_probe = spin.make_schedule("GSS")
    mesh = spin.si_mesh_create(tp, tn, n, stream)
    culled = torch.zeros(m, dtype=torch.int64, device=dev)
    support = torch.zeros(m, dtype=torch.int64, device=dev)
    examined = torch.zeros(m, dtype=torch.int64, device=dev)
    angle = torch.zeros(m, dtype=torch.int64, device=dev)
    spin.si_generate_probe(mesh, None, m, W, B, cs, sched_probe, out, culled=culled, support=support,
                           examined=examined, angle=angle, stream=stream)
    torch.cuda.synchronize()
    spin.si_get_stats(mesh)
    spin.si_mesh_destroy(mesh)
    n_culled = int(culled.sum().item())
    n_support = int(support.sum().item())
    n_examined = int(examined.sum().item())
    n_angle = int(angle.sum().item())
    examined_per_image = examined.cpu().numpy()
    # measured shared-atomic peak (denominator of the splat roofline)
    atom_peak = spin.si_peak_smem_atomics(0, stream)
    atom_spread = spin.si_peak_smem_atomics(1, stream)
    # the autotuner's choice (untimed): rule, chunk, workers, group order and
    # launch shape, timed below as "tuned"
    mesh = spin.si_mesh_create(tp, tn, n, stream)
    tuned, tuned_ms = spin.si_tune_mesh(mesh, None, m, W, B, cs, out, reps=3, stream=stream)
    spin.si_mesh_destroy(mesh)
    # the paper's rules (and the extra runs below) at the library's default
    # shape, so that STATIC and the dynamic rules launch alike; "tuned" with
    # the tuner's own shape
    shape = {}
    configs = {name: spin.make_schedule(name, **shape) for name in SCHEDULES}
    configs["tuned"] = spin.make_schedule(tuned.kind, min_chunk=tuned.min_chunk, num_workers=tuned.num_workers,
                                          order=tuned.order, group=tuned.group, grid_div=tuned.grid_div)
    tuned_desc = {"kind": [k for k, v in spin.SCHED_NAMES.items() if v == tuned.kind][0],
                  "min_chunk": tuned.min_chunk, "num_workers": tuned.num_workers, "group": tuned.group,
                  "grid_div": tuned.grid_div,
                  "order": "decreasing estimated cost" if tuned.order else "grid"}

    results = {}
    clocks = ClockSampler(local)
    timed_launches = 0
    kernel_ms = {}
    clocks.start()
    for name, sched in configs.items():
        for _ in range(args.warmup):
            mesh = one_step(sched)
            stream.synchronize()
            spin.si_mesh_destroy(mesh)
        times = []
        kms = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            spin.si_set_timing(True)
            l0 = spin.si_kernel_launches()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mesh = one_step(sched)
            e1.record(stream)
            torch.cuda.synchronize()
            timed_launches += spin.si_kernel_launches() - l0
            spin.si_set_timing(False)
            st, _ = spin.si_get_stats(mesh)
            kms.append(st["kernel_ms"] / max(1, st["kernel_launches"]))
            spin.si_mesh_destroy(mesh)
            times.append(e0.elapsed_time(e1))
        total_ms = aggregate_max_ms(sum(times), world)
        results[name] = {"ms_per_step": total_ms / args.steps,
                         "images_per_s": job_throughput(m, args.steps, world, total_ms),
                         "culled_pairs_per_s": job_throughput(n_culled, args.steps, world, total_ms),
                         "kernel_ms": statistics.median(kms),
                         "kernel_ms_quartiles": _quartiles(kms),
                         "step_ms_quartiles": _quartiles(times),
                         "setup_ms": statistics.median([t - k for t, k in zip(times, kms)])}
        kernel_ms[name] = statistics.median(kms)
    clk = clocks.stop()

    dls = ["SS", "GSS", "FAC"] + (["tuned"] if tuned_desc["kind"] != "STATIC" else [])
    best = max(dls, key=lambda k: results[k]["images_per_s"])
    r = results[best]

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if rank == 0 or world > 1:
        hp = torch.from_numpy(c["points"]).pin_memory()
        hn = torch.from_numpy(c["normals"]).pin_memory()
        hout = torch.empty((m, W, W), dtype=torch.int32).pin_memory()
        sched = configs[best]
        for _ in range(max(1, args.warmup)):
            spin.si_generate_host(hp, hn, n, None, m, W, B, cs, sched, hout, stream)
        et = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            spin.si_generate_host(hp, hn, n, None, m, W, B, cs, sched, hout, stream)
            et.append(time.perf_counter() - t0)
        # whole job: every rank's images over the slowest rank's time
        e2e_ms = aggregate_max_ms(1e3 * sum(et), world) / args.steps
        e2e = {"value": job_throughput(m, 1, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(2 * n * 3 * 4),
               "d2h_bytes_per_step": int(m * W * W * 4), "ms_per_step": e2e_ms,
               "api": "si_generate_host (host buffers; mesh/grid build inside; the kernel writes the images "
                      "straight into the page-locked host output)"}

    # ---- roofline of the spin kernel (the dominant kernel)
    peaks, peak_src = _measured_peaks()
    f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = sms_count(torch, dev)
    alu_peak = sms * 128 * f_mhz * 1e6  # lane-ops/s at the maximum SM clock
    ops = alu_ops(n_culled, n_angle, n_support)
    k_ms = kernel_ms[best]
    achieved = ops / (k_ms / 1e3)
    achieved_s = alu_ops(n_culled, n_angle, n_support, COARSE_OPS) / (k_ms / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12, "unit": "Tlane-op/s",
                "frac": achieved / alu_peak, "traffic": _ncu_traffic(c["name"]),
                "kernel": "spin_kernel (persistent, %s)" % best, "kernel_ms": k_ms,
                "peak_source": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)" % (sms, f_mhz, peak_src),
                "ops_per_culled_pair": OPS_PER_CULLED, "ops_per_angle_pair": OPS_PER_ANGLE,
                "ops_per_support_pair": OPS_PER_SUPPORT,
                "coarse_counts": {"ops_per_culled_pair": COARSE_OPS[0], "ops_per_angle_pair": COARSE_OPS[1],
                                  "ops_per_support_pair": COARSE_OPS[2], "achieved": achieved_s / 1e12,
                                  "frac": achieved_s / alu_peak},
                "peak_at_clocks": {"%.0f_mhz" % f: {"peak": sms * 128 * f * 1e6 / 1e12,
                                                    "frac": achieved / (sms * 128 * f * 1e6)}
                                   for f in _peak_clocks(peaks, clk)},
                "write_gbs": m * W * W * 4 / (k_ms / 1e3) / 1e9,
                "write_frac_of_hbm": (m * W * W * 4 / (k_ms / 1e3) / 1e9) / float(peaks.get("hbm_gbs", 6800.0)),
                "smem_atomics": {"achieved_per_s": 4 * n_support / (k_ms / 1e3),
                                 "peak_per_s": atom_peak, "frac": 4 * n_support / (k_ms / 1e3) / atom_peak,
                                 "spread_pattern_per_s": atom_spread,
                                 "peak_source": "measured (si_peak_smem_atomics, conflict-free)"}}

    line = {"metric": METRIC, "value": r["images_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(c, {"schedule": best, "tuned": tuned_desc, "shape": shape or "library default",
                                  "parallelism": "replicas" if world > 1 else "single GPU"}),
            "culled_pairs_per_s": r["culled_pairs_per_s"], "culled_pairs_per_step": n_culled,
            "support_pairs_per_step": n_support, "examined_pairs_per_step": n_examined,
            "angle_pairs_per_step": n_angle,
            "stencil_overhead": n_examined / max(1, n_culled),
            "by_schedule": {k: {"images_per_s": v["images_per_s"], "ms_per_step": v["ms_per_step"],
                                "kernel_ms": v["kernel_ms"], "kernel_ms_quartiles": v["kernel_ms_quartiles"],
                                "step_ms_quartiles": v["step_ms_quartiles"],
                                "mesh_and_grid_ms": v["setup_ms"]} for k, v in results.items()},
            "dls_over_static": r["images_per_s"] / results["STATIC"]["images_per_s"],
            "e2e": e2e, "roofline": roofline,
            "gpu_launches": int(timed_launches), "clocks": clk}
    if not args.no_extra:
        from paper_1811_00901_gb300 import workloads as wl
        import tempfile
        # the tuning table as tuned on the bench workload; the sphere and scene
        # tunings below add their own size classes, which the batched run
        # (one rule per item from the nearest class) should not inherit
        table = os.path.join(tempfile.mkdtemp(), "tuning.json")
        spin.si_tune_save(table)
        ex_steps = args.steps
        extra = {}
        sph = wl.plain_sphere()
        sph_tuned = _tuned_schedule(spin, torch, dev, sph, stream)
        extra["sphere-4096-W16"] = bench_single(spin, torch, dev, sph, args.steps, args.warmup, flush, stream,
                                                scheds=dict({k: spin.make_schedule(k) for k in
                                                             ("STATIC", "SS", "GSS", "FAC")}, tuned=sph_tuned),
                                                pairs=True)
        extra["sphere-4096-W16"]["tuned"] = {
            "kind": [k for k, v in spin.SCHED_NAMES.items() if v == sph_tuned.kind][0],
            "min_chunk": sph_tuned.min_chunk, "num_workers": sph_tuned.num_workers, "group": sph_tuned.group,
            "grid_div": sph_tuned.grid_div, "order": sph_tuned.order}
        scn = wl.large_scene()
        scn_tuned = _tuned_schedule(spin, torch, dev, scn, stream, reps=3)
        extra["scene-1M-W64"] = bench_single(spin, torch, dev, scn, ex_steps, args.warmup, flush, stream,
                                             scheds=dict({k: spin.make_schedule(k) for k in
                                                          ("STATIC", "SS", "GSS", "FAC")}, tuned=scn_tuned),
                                             pairs=True, e2e=True)
        extra["scene-1M-W64"]["tuned"] = {
            "kind": [k for k, v in spin.SCHED_NAMES.items() if v == scn_tuned.kind][0],
            "min_chunk": scn_tuned.min_chunk, "num_workers": scn_tuned.num_workers, "group": scn_tuned.group,
            "grid_div": scn_tuned.grid_div, "order": scn_tuned.order}
        # probabilistic factoring with sigma / mu of the group cost measured by
        # the probe run (a group's cost follows its candidate stream length)
        cov = _group_cost_cov(examined_per_image)
        extra["factoring-heightfield-100k-W32"] = dict(
            bench_single(spin, torch, dev, c, ex_steps, args.warmup, flush, stream, scheds={
                "FAC": spin.make_schedule("FAC", **shape),
                "FAC_PROB": spin.make_schedule("FAC_PROB", fac_cov=cov, **shape),
                "AWF": spin.make_schedule("AWF", **shape),
                "AF": spin.make_schedule("AF", **shape)}), fac_cov=cov)
        # heterogeneity emulation (Sec. 5.2's Type2 + Type1 runs): the first half
        # of the resident workers 3x slower, and they request first
        P = spin.si_default_workers(c["W"], spin.make_schedule("FAC", **shape))
        het = {k: spin.make_schedule(k, num_workers=P, slow_workers=P // 2, slowdown=3.0, fac_cov=cov, **shape)
               for k in ("STATIC", "SS", "GSS", "FAC", "FAC_PROB", "AWF", "AF")}
        for k in ("SS", "FAC", "AWF"):
            het[k + "+cost order"] = spin.make_schedule(k, num_workers=P, slow_workers=P // 2, slowdown=3.0,
                                                        order=1, **shape)
        h = bench_single(spin, torch, dev, c, ex_steps, args.warmup, flush, stream, scheds=het)
        h["emulation"] = {"workers": P, "slow_workers": P // 2, "slowdown": 3.0, "slow_request_first": True}
        h["over_static"] = {k: v["images_per_s"] / h["by_schedule"]["STATIC"]["images_per_s"]
                            for k, v in h["by_schedule"].items()}
        extra["heterogeneous-heightfield-100k-W32"] = h
        extra["trace-heightfield-100k-W32"] = bench_trace(spin, torch, dev, c, shape, stream)
        extra["trace-heterogeneous-heightfield-100k-W32"] = bench_trace(
            spin, torch, dev, c, shape, stream, het=dict(num_workers=P, slow_workers=P // 2, slowdown=3.0))
        extra["matching-16k-vs-100k-W32"] = bench_matching(spin, torch, dev, c, ex_steps, args.warmup, stream)
        # Algorithm 1's own nearest-bin count on the bench workload
        extra["nearest-bin-heightfield-100k-W32"] = bench_single(
            spin, torch, dev, c, ex_steps, args.warmup, flush, stream,
            scheds={k: spin.make_schedule(k, binning="NEAREST") for k in ("STATIC", "FAC")})
        del out
        torch.cuda.empty_cache()
        spin.si_tune_clear()
        spin.si_tune_load(table)
        # one batched step writes 140 GB of images (about a second): 7 timed steps
        extra["batched-512-spheres"] = bench_batched(spin, torch, dev, min(ex_steps, 7), args.warmup, stream)
        torch.cuda.empty_cache()
        extra["serving-64-meshes"] = bench_serving(spin, torch, dev, args.serve_requests, args.serve_pool)
        line["workloads"] = extra
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(c, budget_s=args.cpu_seconds)
        line["cpu_baseline"]["host"] = _host_cpu()
        line["cpu_dls_baseline"] = cpu_dls_baseline(c)
        line["cpu_oracle_other_workloads"] = cpu_oracle_other_workloads()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# the other workloads (secondary keys of the same line)
# --------------------------------------------------------------------------

def bench_single(spin, torch, dev, c, steps, warmup, flush, stream, kinds=("STATIC", "FAC"), scheds=None,
                 pairs=False, e2e=False):
    """One mesh, all its images (or its query list), per rule; step and kernel
    time by events (medians and quartiles over `steps`).  ``scheds`` (name ->
    si_schedule) replaces ``kinds`` when given.  With ``pairs`` a probe run
    counts the pairs and the line carries the kernel's ALU roofline; with
    ``e2e`` the best rule is timed again through si_generate_host from
    page-locked host buffers."""
    n, m, W, B, cs = c["points"].shape[0], c["m"], c["W"], float(c["bin_size"]), float(c["cos_s"])
    tp = torch.from_numpy(c["points"]).to(dev)
    tn = torch.from_numpy(c["normals"]).to(dev)
    tq = None if c["query_idx"] is None else torch.from_numpy(c["query_idx"]).to(dev)
    out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    res = {}
    if scheds is None:
        scheds = {kind: spin.make_schedule(kind) for kind in kinds}
    for kind, sched in scheds.items():
        times, kms = [], []
        for k in range(warmup + steps):
            flush.zero_()
            torch.cuda.synchronize()
            spin.si_set_timing(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mesh = spin.si_mesh_create(tp, tn, n, stream)
            spin.si_generate(mesh, tq, m, W, B, cs, sched, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            spin.si_set_timing(False)
            st, _ = spin.si_get_stats(mesh)
            spin.si_mesh_destroy(mesh)
            if k >= warmup:
                times.append(e0.elapsed_time(e1))
                kms.append(st["kernel_ms"] / max(1, st["kernel_launches"]))
        res[kind] = {"images_per_s": m / (statistics.median(times) / 1e3), "ms_per_step": statistics.median(times),
                     "kernel_ms": statistics.median(kms), "kernel_ms_quartiles": _quartiles(kms),
                     "step_ms_quartiles": _quartiles(times)}
    line = {"images": m, "W": W, "points": n, "steps": steps, "by_schedule": res}
    best = max(res, key=lambda k: res[k]["images_per_s"])
    if pairs:
        # pair counts from one probe run (untimed): the kernel's ALU roofline here
        mesh = spin.si_mesh_create(tp, tn, n, stream)
        culled = torch.zeros(m, dtype=torch.int64, device=dev)
        support = torch.zeros(m, dtype=torch.int64, device=dev)
        examined = torch.zeros(m, dtype=torch.int64, device=dev)
        angle = torch.zeros(m, dtype=torch.int64, device=dev)
        spin.si_generate_probe(mesh, tq, m, W, B, cs, spin.make_schedule("GSS"), out, culled=culled,
                               support=support, examined=examined, angle=angle, stream=stream)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
        spin.si_mesh_destroy(mesh)
        nc, ns, ne, na = (int(t.sum().item()) for t in (culled, support, examined, angle))
        peaks, src = _measured_peaks()
        f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        alu_peak = sms_count(torch, dev) * 128 * f_mhz * 1e6
        k_s = res[best]["kernel_ms"] / 1e3
        line.update(culled_pairs_per_step=nc, angle_pairs_per_step=na, support_pairs_per_step=ns,
                    examined_pairs_per_step=ne, stencil_overhead=ne / max(1, nc),
                    culled_pairs_per_s=nc / (res[best]["ms_per_step"] / 1e3),
                    roofline={"bound": "alu", "unit": "Tlane-op/s", "rule": best, "kernel_ms": res[best]["kernel_ms"],
                              "achieved": alu_ops(nc, na, ns) / k_s / 1e12, "peak": alu_peak / 1e12,
                              "frac": alu_ops(nc, na, ns) / k_s / alu_peak,
                              "coarse_counts": {"achieved": alu_ops(nc, na, ns, COARSE_OPS) / k_s / 1e12,
                                                "frac": alu_ops(nc, na, ns, COARSE_OPS) / k_s / alu_peak},
                              "peak_source": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)" % (
                                  sms_count(torch, dev), f_mhz, src),
                              "write_gbs": m * W * W * 4 / k_s / 1e9})
    del out
    if e2e:
        hp = torch.from_numpy(c["points"]).pin_memory()
        hn = torch.from_numpy(c["normals"]).pin_memory()
        hq = None if c["query_idx"] is None else torch.from_numpy(c["query_idx"]).pin_memory()
        hout = torch.empty((m, W, W), dtype=torch.int32).pin_memory()
        sched = scheds[best]
        et = []
        for k in range(warmup + steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            spin.si_generate_host(hp, hn, n, hq, m, W, B, cs, sched, hout, stream)
            if k >= warmup:
                et.append(time.perf_counter() - t0)
        ms = 1e3 * statistics.median(et)
        line["e2e"] = {"value": m / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                       "ms_quartiles": _quartiles([1e3 * t for t in et]), "rule": best,
                       "h2d_bytes_per_step": int(2 * n * 3 * 4 + (0 if hq is None else 4 * m)),
                       "d2h_bytes_per_step": int(m * W * W * 4),
                       "api": "si_generate_host (host buffers; mesh/grid build inside; page-locked output "
                              "written by the kernel)"}
        del hout
    return line


def bench_trace(spin, torch, dev, c, shape, stream, het=None):
    """Each worker's finishing time under STATIC and the dynamic rules (the GPU
    analogue of the per-rank finishing times of the paper's Fig. 2): one traced
    run per rule (si_generate_traced, %globaltimer at every claim); times from
    the first claim's start.  With ``het`` the heterogeneity emulation's
    schedule fields are applied."""
    n, m, W, B, cs = c["points"].shape[0], c["m"], c["W"], float(c["bin_size"]), float(c["cos_s"])
    tp = torch.from_numpy(c["points"]).to(dev)
    tn = torch.from_numpy(c["normals"]).to(dev)
    out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    mesh = spin.si_mesh_create(tp, tn, n, stream)
    res = {}
    try:
        for name in ("STATIC", "SS", "GSS", "FAC", "AWF", "AF", "SS+cost order", "FAC+cost order", "AWF+cost order"):
            kind = name.split("+")[0]
            sched = spin.make_schedule(kind, order=1 if "+" in name else 0, **shape, **(het or {}))
            P = spin.si_default_workers(W, sched) if not het else het["num_workers"]
            claims = torch.zeros((200000, 4), dtype=torch.int64, device=dev)
            count = torch.zeros(1, dtype=torch.int64, device=dev)
            spin.si_generate(mesh, None, m, W, B, cs, sched, out, stream)  # grid and warm-up
            spin.si_generate_traced(mesh, None, m, W, B, cs, sched, out, claims, count, stream)
            torch.cuda.synchronize()
            nc = min(int(count.item()), claims.shape[0])
            tr = claims[:nc].cpu().numpy()
            t0 = tr[:, 2].min()
            finish = np.zeros(P)
            busy = np.zeros(P)
            for w, _, a, b in tr:
                finish[w] = max(finish[w], (b - t0) / 1e6)
                busy[w] += (b - a) / 1e6
            res[name] = {"claims": nc, "workers": int(P), "finish_ms_max": float(finish.max()),
                         "finish_ms_mean": float(finish.mean()), "finish_ms_min": float(finish.min()),
                         "finish_quartiles_ms": _quartiles(finish),
                         "imbalance": float((finish.max() - finish.mean()) / finish.max()),
                         "busy_ms_mean": float(busy.mean())}
        spin.si_get_stats(mesh)
    finally:
        spin.si_mesh_destroy(mesh)
    return {"workload": c["name"], "by_schedule": res,
            "note": "imbalance = (latest - mean finishing time) / latest finishing time of the workers"}


def _tuned_schedule(spin, torch, dev, c, stream, reps=5):
    """The autotuner's choice for workload c (untimed; on its own mesh)."""
    n, m, W = c["points"].shape[0], c["m"], c["W"]
    tq = None if c["query_idx"] is None else torch.from_numpy(c["query_idx"]).to(dev)
    mesh = spin.si_mesh_create(torch.from_numpy(c["points"]).to(dev), torch.from_numpy(c["normals"]).to(dev), n,
                               stream)
    out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    try:
        best, _ = spin.si_tune_mesh(mesh, tq, m, W, float(c["bin_size"]), float(c["cos_s"]), out, reps=reps,
                                    stream=stream)
    finally:
        spin.si_mesh_destroy(mesh)
    return best


def _matching_inputs(spin, torch, dev, c, n_scene, stream):
    """The matching workload: every image of the bench mesh (the model) and
    n_scene images of a rigidly moved copy of it at randomly drawn points (the
    scene); returns (scene, model, the drawn point of each scene image)."""
    n, m, W, B, cs = c["points"].shape[0], c["m"], c["W"], float(c["bin_size"]), float(c["cos_s"])
    tp = torch.from_numpy(c["points"]).to(dev)
    tn = torch.from_numpy(c["normals"]).to(dev)
    model = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    mesh = spin.si_mesh_create(tp, tn, n, stream)
    spin.si_generate(mesh, None, m, W, B, cs, spin.make_schedule("FAC"), model, stream)
    torch.cuda.synchronize()
    spin.si_mesh_destroy(mesh)
    g = torch.Generator().manual_seed(1811009021)
    rot, _ = torch.linalg.qr(torch.randn(3, 3, generator=g, dtype=torch.float64))
    rot = rot.to(torch.float32).to(dev)
    mesh = spin.si_mesh_create((tp @ rot.T + 0.25).contiguous(), (tn @ rot.T).contiguous(), n, stream)
    q = torch.randperm(m, generator=g)[:n_scene].to(torch.int32).to(dev)
    scene = torch.empty((n_scene, W, W), dtype=torch.int32, device=dev)
    spin.si_generate(mesh, q, n_scene, W, B, cs, spin.make_schedule("FAC"), scene, stream)
    torch.cuda.synchronize()
    spin.si_mesh_destroy(mesh)
    return scene, model, q


def bench_matching(spin, torch, dev, c, steps, warmup, stream, n_scene=16384, k=5):
    """Spin-image matching: n_scene images of a rigidly moved copy of the bench
    mesh against all images of the mesh (correlation over all bins, k best)."""
    m, W = c["m"], c["W"]
    scene, model, q = _matching_inputs(spin, torch, dev, c, n_scene, stream)
    idx = torch.empty((n_scene, k), dtype=torch.int32, device=dev)
    val = torch.empty((n_scene, k), dtype=torch.float32, device=dev)
    peaks, src = _measured_peaks()
    res = {}
    kp = (W * W + 63) // 64 * 64
    for prec, ksplit in (("BF16", 1), ("FP32", 6)):
        times = []
        for it in range(warmup + steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            spin.si_match(scene, n_scene, model, m, W, k, prec, idx, val, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= warmup:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        # the correlation's algorithmic flops, and the BF16 tensor-core flops
        # the call executes (K padded to 64; FP32 mode: six BF16 products per term)
        flops = 2.0 * n_scene * m * W * W
        tc_flops = 2.0 * n_scene * m * kp * ksplit
        res[prec] = {"ms": ms, "ms_quartiles": _quartiles(times), "steps": steps,
                     "correlations_per_s": n_scene * m / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12,
                     "tensor_tflops": tc_flops / (ms / 1e3) / 1e12,
                     # how many scene images found their own point of the unmoved mesh first
                     "top1_is_the_same_point": float((idx[:, 0].long().cpu() == q.long().cpu()).float().mean().item())}
        if "bf16_tflops" in peaks:
            res[prec]["roofline"] = {"bound": "tensor", "achieved": res[prec]["tensor_tflops"],
                                     "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
                                     "frac": res[prec]["tensor_tflops"] / float(peaks["bf16_tflops"]),
                                     "peak_source": "measured bf16_tflops (burst; whole call: centring + GEMM "
                                                    "with fused top-k + merge)"}
    del model, scene
    return {"scene_images": n_scene, "model_images": m, "W": W, "k": k, "by_precision": res, "peak_source": src,
            "kernel": "match_tc_kernel (tcgen05, TMEM accumulators, top-k fused in the epilogue)"}


def bench_batched(spin, torch, dev, steps, warmup, stream):
    """512 sphere meshes with their own W, B, angle: one graph-captured persistent
    launch per step (tuned rules per size class vs PSIA-STATIC)."""
    from paper_1811_00901_gb300 import workloads as wl
    items = wl.batched_spheres()
    meshes, batch = [], []
    total_images = 0
    free, _ = torch.cuda.mem_get_info(dev)
    need = sum(it["m"] * it["W"] * it["W"] * 4 for it in items)
    if need > 0.8 * free:
        return {"skipped": "needs %.1f GB of image output, %.1f GB free" % (need / 1e9, free / 1e9)}
    for it in items:
        mesh = spin.si_mesh_create(torch.from_numpy(it["points"]).to(dev), torch.from_numpy(it["normals"]).to(dev),
                                   stream=stream)
        meshes.append(mesh)
        out = torch.empty((it["m"], it["W"], it["W"]), dtype=torch.int32, device=dev)
        batch.append(dict(mesh=mesh, query_idx=None, m=it["m"], W=it["W"], bin_size=float(it["bin_size"]),
                          cos_s=float(it["cos_s"]), out=out))
        total_images += it["m"]
    res = {}
    try:
        for name, sched in (("tuned_or_GSS", None), ("STATIC", spin.make_schedule("STATIC"))):
            times = []
            for k in range(warmup + steps):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                spin.si_generate_batched(batch, sched, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if k >= warmup:
                    times.append(e0.elapsed_time(e1))
            res[name] = {"images_per_s": total_images / (statistics.median(times) / 1e3),
                         "ms_per_step": statistics.median(times), "step_ms_quartiles": _quartiles(times),
                         "steps": steps}
    finally:
        for mesh in meshes:
            spin.si_mesh_destroy(mesh)
    return {"meshes": len(items), "images": total_images, "output_gb": need / 1e9, "by_schedule": res,
            "dls_over_static": res["tuned_or_GSS"]["images_per_s"] / res["STATIC"]["images_per_s"]}


def bench_serving(spin, torch, dev, n_requests, pool_size, load_factors=(0.5, 0.8, 0.95)):
    """Resident mesh pool, Poisson request stream, continuous batching:
    saturated request rate, then p50/p99 latency at fractions of it."""
    from paper_1811_00901_gb300 import workloads as wl
    pool = wl.serving_pool(count=pool_size)
    meshes = [spin.si_mesh_create(torch.from_numpy(p["points"]).to(dev), torch.from_numpy(p["normals"]).to(dev))
              for p in pool]
    sizes = [p["points"].shape[0] for p in pool]
    srv = spin.si_serve_create(16 << 30, 256)
    try:
        for mh in meshes:
            spin.si_serve_add_mesh(srv, mh)
        # resident grids for both widths (the pool keeps them)
        for mh in meshes:
            for W in (16, 32):
                spin.si_mesh_prepare(mh, W, 0.8 / W)
        torch.cuda.synchronize()

        def run(reqs, rate=None):
            import threading
            qs = [torch.from_numpy(r["query_idx"]).to(dev) for r in reqs]
            torch.cuda.synchronize()
            tickets = [None] * len(reqs)
            lat = [0.0] * len(reqs)
            done = threading.Event()

            def waiter():
                for k in range(len(reqs)):
                    while tickets[k] is None:
                        time.sleep(0.0001)
                    spin.si_serve_wait(srv, tickets[k], -1)
                    _, lat[k] = spin.si_serve_result(srv, tickets[k])
                    spin.si_serve_release(srv, tickets[k])
                done.set()
            th = threading.Thread(target=waiter, daemon=True)
            th.start()
            t0 = time.perf_counter()
            for k, r in enumerate(reqs):
                if rate is not None:
                    wait = r["t"] * (1.0 / rate) * r["rate0"] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                item = dict(mesh=meshes[r["mesh"]], query_idx=qs[k], m=r["m"], W=r["W"],
                            bin_size=float(r["bin_size"]), cos_s=float(r["cos_s"]), out=None)
                t = None
                while t is None:
                    t = spin.si_serve_submit(srv, item)
                tickets[k] = t
            done.wait()
            wall = time.perf_counter() - t0
            images = sum(r["m"] for r in reqs)
            return wall, images, lat

        base_rate = 1000.0
        reqs = wl.request_stream(sizes, count=n_requests, rate_per_s=base_rate)
        for r in reqs:
            r["rate0"] = base_rate
        wall, images, lat = run(reqs)  # burst: everything at once -> saturated throughput
        sat_rps = n_requests / wall
        out = {"meshes": pool_size, "points": int(sum(sizes)), "requests": n_requests,
               "saturated": {"requests_per_s": sat_rps, "images_per_s": images / wall,
                             "p50_ms": float(np.percentile(lat, 50)) / 1e3,
                             "p99_ms": float(np.percentile(lat, 99)) / 1e3}}
        for f in load_factors:
            wall, images, lat = run(reqs, rate=f * sat_rps)
            out["load_%.2f" % f] = {"offered_requests_per_s": f * sat_rps, "images_per_s": images / wall,
                                    "p50_ms": float(np.percentile(lat, 50)) / 1e3,
                                    "p99_ms": float(np.percentile(lat, 99)) / 1e3}
        return out
    finally:
        spin.si_serve_destroy(srv)
        for mh in meshes:
            spin.si_mesh_destroy(mh)


# --------------------------------------------------------------------------
# CPU legs: the FP64 oracle as it stands
# --------------------------------------------------------------------------

def _oracle_rate(c, nq, seed=0):
    import oracle
    rng = np.random.default_rng(seed)
    q = np.sort(rng.choice(c["points"].shape[0], nq, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    oracle.spin_images(c["points"], c["normals"], c["W"], c["bin_size"], c["cos_s"], query_idx=q)
    return time.perf_counter() - t0


def cpu_baseline(c, budget_s=12.0):
    """Oracle images/s on a random sample sized for ~budget_s seconds."""
    t = _oracle_rate(c, 8, seed=1)
    per = t / 8
    nq = max(8, min(c["m"], int(budget_s / max(per, 1e-6))))
    t = _oracle_rate(c, nq, seed=2)
    return {"value": nq / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d random images of the %s workload (all %d points each, FP64, single thread)" % (
                nq, c["name"], c["points"].shape[0])}


def cpu_dls_baseline(c, budget_s=3.0):
    """The oracle's image loop under OpenMP schedule(static), (dynamic, 1) and
    (guided) on all host cores: the shared-memory CPU analogue of PSIA-STATIC,
    EPSIA-SS and EPSIA-GSS.  The first nq images, nq sized for ~budget_s each."""
    import oracle
    if not oracle.omp_available():
        return {"unavailable": "the host compiler has no OpenMP"}
    cores = oracle.omp_max_threads()
    pts, nrm = c["points"], c["normals"]
    W, B, cs = c["W"], c["bin_size"], c["cos_s"]
    probe = np.arange(2 * cores, dtype=np.int32)
    t0 = time.perf_counter()
    oracle.spin_images_omp(pts, nrm, W, B, cs, query_idx=probe, rule="static")
    per = (time.perf_counter() - t0) / len(probe)
    nq = int(max(2 * cores, min(c["m"], budget_s / max(per, 1e-9))))
    q = np.arange(nq, dtype=np.int32)
    out = {"kind": "oracle, OpenMP image loop", "cores": cores, "unit": UNIT,
           "sample": "images 0..%d of the %s workload (all %d points each, FP64)" % (nq - 1, c["name"],
                                                                                    pts.shape[0])}
    for rule, name in (("static", "static"), ("dynamic", "dynamic_1"), ("guided", "guided")):
        t0 = time.perf_counter()
        oracle.spin_images_omp(pts, nrm, W, B, cs, query_idx=q, rule=rule)
        out[name] = nq / (time.perf_counter() - t0)
    return out


def _host_cpu():
    """Host core count and CPU model (the oracle's timings depend on them)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def cpu_oracle_other_workloads():
    """The single-thread FP64 oracle on the other single-mesh workloads: every
    image of the 4,096-point sphere, and 128 of the 1M-point scene's queries."""
    import oracle
    from paper_1811_00901_gb300 import workloads as wl
    res = {}
    sp = wl.plain_sphere()
    t0 = time.perf_counter()
    oracle.spin_images(sp["points"], sp["normals"], sp["W"], sp["bin_size"], sp["cos_s"])
    res["sphere-4096-W16"] = {"images_per_s": sp["m"] / (time.perf_counter() - t0), "sample": "all 4096 images"}
    sc = wl.large_scene()
    q = sc["query_idx"][:128]
    t0 = time.perf_counter()
    oracle.spin_images(sc["points"], sc["normals"], sc["W"], sc["bin_size"], sc["cos_s"], query_idx=q)
    res["scene-1M-W64"] = {"images_per_s": len(q) / (time.perf_counter() - t0),
                           "sample": "the first 128 of its 262,144 queries (all 1M points each)"}
    return res


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    c = _workload()
    per = _oracle_rate(c, 4, seed=3) / 4
    nq = max(4, int(args.ref_step_seconds / max(per, 1e-6)))
    for k in range(args.warmup):
        _oracle_rate(c, max(2, nq // 4), seed=100 + k)
    times = [_oracle_rate(c, nq, seed=200 + k) for k in range(args.steps)]
    total = sum(times)
    value = nq * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(c, {"schedule": "single thread", "sample_images_per_step": nq}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d random images per step of the %s workload" % (nq, c["name"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile_case(args):
    """A short run for profilers: the bench workload's full path, `reps`
    times, under one schedule; no flush buffer, probes or CPU legs."""
    import torch

    import paper_1811_00901_gb300 as spin
    from paper_1811_00901_gb300 import _build
    _build.build()
    dev = torch.device("cuda", 0)
    c = _workload() if args.profile_workload == "heightfield" else _small_workload(args.profile_workload)
    n, m, W = c["points"].shape[0], c["m"], c["W"]
    tp = torch.from_numpy(c["points"]).to(dev)
    tn = torch.from_numpy(c["normals"]).to(dev)
    tq = None if c["query_idx"] is None else torch.from_numpy(c["query_idx"]).to(dev)
    out = torch.empty((m, W, W), dtype=torch.int32, device=dev)
    sched = spin.make_schedule(args.profile_case)
    for _ in range(args.reps):
        mesh = spin.si_mesh_create(tp, tn, n)
        spin.si_generate(mesh, tq, m, W, float(c["bin_size"]), float(c["cos_s"]), sched, out)
        torch.cuda.synchronize()
        spin.si_get_stats(mesh)
        spin.si_mesh_destroy(mesh)
    print(json.dumps({"profile_case": args.profile_case, "workload": c["name"], "reps": args.reps}))


def run_profile_match(args):
    """A short run for profilers: `--profile-match` scene images of the
    matching workload against the bench mesh's 100,000, `reps` calls in
    `--profile-precision` (BF16 or FP32)."""
    import torch

    import paper_1811_00901_gb300 as spin
    from paper_1811_00901_gb300 import _build
    _build.build()
    dev = torch.device("cuda", 0)
    c = _workload()
    stream = torch.cuda.current_stream(dev)
    scene, model, _ = _matching_inputs(spin, torch, dev, c, args.profile_match, stream)
    k = 5
    idx = torch.empty((args.profile_match, k), dtype=torch.int32, device=dev)
    val = torch.empty((args.profile_match, k), dtype=torch.float32, device=dev)
    for _ in range(args.reps):
        spin.si_match(scene, args.profile_match, model, c["m"], c["W"], k, args.profile_precision, idx, val, stream)
        torch.cuda.synchronize()
    print(json.dumps({"profile_match": args.profile_match, "model_images": c["m"], "W": c["W"], "reps": args.reps,
                      "precision": args.profile_precision}))


def _small_workload(name):
    from paper_1811_00901_gb300 import workloads as wl
    if name == "sphere":
        return wl.plain_sphere()
    if name == "scene":
        # the 1M-point scene with an eighth of its queries: 537 MB of images,
        # above L2 and small enough for a many-pass profiler capture
        c = wl.large_scene(m=32768)
        c["name"] = "scene-1M-W64, 32,768 of its queries"
        return c
    raise ValueError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", default=None, choices=list(SCHEDULES),
                    help="run the workload `--reps` times under one schedule (for ncu)")
    ap.add_argument("--profile-workload", default="heightfield", choices=["heightfield", "sphere", "scene"])
    ap.add_argument("--profile-match", type=int, default=0, metavar="N_SCENE",
                    help="run matching of N_SCENE images `--reps` times (for ncu)")
    ap.add_argument("--profile-precision", default="BF16", choices=["BF16", "FP32"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the sphere, 1M-scene, batched and serving runs")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_match:
        run_profile_match(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

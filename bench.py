#!/usr/bin/env python3
"""Benchmark of the registration hot path on GB300.

One step = one full multilevel registration of a synthetic CT-like pair
(default: 256^3 at 1 mm, 4 levels, 129^3 finest deformation nodes): pyramid,
prolongation, and at every level L-BFGS with Armijo backtracking, each trial
one matrix-free NGF + curvature objective+gradient evaluation.

Metric: objective+gradient evaluations per second, counted in full-resolution
equivalents (an evaluation at level l counts voxels_l / voxels_0), so that the
GPU registration and the CPU oracle are compared on the same work.  Also
reported: seconds per registration (ms_per_step), the isolated full-resolution
evaluation time and its HBM roofline fraction, the end-to-end rate from host
buffers, and the FP64 CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank registers its own pair (independent
replicas, no collective on the data path); value = all ranks' evaluations over
the slowest rank's time.
"""
import argparse
import hashlib
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

METRIC = "NGF+curvature objective+gradient evals/s and % HBM roofline; s per 256³ registration"
UNIT = "evals/s (full-resolution equivalent)"
L2_BYTES = 129 * 1024 * 1024
# the translation unit of the fused pass and every header it includes: the
# committed ncu traffic is valid only for this exact source
FUSED_KERNEL_SOURCES = ["paper_1812_06765_gb300/csrc/" + f
                        for f in ("k_ngf_fused.cu", "fused_pass.cuh", "k_pyramid.cu", "ngf_math.cuh", "common.cuh",
                                  "batch.h", "internal.h", "lbfgs_control.cuh", "lbfgs_state.h")] + ["include/reg.h"]


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, help="workload id (default 2: 256^3 CT, 4 levels)")
    ap.add_argument("--eval-iters", type=int, default=50, help="isolated evaluations for the roofline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eval-impl", type=int, default=None, help="0 fused, 1 multi-pass (default: library)")
    ap.add_argument("--eval-only", action="store_true", help="time only the isolated evaluation (profiling)")
    ap.add_argument("--host-loop", action="store_true",
                    help="queue every L-BFGS step from the host instead of one graph per level (the same kernels "
                         "in the same order; ncu cannot list kernels inside graphs with conditional nodes)")
    ap.add_argument("--fused-tz", type=int, default=None,
                    help="force the fused pass's z segment length (no autotuning launches; for profiling)")
    ap.add_argument("--fused-split", type=int, nargs=5, default=None, metavar=("L1", "N1", "L2", "N2", "LR"),
                    help="force the fused pass's z split on levels of that depth (for profiling)")
    ap.add_argument("--report", action="store_true",
                    help="one JSON line per single-pair workload (64^3, 128^3, 256^3, 4D-CT shape): GPU registration "
                         "and evaluation times, accuracy, and the FP64 oracle on all host cores and on one core")
    ap.add_argument("--pt-ab", action="store_true",
                    help="time one full-resolution evaluation with each P^T design: fused gather, multi-pass "
                         "gather (Eq. 3), multi-pass atomic scatter, multi-pass 8-colour scatter")
    ap.add_argument("--pairs", type=int, default=None, help="pairs of the uneven batch (workload 4; default 64)")
    ap.add_argument("--sub-batches", type=int, default=1,
                    help="workload 4: register the pairs in this many batches one after another, smallest "
                         "pairs first (each pair is done when its batch is)")
    ap.add_argument("--gen-procs", type=int, default=None, help="processes that generate the batch's pairs")
    ap.add_argument("--dims", type=int, nargs=3, default=None, metavar=("X", "Y", "Z"),
                    help="image size of the full-resolution workload (5) instead of its 512^3")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------
# distributed helpers (NCCL on GPUs; gloo in the CPU tests)
# ----------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def dist_reduce(x, op="max", device="cpu"):
    """Reduce a float over ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def dist_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for ln in f:
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------
# measurement helpers
# ----------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fused_tile_node_entries():
    """Partial sums one fused-pass tile writes per node plane: 3 components x the
    node columns an ox x oy output tile reaches (o / 2 + 1 per dimension)."""
    from paper_1812_06765_gb300 import _lib
    ox, oy, _ = _lib.reg_fused_tile_shape()
    return 3 * (ox // 2 + 1) * (oy // 2 + 1)


def committed_profile(kernel, digest, workload_name, split):
    """The committed ncu figures of a kernel launch (DRAM bytes, warp instructions),
    if they were taken on this source, this workload and this z split (else {})."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_digest") != digest:
        return {}
    if e.get("workload") != workload_name or split_lengths(e.get("fused_split", [0] * 5)) != split_lengths(split):
        return {}
    return e


def split_lengths(split):
    """Segment lengths of a split, sorted: splits with the same lengths launch the same tiles."""
    l1, n1, l2, n2, lr = split
    return sorted([l1] * n1 + [l2] * n2 + ([lr] if lr else []), reverse=True)


def split_partial_floats_per_column(split):
    """Node planes x entries one tile column keeps over all z segments of a split."""
    l1, n1, l2, n2, lr = split
    planes = n1 * (l1 // 2 + 1) + n2 * (l2 // 2 + 1) + (lr // 2 + 1 if lr else 0)
    return planes * fused_tile_node_entries()


def issue_peak_warp_inst_per_s():
    """GB300 instruction issue ceiling: 152 SMs x 4 schedulers x 1 warp
    instruction per cycle at the maximum SM clock (MEASURED_PEAKS.json, else 2070 MHz)."""
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return 152 * 4 * mhz * 1e6


def workload(config_id, rank, dims=None):
    from synth import CONFIGS, make_pair, make_pair_parallel, batch_sizes
    c = CONFIGS[config_id]
    if c.get("slab_noise"):   # full-resolution volume: planes generated by a process pool
        return c, make_pair_parallel(config_id, pair=rank, dims=dims)
    dims = batch_sizes(rank + 1)[rank] if c["dims"] is None else None
    p = make_pair(config_id, pair=rank, dims=dims)
    return c, p


def full_res_equivalent(stats, reg, levels):
    nv0 = np.prod(reg.level_info(0)["dims"])
    return sum(stats["evals"][lv] * np.prod(reg.level_info(lv)["dims"]) / nv0 for lv in range(levels))


def cpu_oracle_rate(p, c, budget_s):
    """FP64 oracle objective+gradient evaluations per second at full resolution (bounded sample)."""
    import oracle
    oracle.build()
    dims, h = p["dims"], p["spacing"]
    nodes = oracle.default_nodes(dims)
    from synth import random_field
    u = random_field(nodes, 7, 5.0).astype(np.float64)
    R, T = p["R"].astype(np.float64), p["T"].astype(np.float64)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.objective(dims, h, R, T, nodes, u, c["eta"], c["eta"], c["alpha"])
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return n / el, n, el, oracle.num_threads()


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_1812_06765_gb300 as reg_pkg
    from paper_1812_06765_gb300 import _lib
    from synth import random_field

    rank, world = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c, p = workload(args.config, rank, args.dims)
    kw = dict(levels=c["levels"], tau=c["eta"], alpha=c["alpha"], mem=c["mem"], max_iter=c["max_iter"], c1=c["c1"])
    if args.eval_impl is not None:
        kw["eval_impl"] = args.eval_impl
    if args.host_loop:
        kw["use_graph"] = False
    if args.fused_tz is not None:
        kw["fused_tz"] = args.fused_tz
    if args.fused_split is not None:
        kw["fused_split"] = args.fused_split
    cfg = reg_pkg.make_config(**kw)
    stream = torch.cuda.current_stream(dev)
    reg = reg_pkg.Registration(cfg, stream=stream)
    R_d = torch.from_numpy(p["R"]).to(dev)
    T_d = torch.from_numpy(p["T"]).to(dev)
    R_h = torch.from_numpy(p["R"]).pin_memory()
    T_h = torch.from_numpy(p["T"]).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    levels = c["levels"]

    def step_device():
        reg.set_images(R_d, T_d, p["spacing"])
        u, st = reg.register(out="torch")
        return st

    def isolated_eval(r=None):
        """Median device time (ms) of one full-resolution objective+gradient evaluation."""
        r = reg if r is None else r
        r.set_images(R_d, T_d, p["spacing"])
        info = r.level_info(0)
        u = torch.from_numpy(random_field(info["nodes"], 5, 5.0)).to(dev)
        grad = torch.empty_like(u)
        for _ in range(5):
            _lib.reg_eval_objective_grad(r.h, 0, u.data_ptr(), grad.data_ptr(), want_scalars=False)
        ev_ms, ngf_ms = [], []
        for _ in range(args.eval_iters):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.reg_eval_objective_grad(r.h, 0, u.data_ptr(), grad.data_ptr(), want_scalars=False)
            e1.record(stream)
            e1.synchronize()
            ev_ms.append(e0.elapsed_time(e1))
            ngf_ms.append(_lib.reg_last_ngf_ms(r.h))   # events around the fused kernel, same stream
        return statistics.median(ev_ms), info, statistics.median(ngf_ms)

    def isolated_eval_bf16():
        """The same evaluation with BF16 image storage (FP32 arithmetic)."""
        cfg_b = reg_pkg.make_config(image_dtype="bf16", **kw)
        rb = reg_pkg.Registration(cfg_b, stream=stream)
        try:
            return isolated_eval(rb)[0]   # whole evaluation with BF16 image storage
        finally:
            rb.close()

    if args.eval_only:   # profiling aid: the isolated evaluation alone
        eval_ms, info, _ = isolated_eval()
        eval_ms_bf16 = isolated_eval_bf16()
        if rank == 0:
            print(json.dumps({"eval_ms_full_res": eval_ms, "eval_ms_full_res_bf16_images": eval_ms_bf16,
                              "workload": c["name"], "eval_impl": reg.cfg.eval_impl, "iters": args.eval_iters}))
        reg.close()
        return

    # warm-up (untimed)
    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize(dev)

    # timed region: K registrations from device-resident images
    dist_barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local).start()
    times, eq_evals, launches, evals_per_level, iters_per_level, level_s = [], 0.0, 0, None, None, None
    for _ in range(args.steps):
        flush.zero_()                       # evict the previous step from L2 (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step_device()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        eq_evals += full_res_equivalent(st, reg, levels)
        launches += st["kernel_launches"] + 2 * (levels - 1)
        evals_per_level, iters_per_level, level_s = st["evals"], st["iters"], st["level_seconds"]
    torch.cuda.synchronize(dev)
    dist_barrier()
    clk = clocks.stop()
    total_ms = dist_reduce(sum(times), "max", dev)
    eq_all = dist_reduce(eq_evals, "sum", dev)
    value = eq_all / (total_ms / 1000.0)

    # end to end through the C ABI from pinned host buffers (copies inside the timed region)
    e2e_times = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reg.set_images(R_h, T_h, p["spacing"])
        u_h, st_h = reg.register(out="pinned")
        e2e_times.append(time.perf_counter() - t0)
    e2e_eq = full_res_equivalent(st_h, reg, levels)
    e2e_s = dist_reduce(statistics.mean(e2e_times), "max", dev)
    e2e_value = world * e2e_eq / e2e_s

    # isolated full-resolution evaluation: the objective+gradient pass
    eval_ms, info, ngf_ms = isolated_eval()
    eval_ms_bf16 = isolated_eval_bf16()
    nv = int(np.prod(info["dims"]))
    nn = int(np.prod(info["nodes"]))
    eval_bytes = 4 * nv + 4 * nv + 12 * nn + 12 * nn      # the evaluation: read R, T, u; write grad J
    peak, peak_kind = measured_peaks()
    eval_achieved = eval_bytes / (eval_ms * 1e-3) / 1e9
    impl = reg.cfg.eval_impl
    kernel = "objective_pass_fused" if impl == 0 else "objective_pass_multipass"
    tz, tiles = reg.level_tiling(0)
    split = reg.level_split(0)
    nseg = split[1] + split[3] + (1 if split[4] else 0)
    # the dominant kernel against the evaluation's algorithmic bytes (read R, T and u once, write
    # grad J: about 11 B per voxel); the tile partials of P^T r it writes for the gather are an
    # intermediate, reported beside them as overhead
    part_bytes = (4 * (tiles // nseg) * split_partial_floats_per_column(split) if impl == 0 and nseg
                  else 12 * nn)
    kernel_bytes = eval_bytes
    achieved = kernel_bytes / (ngf_ms * 1e-3) / 1e9
    prof = committed_profile(kernel, source_digest(FUSED_KERNEL_SOURCES), c["name"], split)
    traffic = prof.get("dram_bytes_per_launch_full_size")
    issue = None
    if prof.get("warp_instructions_per_launch"):
        rate = prof["warp_instructions_per_launch"] / (ngf_ms * 1e-3)
        peak_issue = issue_peak_warp_inst_per_s()
        issue = {"bound": "issue", "kernel": "k_ngf_fused", "achieved": rate, "peak": peak_issue,
                 "unit": "warp instructions/s", "frac": rate / peak_issue,
                 "warp_instructions_per_launch": prof["warp_instructions_per_launch"],
                 "what": "the kernel's binding limit: ncu instruction count per launch over the live event time, "
                         "against 152 SMs x 4 schedulers x 1 instruction/cycle at the maximum SM clock"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, el, cores = cpu_oracle_rate(p, c, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d FP64 oracle objective+gradient evaluations of the full-resolution %s pair "
                         "(%.1f s); a registration costs its full-resolution-equivalent evaluations" %
                         (n, "x".join(map(str, p["dims"])), el)}

    if rank == 0:
        mz = p["R"].shape
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": c["name"], "image": list(p["dims"]), "spacing_mm": list(p["spacing"]),
                       "levels": levels, "finest_nodes": list(info["nodes"]), "eta": c["eta"],
                       "alpha": c["alpha"], "lbfgs_mem": c["mem"], "max_iter_per_level": c["max_iter"],
                       "evals_per_level": evals_per_level, "iters_per_level": iters_per_level,
                       "level_device_s": level_s,
                       "eval_impl": "fused" if impl == 0 else "multi-pass",
                       "fused_tz_per_level": [reg.level_tiling(lv)[0] for lv in range(levels)],
                       "fused_split_per_level": [list(reg.level_split(lv)) for lv in range(levels)],
                       "tiling": "autotuned (z split timed per level)" if reg.cfg.autotune else "load model",
                       "lbfgs_loop": ("one CUDA graph per level; levels of at most 40k nodes one cooperative "
                                      "kernel" if reg.cfg.use_graph else "host-driven"),
                       "l2": "flushed between steps (2x L2 buffer written, untimed)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "image_shape_zyx": list(mz)},
            "registration_s": total_ms / args.steps / 1000.0,
            "eval_ms_full_res": eval_ms,
            "eval_ms_full_res_bf16_images": eval_ms_bf16,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_ngf_fused" if impl == 0 else kernel,
                         "algorithmic_bytes": kernel_bytes, "overhead_bytes": part_bytes, "launch_ms": ngf_ms,
                         "peak_kind": peak_kind,
                         "note": "algorithmic bytes: read R, T, u and write grad J once per evaluation; "
                                 "overhead: the tile partials the pass writes for the node gather; traffic also "
                                 "holds R's normalized gradient field, which the pass reads instead of R (16 "
                                 "bytes per voxel instead of 4, formed once per level: bytes traded for "
                                 "instructions); the pass is bound by latency and instruction issue, not HBM: "
                                 "see the ncu summary"},
            "issue_roofline": issue,
            "eval_roofline": {"bound": "hbm", "achieved": eval_achieved, "peak": peak, "unit": "GB/s",
                              "frac": eval_achieved / peak, "algorithmic_bytes": eval_bytes, "eval_ms": eval_ms,
                              "what": "whole objective+gradient evaluation (fused pass, curvature, gather, "
                                      "final reduction): read R, T, u once, write grad J"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * nv,
                    "d2h_bytes_per_step": 3 * 4 * nn, "registration_s": e2e_s},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    reg.close()


# ----------------------------------------------------------------------------
# the uneven batch: batched, graph-captured form against the per-pair loop
# ----------------------------------------------------------------------------
def _batch_pair(job):
    """One pair of the uneven batch (runs in a generator process)."""
    i, dims = job
    from synth import make_pair
    p = make_pair(4, pair=i, dims=dims)
    return p["R"], p["T"], tuple(p["dims"]), tuple(p["spacing"])


def batch_inputs(n_pairs, first_pair, procs):
    """The pairs of the batch, generated in a spawn pool (before any CUDA call)."""
    import multiprocessing as mp
    from synth import batch_sizes
    jobs = [(first_pair + i, d) for i, d in enumerate(batch_sizes(n_pairs))]
    procs = procs or min(len(jobs), os.cpu_count() or 1, 16)
    if procs <= 1:
        return [_batch_pair(j) for j in jobs]
    order = sorted(range(len(jobs)), key=lambda k: -int(np.prod(jobs[k][1])))   # largest first
    with mp.get_context("spawn").Pool(procs) as pool:
        made = pool.map(_batch_pair, [jobs[k] for k in order], chunksize=1)
    out = [None] * len(jobs)
    for k, v in zip(order, made):
        out[k] = v
    return out


def percentile_ms(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def run_batch(args):
    """Workload 4: 64 pairs of uneven size, registered (a) together, one graph
    launch per pyramid level for the whole batch, and (b) one after another
    through reg_register.  Both start from device-resident images and include
    the pyramid; pairs/s and per-pair completion times (from the step start to
    the moment the pair's result is in memory) are reported for both."""
    from synth import CONFIGS
    rank, world = dist_init("nccl")
    _, _, local = dist_env()
    c = CONFIGS[4]
    n = args.pairs or c["pairs"]
    pairs = batch_inputs(n, rank * n, args.gen_procs)
    import torch
    import paper_1812_06765_gb300 as reg_pkg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    levels = c["levels"]
    kw = dict(levels=levels, tau=c["eta"], alpha=c["alpha"], mem=c["mem"], max_iter=c["max_iter"], c1=c["c1"])
    if args.fused_tz is not None:
        kw["fused_tz"] = args.fused_tz
    if args.fused_split is not None:
        kw["fused_split"] = args.fused_split
    if args.host_loop:
        kw["use_graph"] = False
    regs = [reg_pkg.Registration(reg_pkg.make_config(**kw), stream=stream) for _ in range(n)]
    Rd = [torch.from_numpy(p[0]).to(dev) for p in pairs]
    Td = [torch.from_numpy(p[1]).to(dev) for p in pairs]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    restrict_launches = 2 * (levels - 1)

    # sub-batches, smallest pairs first: a pair's result is complete when its batch returns
    nsub = max(1, min(args.sub_batches, n))
    by_size = sorted(range(n), key=lambda i: int(np.prod(pairs[i][2])))
    subs = [by_size[k * n // nsub:(k + 1) * n // nsub] for k in range(nsub)]

    def step_batch(marks=None):
        res = [None] * n
        for k, idx in enumerate(subs):
            for i in idx:
                regs[i].set_images(Rd[i], Td[i], pairs[i][3])
            for i, r in zip(idx, reg_pkg.register_batch([regs[i] for i in idx], out="torch")):
                res[i] = r
            if marks is not None:
                marks[k].record(stream)
        return res

    def step_loop(marks=None):
        res = []
        for i in range(n):
            regs[i].set_images(Rd[i], Td[i], pairs[i][3])
            res.append(regs[i].register(out="torch"))
            if marks is not None:
                marks[i].record(stream)
        return res

    for _ in range(args.warmup):
        step_batch()
        step_loop()
    torch.cuda.synchronize(dev)

    dist_barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local).start()
    t_batch, done_batch, launches_batch = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in subs]
        e0.record(stream)
        res_b = step_batch(marks)
        marks[-1].synchronize()
        ms = e0.elapsed_time(marks[-1])
        t_batch.append(ms)
        for k, idx in enumerate(subs):              # every result of a batch lands when it returns
            done_batch += [e0.elapsed_time(marks[k])] * len(idx)
        launches_batch += sum(res_b[idx[0]][1]["kernel_launches"] for idx in subs) + restrict_launches * n
    t_loop, done_loop, own_loop, launches_loop = [], [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        e0.record(stream)
        res_l = step_loop(marks)
        marks[-1].synchronize()
        t = [e0.elapsed_time(m) for m in marks]
        t_loop.append(t[-1])
        done_loop += t
        own_loop += [t[0]] + [b - a for a, b in zip(t[:-1], t[1:])]
        launches_loop += sum(s["kernel_launches"] for _, s in res_l) + restrict_launches * n
    torch.cuda.synchronize(dev)
    dist_barrier()
    clk = clocks.stop()
    tb = dist_reduce(sum(t_batch), "max", dev)
    tl = dist_reduce(sum(t_loop), "max", dev)
    pairs_all = world * n * args.steps
    pairs_s_batch = pairs_all / (tb / 1000.0)
    pairs_s_loop = pairs_all / (tl / 1000.0)

    # accuracy of both forms: the batch tiles the fused pass for throughput and the
    # loop for one pair at a time, so the two runs round differently; compare the
    # reached NGF distance and the displacements
    max_diff = max(float((ub - ul).abs().max()) for (ub, _), (ul, _) in zip(res_b, res_l))
    mean_diff = statistics.mean(float((ub - ul).abs().mean()) for (ub, _), (ul, _) in zip(res_b, res_l))
    d_ratio, d_ratio_l = [], []
    for i in range(n):
        z = torch.zeros(regs[i].node_shape(0), dtype=torch.float32, device=dev)
        J0, D0, _, _ = regs[i].eval(z, 0)
        d_ratio.append(res_b[i][1]["D_final"] / D0)
        d_ratio_l.append(res_l[i][1]["D_final"] / D0)

    # algorithmic evaluation bytes (images, u and grad J at every evaluation) over the batch's step time
    eval_bytes = 0
    for i in range(n):
        for lv in range(levels):
            info = regs[i].level_info(lv)
            eval_bytes += res_b[i][1]["evals"][lv] * (8 * int(np.prod(info["dims"])) + 24 * int(np.prod(info["nodes"])))
    eff_gbs = eval_bytes / (statistics.mean(t_batch) * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()

    # end to end from pinned host images, results back into pinned host memory
    Rh = [torch.from_numpy(p[0]).pin_memory() for p in pairs]
    Th = [torch.from_numpy(p[1]).pin_memory() for p in pairs]
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for idx in subs:
            for i in idx:
                regs[i].set_images(Rh[i], Th[i], pairs[i][3])
            reg_pkg.register_batch([regs[i] for i in idx], out="pinned")
        e2e.append(time.perf_counter() - t0)
    e2e_s = dist_reduce(statistics.mean(e2e), "max", dev)
    h2d = sum(8 * int(np.prod(p[2])) for p in pairs)
    d2h = sum(12 * int(np.prod(r.level_info(0)["nodes"])) for r in regs)

    if rank == 0:
        vox = [int(np.prod(p[2])) for p in pairs]
        line = {
            "metric": "registration pairs/s of a batch of 64 uneven CT-like pairs (batched, graph-captured) "
                      "against the per-pair loop; p50/p99 per-pair completion time",
            "value": pairs_s_batch, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tb / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": c["name"], "pairs": n, "sizes": sorted({p[2] for p in pairs}),
                       "voxels_total": sum(vox), "spacing_mm": list(c["spacing"]), "levels": levels,
                       "eta": c["eta"], "alpha": c["alpha"], "lbfgs_mem": c["mem"],
                       "max_iter_per_level": c["max_iter"],
                       "l2": "flushed between steps (2x L2 buffer written, untimed); inputs exceed L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "batched": {"pairs_s": pairs_s_batch, "sub_batches": nsub, "p50_ms": percentile_ms(done_batch, 50),
                        "p99_ms": percentile_ms(done_batch, 99), "step_ms": statistics.mean(t_batch),
                        "level_device_s": res_b[subs[-1][0]][1]["level_seconds"],
                        "tiling_rule_per_level": res_b[subs[-1][0]][1]["tiling"],
                        "gpu_launches_per_step": launches_batch // max(1, args.steps)},
            "per_pair_loop": {"pairs_s": pairs_s_loop, "p50_ms": percentile_ms(done_loop, 50),
                              "p99_ms": percentile_ms(done_loop, 99), "step_ms": statistics.mean(t_loop),
                              "own_time_p50_ms": percentile_ms(own_loop, 50),
                              "own_time_p99_ms": percentile_ms(own_loop, 99),
                              "gpu_launches_per_step": launches_loop // max(1, args.steps)},
            "batched_over_loop": pairs_s_batch / pairs_s_loop,
            "equal_accuracy": {"D_final_over_D0_median_batched": float(np.median(d_ratio)),
                               "D_final_over_D0_median_loop": float(np.median(d_ratio_l)),
                               "D_final_over_D0_max_batched": float(np.max(d_ratio)),
                               "D_final_over_D0_max_loop": float(np.max(d_ratio_l)),
                               "mean_abs_u_diff_mm": mean_diff, "max_abs_u_diff_mm": max_diff,
                               "tiling": "batched: the batch autotuner's rule per level (batched.tiling_rule_per_level); "
                                         "loop: each pair's single-pair autotuned tiling (tests/test_gpu_batch.py: "
                                         "with the same tiling the two forms are bit-identical)"},
            "effective_eval_gbs": eff_gbs,
            "roofline": {"bound": "hbm", "achieved": eff_gbs, "peak": peak, "unit": "GB/s", "frac": eff_gbs / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "what": "whole batched step: every pair's evaluation bytes (read R, T, u, write grad J "
                                 "per evaluation, all levels) over the batch's step time, which also holds the "
                                 "L-BFGS vector passes and the pyramids"},
            "e2e": {"value": world * n / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "batch_s": e2e_s},
            "gpu_launches": launches_batch + launches_loop,
            "clocks": clk,
        }
        print(json.dumps(line))
    for r in regs:
        r.close()


# ----------------------------------------------------------------------------
# per-workload report: GPU times, accuracy, FP64 oracle on all cores and one core
# ----------------------------------------------------------------------------
_ONE_CORE_EVAL = """
import sys, time, json, numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from synth import CONFIGS, make_pair, random_field
cid = int(sys.argv[2])
c = CONFIGS[cid]
p = make_pair(cid)
nodes = oracle.default_nodes(p["dims"])
u = random_field(nodes, 7, 5.0).astype(np.float64)
R, T = p["R"].astype(np.float64), p["T"].astype(np.float64)
t0 = time.perf_counter()
oracle.objective(p["dims"], p["spacing"], R, T, nodes, u, c["eta"], c["eta"], c["alpha"])
print(json.dumps({"s_per_eval": time.perf_counter() - t0, "threads": oracle.num_threads()}))
"""


def oracle_one_core_eval_s(cid):
    """Seconds of one FP64 oracle evaluation at full resolution on one core (child process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", _ONE_CORE_EVAL, ROOT, str(cid)], env=env, capture_output=True,
                         text=True, timeout=600)
    if out.returncode != 0:
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_report(args):
    import torch
    import oracle
    import paper_1812_06765_gb300 as reg_pkg
    from synth import CONFIGS, random_field, true_inverse_displacement
    from scipy.ndimage import map_coordinates
    rank, world, local = dist_env()
    if rank != 0:
        return
    oracle.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = measured_peaks()

    def u_at(u, points, H):   # nodal trilinear value of u (3, nz, ny, nx) at points (N, 3) in mm
        idx = (np.asarray(points) / np.asarray(H))[:, ::-1].T
        return np.stack([map_coordinates(u[cc].astype(np.float64), idx, order=1, mode="nearest")
                         for cc in range(3)], 1)

    for cid in (0, 1, 2, 3):
        c, p = workload(cid, 0)
        kw = dict(levels=c["levels"], tau=c["eta"], alpha=c["alpha"], mem=c["mem"], max_iter=c["max_iter"],
                  c1=c["c1"])
        reg = reg_pkg.Registration(reg_pkg.make_config(**kw), stream=stream)
        R_d, T_d = torch.from_numpy(p["R"]).to(dev), torch.from_numpy(p["T"]).to(dev)
        R_h, T_h = torch.from_numpy(p["R"]).pin_memory(), torch.from_numpy(p["T"]).pin_memory()
        for _ in range(2):   # warm-up (tiling autotuned on the first call)
            reg.set_images(R_d, T_d, p["spacing"])
            reg.register(out="torch")
        dev_ms, host_s = [], []
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reg.set_images(R_d, T_d, p["spacing"])
            u_dev, st = reg.register(out="torch")
            e1.record(stream)
            e1.synchronize()
            dev_ms.append(e0.elapsed_time(e1))
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            reg.set_images(R_h, T_h, p["spacing"])
            u_h, st_h = reg.register(out="pinned")
            host_s.append(time.perf_counter() - t0)
        u_np = u_h.numpy()
        # one full-resolution evaluation
        info = reg.level_info(0)
        u = torch.from_numpy(random_field(info["nodes"], 5, 5.0)).to(dev)
        g = torch.empty_like(u)
        ev = []
        for i in range(23):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reg.eval(u, 0, grad=g)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ev.append(e0.elapsed_time(e1))
        eval_ms = statistics.median(ev)
        nv, nn = int(np.prod(info["dims"])), int(np.prod(info["nodes"]))
        eval_gbs = (8 * nv + 24 * nn) / (eval_ms * 1e-3) / 1e9
        eq = full_res_equivalent(st, reg, c["levels"])
        line = {"workload": c["name"], "image": list(p["dims"]), "spacing_mm": list(p["spacing"]),
                "levels": c["levels"], "finest_nodes": list(info["nodes"]),
                "iters_per_level": st["iters"], "evals_per_level": st["evals"],
                "fused_tz_per_level": [reg.level_tiling(lv)[0] for lv in range(c["levels"])],
                "fused_split_per_level": [list(reg.level_split(lv)) for lv in range(c["levels"])],
                "gpu": {"registration_s_device_resident": statistics.median(dev_ms) / 1000.0,
                        "registration_s_from_host_arrays": statistics.median(host_s),
                        "level_device_s": st["level_seconds"],
                        "eval_ms_full_res": eval_ms, "evals_per_s_full_res": 1000.0 / eval_ms,
                        "eval_hbm_frac": eval_gbs / peak, "peak_kind": peak_kind,
                        "full_res_equivalent_evals_per_registration": eq,
                        "l2": "flushed before every timed call"}}
        acc = {}
        if cid == 0:   # trajectory parity with the FP64 oracle, and the known warp as a sanity value
            ocfg = oracle.make_config(**kw)
            t0 = time.perf_counter()
            uo, sto = oracle.register(p["dims"], p["spacing"], p["R"], p["T"], ocfg)
            cpu_reg_s = time.perf_counter() - t0
            du = np.sqrt(((u_np.astype(np.float64) - uo) ** 2).sum(axis=0))
            H = info["node_spacing"]
            nz, ny, nx = u_np.shape[1:]
            Z, Y, X = np.meshgrid(np.arange(nz) * H[2], np.arange(ny) * H[1], np.arange(nx) * H[0], indexing="ij")
            pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
            ut = true_inverse_displacement(p["field"], pts)
            err_true = np.linalg.norm(u_np.reshape(3, -1).T - ut, axis=1)
            acc = {"mean_abs_u_gpu_minus_oracle_vox": float(du.mean() / min(p["spacing"])),
                   "J_gpu": st["J_final"], "J_oracle": sto["J"][0],
                   "mean_abs_u_minus_true_vox_sanity": float(err_true.mean() / min(p["spacing"])),
                   "cpu_registration_s_measured": cpu_reg_s}
        elif cid == 1:
            ocfg = oracle.make_config(**kw)
            t0 = time.perf_counter()
            uo, sto = oracle.register(p["dims"], p["spacing"], p["R"], p["T"], ocfg)
            cpu_reg_s = time.perf_counter() - t0
            du = np.sqrt(((u_np.astype(np.float64) - uo) ** 2).sum(axis=0))
            acc = {"mean_abs_u_gpu_minus_oracle_vox": float(du.mean() / min(p["spacing"])),
                   "J_gpu": st["J_final"], "J_oracle": sto["J"][0], "cpu_registration_s_measured": cpu_reg_s}
        elif cid == 3:
            H = info["node_spacing"]
            before = np.linalg.norm(p["lm_R"] - p["lm_T"], axis=1)
            after = np.linalg.norm(p["lm_R"] + u_at(u_np, p["lm_R"], H) - p["lm_T"], axis=1)
            acc = {"landmarks": len(before), "lme_before_mm": [float(before.mean()), float(before.std())],
                   "lme_after_mm": [float(after.mean()), float(after.std())]}
        line["accuracy"] = acc
        # FP64 oracle on the host: all cores, and one core (child process)
        nodes = oracle.default_nodes(p["dims"])
        uo64 = random_field(nodes, 7, 5.0).astype(np.float64)
        R64, T64 = p["R"].astype(np.float64), p["T"].astype(np.float64)
        n, t0 = 0, time.perf_counter()
        while n < 20 and (n < 2 or time.perf_counter() - t0 < 4.0):
            oracle.objective(p["dims"], p["spacing"], R64, T64, nodes, uo64, c["eta"], c["eta"], c["alpha"])
            n += 1
        all_s = (time.perf_counter() - t0) / n
        one = oracle_one_core_eval_s(cid)
        cpu = {"eval_s_full_res_all_cores": all_s, "cores": oracle.num_threads(),
               "eval_s_full_res_one_core": one["s_per_eval"] if one else None,
               "registration_s_estimate_all_cores": all_s * eq,
               "estimate": "oracle seconds per full-resolution evaluation x the GPU run's full-resolution-"
                           "equivalent evaluation count (an extrapolation)",
               "gpu_speedup_eval_vs_all_cores": all_s / (eval_ms * 1e-3)}
        if "cpu_registration_s_measured" in acc:
            cpu["registration_s_measured_all_cores"] = acc.pop("cpu_registration_s_measured")
        line["cpu_oracle"] = cpu
        print(json.dumps(line), flush=True)
        reg.close()


def run_pt_ab(args):
    """One full-resolution evaluation of the workload with each P^T design; the
    multi-pass forms differ only in their last step (gather, atomic, 8 colours)."""
    import torch
    import paper_1812_06765_gb300 as reg_pkg
    from paper_1812_06765_gb300 import _lib
    from synth import random_field
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    c, p = workload(args.config, 0)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    R_d, T_d = torch.from_numpy(p["R"]).to(dev), torch.from_numpy(p["T"]).to(dev)
    out = {"workload": c["name"], "image": list(p["dims"]), "evals_timed": args.eval_iters,
           "l2": "flushed before every timed evaluation"}
    names = {0: "fused pass (tile partials + node gather)", 1: "multi-pass, P^T gather (Eq. 3)",
             2: "multi-pass, P^T atomic scatter", 3: "multi-pass, P^T 8-colour scatter"}
    ref = None
    for impl in (0, 1, 2, 3):
        reg = reg_pkg.Registration(reg_pkg.make_config(levels=1, tau=c["eta"], alpha=c["alpha"], eval_impl=impl),
                                   stream=stream)
        reg.set_images(R_d, T_d, p["spacing"])
        u = torch.from_numpy(random_field(reg.level_info(0)["nodes"], 5, 5.0)).to(dev)
        g = torch.empty_like(u)
        ms, ngf = [], []
        for i in range(args.eval_iters + 3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            J, D, S, _ = reg.eval(u, 0, grad=g)
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ms.append(e0.elapsed_time(e1))
                ngf.append(_lib.reg_last_ngf_ms(reg.h))
        if ref is None:
            ref = (J, g.clone())
        out[names[impl]] = {"eval_ms": statistics.median(ms), "ngf_pass_ms": statistics.median(ngf),
                            "J_rel_diff_vs_fused": abs(J - ref[0]) / abs(ref[0]),
                            "grad_rel_l2_vs_fused": float((g - ref[1]).norm() / ref[1].norm())}
        reg.close()
    print(json.dumps(out))


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ----------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    c, p = workload(args.config, 0)
    import oracle
    oracle.build()
    from synth import random_field
    dims, h = p["dims"], p["spacing"]
    nodes = oracle.default_nodes(dims)
    u = random_field(nodes, 7, 5.0).astype(np.float64)
    R, T = p["R"].astype(np.float64), p["T"].astype(np.float64)

    def step():
        oracle.objective(dims, h, R, T, nodes, u, c["eta"], c["eta"], c["alpha"])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps / el
    sample = ("each step: one FP64 oracle objective+gradient evaluation of the full-resolution %s pair"
              % "x".join(map(str, dims)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": c["name"], "image": list(dims), "levels": c["levels"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": oracle.num_threads(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.report:
        run_report(args)
    elif args.pt_ab:
        run_pt_ab(args)
    elif args.config == 4:
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

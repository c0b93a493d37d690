#!/usr/bin/env python
"""Benchmark of exact grid pair counting on GB300.

Default workload: 100,000,000 points in a periodic 3000 Mpc/h cube (half
uniform, half Neyman-Scott clusters with sigma = 5 Mpc/h), unit-mean
lognormal binary32 weights (sigma_ln = 0.3), weighted auto counts in 40
linear s bins of 5 Mpc/h on [0, 200): FP32 separations with binary64 rescue
near bin edges, int64 counts and binary64 weighted sums.  The same line also
carries the plain FP64 path on the same GPU, the measured FP32/FP64 peaks,
and the 2,000,000-point clustered cube in (s, mu) 40 x 100 bins under its
own workload name.

One step = one pass of the whole path over the catalogue already resident in
HBM: canonicalise + grid build (bounds, per-cell counts, scan, scatter,
weight packing), i-block list, pair kernel (separation, bin lookup, shared
histograms, weight products), the binary64 re-evaluation of near-edge pairs
(inside the pair kernel or by the rescue kernel, as tuned), histogram
read-back.  The value is in-range pairs binned per second: the one unit
every exact method shares, whatever its cell size or pruning.

Prints one JSON line.  --impl reference times the CPU oracle (brute force,
binary64) on a bounded sample of the same workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs evaluated/sec on 1 GB300, FP32+FP64-rescue vs plain FP64 at exact counts"
UNIT = "pairs/s"                 # in-range pairs binned per second (every arm)
FLOPS_PER_CANDIDATE = 8          # separation: 3 subtractions, 3 multiplies, 2 adds
FLOPS_PER_IN_RANGE = 6           # bin locate per in-range pair
FP32_LANES_PER_SM = 128
DEFAULT_WORKLOAD = "mixed_periodic_n100m_s40_w"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-mocks", type=int, default=4,
                    help="batched mocks: time the plain FP64 kernel on this many of them")
    ap.add_argument("--fp64-shards", type=int, default=0,
                    help="plain FP64 arm of the weighted workloads: time it on 1/S of the "
                         "i-blocks (0: 64 for catalogues of 5e7 points or more, 16 from 1e7, "
                         "else 1)")
    ap.add_argument("--no-weights", action="store_true",
                    help="weighted workloads: count the same catalogues without their weights "
                         "(to compare the weighted and unweighted kernels)")
    ap.add_argument("--config2-steps", type=int, default=5,
                    help="default line only: also time the 2M-point (s, mu) benchmark this "
                         "many steps and report it under its workload name (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--tree-steps", type=int, default=3,
                    help="steps of the k-d tree path reported beside the grid line (0: none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--micro", choices=["hist"], default=None,
                    help="run a micro-benchmark instead of the pair-count step: 'hist' times the "
                         "histogram-update algorithms on sampled squared separations")
    ap.add_argument("--structure", choices=["grid", "kdtree"], default="grid",
                    help="space partition: the regular grid (default, tuned) or the k-d tree "
                         "with the dual-tree traversal")
    ap.add_argument("--n-leaf", type=int, default=32, help="k-d tree leaf capacity")
    ap.add_argument("--list-cap", type=int, default=0,
                    help="k-d tree list nodes: at most this many points (0 = automatic)")
    ap.add_argument("--cell-size", type=float, default=0.0)
    ap.add_argument("--rescue-capacity", type=int, default=0,
                    help="rescue-queue slots with fixed options (0 automatic, -1 none: all inline)")
    ap.add_argument("--ipt", type=int, default=0)
    ap.add_argument("--shard", action="store_true",
                    help="with --gpus N > 1: split one catalogue's point blocks across the ranks "
                         "and sum the histograms once at the end (strong scaling) instead of "
                         "one independent catalogue per rank (replicas, weak scaling)")
    ap.add_argument("--volume-scale", type=float, default=1.0,
                    help="same density in a box of this fraction of the volume "
                         "(small cases for profiling; 1 = the full workload); for the "
                         "weighted and multi-catalogue workloads: N scaled in the same volume")
    return ap.parse_args()


def workload_inputs(w, f):
    """Catalogue of workload w; f < 1 keeps the number density and cluster
    shape in a box of f times the volume (periodic clustered workloads)."""
    from synth import catalogs as C
    from synth import workloads as W
    if f == 1.0:
        return W.make_inputs(w)["D"], w.L
    L = w.L * f ** (1.0 / 3.0)
    n = int(round(w.extra["n"] * f))
    if "parents" in w.extra:
        D = C.neyman_scott(n, max(1, int(w.extra["parents"] * f)), w.extra["children"],
                           w.extra["sigma"], L, w.seed)
    else:
        D = C.uniform_box(n, L, w.seed)
    return D, L


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def max_over_ranks(v, dist, dev):
    """The largest of every rank's value v (v itself with one process)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample
# --------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the oracle's line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_rate(D, w, seconds, seed=0, L=None, threads=None, wt=None):
    """Oracle throughput in in-range pairs binned per second: brute force over
    all pairs of a random sample of i-points against the whole catalogue (the
    cross form of the same pair set), self-pairs excluded, with the weighted
    sums when weights wt are given.  Returns (rate, seconds, sample size,
    cores, pair evaluations per second)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    kw = dict(box=w.L if L is None else L, periodic=w.periodic, mode=w.mode, los=w.los,
              edges_a=w.edges_a, edges_b=w.edges_b)
    n = D.shape[0]
    if wt is not None:
        wt = np.asarray(wt, dtype=np.float64)
    m0, dt = 16, 0.0

    def run(idx):
        S = np.ascontiguousarray(D[idx])
        if wt is None:
            return oracle.count(S, D, threads=threads, **kw)
        return oracle.count(S, D, w1=wt[idx], w2=wt, threads=threads, **kw)
    while True:      # calibrate on growing samples until one takes >= 1/8 of the budget
        idx = rng.choice(n, m0, replace=False)
        t = time.perf_counter()
        run(idx)
        dt = max(time.perf_counter() - t, 1e-6)
        if dt >= seconds / 8 or m0 >= n:
            break
        m0 = min(n, m0 * 4)
    m = int(max(1, min(n, m0 * seconds / dt)))
    # a multiple of the thread count: the oracle deals rows out round-robin,
    # so every thread then gets the same number of rows
    cores = threads or oracle.default_threads()
    if m >= cores:
        m = min(n, (m + cores - 1) // cores * cores)
    idx = rng.choice(n, m, replace=False)
    t = time.perf_counter()
    c, _ = run(idx)
    dt = time.perf_counter() - t
    in_range = int(c.sum()) - m        # each sampled point pairs with itself at s = 0
    return in_range / dt, dt, m, cores, m * n / dt


def traffic_record(workload, tree=False, inline=True):
    """DRAM bytes per pair-kernel launch of a workload from the committed ncu
    summary (profiles/traffic_<workload>.json), if the kernel source is
    unchanged since it was captured and the structure and rescue mode match."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
        src = open(os.path.join(ROOT, "paper_2301_12557_gb300", "csrc", "pairs_impl.cuh"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
            return None
        if bool(rec.get("tree", False)) != bool(tree):
            return None
        if (rec.get("rescue") == "inline") != bool(inline):
            return None
        return rec
    except Exception:
        return None


# --------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from synth import workloads as W
    w = W.WORKLOADS[args.workload]
    wt = None
    if w.weighted or len(w.pair_kinds) > 1:
        inp = sets_inputs(w, 1.0)
        big = max([k for k in ("D", "R") if k in inp], key=lambda k: inp[k].shape[0])
        D, wt, L_box = inp[big], inp.get("w" + big), inp["L"]
    else:
        D, L_box = W.make_inputs(w)["D"], w.L
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    samp = None
    for k in range(args.warmup + args.steps):
        r, dt, m, cores, _ = oracle_sample_rate(D, w, per_step, seed=k, L=L_box, wt=wt)
        if k >= args.warmup:
            rates.append((r, dt, m))
        samp = (m, cores)
    tot_pairs = sum(r * dt for r, dt, _ in rates)
    tot_t = sum(dt for _, dt, _ in rates)
    value = tot_pairs / tot_t
    sample = (f"{samp[0]} random i-points x all {D.shape[0]} points per step (brute force, "
              f"binary64{', weighted' if wt is not None else ''}); in-range pairs found per second")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / len(rates), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": int(D.shape[0]), "oracle": "CPU brute force"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": samp[1], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, emit=True):
    """The single-catalogue line (2M-point clustered cube by default of this
    function).  emit=False: return the line instead of printing it (one
    process, no collectives)."""
    import torch
    rank, world, local = dist_env()
    if not emit:
        rank, world = 0, 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2301_12557_gb300 as P
    from synth import workloads as W

    P.lib()
    w = W.WORKLOADS[args.workload]
    D_host, L_box = workload_inputs(w, args.volume_scale)
    if world > 1 and rank > 0 and not args.shard:
        # replicas: every rank counts its own independent catalogue
        from synth import catalogs as C
        D_host = C.neyman_scott(D_host.shape[0], w.extra["parents"], w.extra["children"],
                                w.extra["sigma"], L_box, w.seed + 7919 * rank)
    n = D_host.shape[0]
    dev = torch.device("cuda", local)
    D = torch.from_numpy(D_host).to(dev)
    bins = P.Bins(w.mode, w.los, w.edges_a, w.edges_b)
    box = P.make_box(L_box, w.periodic)
    stream = torch.cuda.current_stream()
    tuning = None
    tree = args.structure == "kdtree"
    list_cap = args.list_cap
    if tree and args.shard:
        raise SystemExit("--shard is a grid-path option")
    if tree and (args.list_cap > 0 or args.ipt > 0):
        opts = P.make_opts("f32", 0.0, args.ipt or 2)
    elif tree:
        # measured list level and i-points per thread, once, before the timed steps
        t0 = time.perf_counter()
        opts, list_cap, trials = P.pc_tune_tree(D, box=box, bins=bins, n_leaf=args.n_leaf,
                                                stream=stream)
        tuning = {"seconds": time.perf_counter() - t0,
                  "trials": [{"list_cap": c, "ipt": i, "ms": round(ms, 3)} for c, i, ms in trials]}
    elif args.cell_size > 0 or args.ipt > 0:
        opts = P.make_opts("f32", args.cell_size, args.ipt, rescue_capacity=args.rescue_capacity)
    else:
        # measured autotuning on this catalogue, once, before the timed steps
        t0 = time.perf_counter()
        opts, trials = P.pc_tune(D, box=box, bins=bins, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0,
                  "trials": [{"cell_size": round(c, 3), "ipt": i, "priv": pv, "ms": round(ms, 3)}
                             for c, i, pv, ms in trials],
                  "last_trial": "near-edge pairs evaluated inside the pair kernel"}
    if args.shard and world > 1:
        from paper_2301_12557_gb300 import shard
        shard.shard_opts(opts, rank, world)
    out = torch.zeros(bins.nbins, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tree_ms = []

    def step(o=opts, x=D, counts=out, structure=args.structure):
        if structure == "kdtree":
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t = P.pc_build_tree(x, box=box, n_leaf=args.n_leaf, list_cap=list_cap,
                                stream=stream)
            b.record(stream)
            try:
                _, _, st = P.pc_count_tree(t, None, bins, o, stream, counts=counts)
            finally:
                t.free()
            tree_ms.append(a.elapsed_time(b))
            return st
        g = P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=o, stream=stream)
        try:
            _, _, st = P.pc_count_auto(g, bins, o, stream, counts=counts)
        finally:
            g.free()
        return st

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = P.pc_launch_count()
    tot_ms, stats = 0.0, []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                        # evict L2 between timed steps
        ev[k][0].record(stream)
        stats.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = P.pc_launch_count() - launches0
    clocks = sampler.stop()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    t_local = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
    # every step bins the same pairs: this rank's in-range pairs (its shard's
    # share under block shards) times the steps
    inr_step = float(out.sum().item())
    work_local = torch.tensor([inr_step * args.steps,
                               float(sum(s.candidates for s in stats))],
                              dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(work_local, op=dist.ReduceOp.SUM)
    t_max = float(t_local.item())
    inr_all, cand_all = (float(v) for v in work_local.tolist())
    value = inr_all / (t_max * 1e-3)
    counts_local = out.cpu().numpy()         # this rank's histogram (its shard's share)
    if args.shard and dist is not None:
        from paper_2301_12557_gb300 import shard
        out = shard.sum_histograms(out)      # the one collective: the final histogram sum
    counts = out.cpu().numpy()

    # ---- e2e: host buffers through the same ABI, copies inside the region --
    e2e = None
    if args.e2e_steps > 0:
        D_pin = torch.from_numpy(D_host).pin_memory()
        host_counts = np.zeros(bins.nbins, dtype=np.int64)
        e2e_ms = []
        for k in range(args.e2e_steps + 1):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st_e = step(x=D_pin, counts=host_counts)
            b.record(stream)
            torch.cuda.synchronize()
            if k > 0:
                e2e_ms.append(a.elapsed_time(b))
        assert np.array_equal(host_counts, counts_local), "host-buffer counts differ from device run"
        e2e_t = max_over_ranks(statistics.mean(e2e_ms), dist, dev)
        e2e = {"value": inr_all / args.steps / (e2e_t * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(n * 3 * 8), "d2h_bytes_per_step": int(bins.nbins * 8),
               "ms_per_step": e2e_t}

    peaks = measured_fp_peaks(P, stream, local)

    # ---- plain FP64 path on the same GB300 -----------------------------------
    fp64 = None
    if args.fp64_steps > 0:
        # the FP64 kernel has no group pruning: its own cost-model cell side
        vol = float(np.prod(np.broadcast_to(np.asarray(L_box, dtype=np.float64), (3,))))
        o64 = P.make_opts("f64", P.pc_suggest_cell_size(n, vol, bins.r_max), 1)
        out64 = torch.zeros_like(out)
        step(o=o64, counts=out64, structure="grid")
        torch.cuda.synchronize()
        ms64 = []
        for _ in range(args.fp64_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64 = step(o=o64, counts=out64, structure="grid")
            b.record(stream)
            torch.cuda.synchronize()
            ms64.append(a.elapsed_time(b))
        exact = bool(torch.equal(out64, out))
        inr64 = float(out64.sum().item())
        # the FP64 kernel evaluates every candidate: the same per-pair flop
        # counts, against the measured FP64 rate
        fl64 = FLOPS_PER_CANDIDATE * float(s64.candidates) + FLOPS_PER_IN_RANGE * inr64
        k64_ms = s64.ms_pairs if s64.ms_pairs > 0 else statistics.mean(ms64)
        ach64 = fl64 / (k64_ms * 1e-3) / 1e12
        fp64 = {"value": inr64 / (statistics.mean(ms64) * 1e-3), "unit": UNIT,
                "cell_size": o64.cell_size,
                "ms_per_step": statistics.mean(ms64), "steps": args.fp64_steps,
                "counts_identical_to_fp32_rescue": exact,
                "roofline": {"bound": "fp64", "achieved": ach64, "peak": peaks["fp64_tflops"],
                             "unit": "TFLOP/s", "frac": ach64 / peaks["fp64_tflops"],
                             "peak_source": "measured: DFMA loop (pc_fp_peak), " + peaks["profile"],
                             "kernel_ms": k64_ms}}

    # ---- the k-d tree path on the same catalogue (grid line only) -----------
    kd = None
    if not tree and args.tree_steps > 0 and world == 1:
        t0 = time.perf_counter()
        o_kd, cap_kd, _ = P.pc_tune_tree(D, box=box, bins=bins, n_leaf=args.n_leaf, stream=stream)
        tune_s = time.perf_counter() - t0
        out_kd = torch.zeros_like(out)

        def kd_step():
            t = P.pc_build_tree(D, box=box, n_leaf=args.n_leaf, list_cap=cap_kd, stream=stream)
            try:
                P.pc_count_tree(t, None, bins, o_kd, stream, counts=out_kd)
            finally:
                t.free()
        kd_step()
        torch.cuda.synchronize()
        kd_ms = []
        for _ in range(args.tree_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kd_step()
            b.record(stream)
            torch.cuda.synchronize()
            kd_ms.append(a.elapsed_time(b))
        kd = {"value": float(out_kd.sum().item()) / (statistics.mean(kd_ms) * 1e-3), "unit": UNIT,
              "ms_per_step": statistics.mean(kd_ms), "steps": args.tree_steps,
              "step": "tree build + dual-tree traversal + pair and rescue kernels",
              "list_cap": cap_kd or "auto", "ipt": o_kd.ipt, "n_leaf": args.n_leaf,
              "rescue": "inline" if o_kd.rescue_capacity < 0 else "queued",
              "tuning_seconds": tune_s,
              "counts_identical_to_grid": bool(torch.equal(out_kd, out))}

    # ---- roofline of the dominant kernel -------------------------------------
    fp32_peak = peaks["fp32_tflops"]
    ms_pairs = statistics.mean(s.ms_pairs for s in stats)
    cand = stats[0].candidates
    flops = FLOPS_PER_CANDIDATE * float(cand)
    achieved = flops / (ms_pairs * 1e-3) / 1e12
    evaluated = cand - stats[0].pruned       # pairs the kernel separated one by one
    flops_ev = FLOPS_PER_CANDIDATE * evaluated + FLOPS_PER_IN_RANGE * inr_step
    ach_ev = flops_ev / (ms_pairs * 1e-3) / 1e12
    trec = traffic_record(w.name, tree, opts.rescue_capacity < 0)
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": trec["bytes_per_launch"] if trec else None,
                "traffic_source": trec.get("source") if trec else None,
                "kernel": "k_pairs_f32<SMU,LOS_Z>" + (" (tree variant)" if tree else ""),
                "flops_per_launch": flops,
                "flops_definition": (f"{FLOPS_PER_CANDIDATE} FP32 flops per candidate pair of the "
                                     f"cell stencil ({float(cand):.4g} per launch)"),
                "achieved_evaluated": ach_ev, "frac_evaluated": ach_ev / fp32_peak,
                "evaluated_definition": (f"{FLOPS_PER_CANDIDATE} per pair evaluated one by one "
                                         f"({evaluated:.4g}) + {FLOPS_PER_IN_RANGE} per in-range "
                                         f"pair ({inr_step:.4g})"),
                "peak_source": "measured: " + peaks["how"] + " (" + peaks["profile"] + ")",
                "kernel_ms": ms_pairs,
                "kernel_share_of_step": ms_pairs / (t_max / args.steps)}

    cpu = None
    if emit and rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, dt, m, cores, evals = oracle_sample_rate(D_host, w, args.cpu_seconds, L=L_box)
        r1, dt1, m1, _, _ = oracle_sample_rate(D_host, w, args.cpu_seconds / 4, seed=1, L=L_box,
                                               threads=1)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{m} random i-points x all {n} points (brute force, binary64), "
                         f"{dt:.1f} s; in-range pairs found per second",
               "pair_evaluations_per_s": evals,
               "cpu_model": cpu_model(),
               "single_core": {"value": r1, "unit": UNIT,
                               "sample": f"{m1} random i-points x all {n} points, {dt1:.1f} s"}}

    if rank == 0:
        s0 = stats[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True,
            # the paper's timing rule (App. A): drop the slowest and the
            # fastest run, average the rest (rank 0's steps)
            "ms_per_step_trimmed": (statistics.mean(sorted(step_ms)[1:-1])
                                    if len(step_ms) >= 3 else None),
            "scaling": "strong" if (args.shard and world > 1) else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name if args.volume_scale == 1.0 else
                       f"{w.name} at volume x{args.volume_scale}", "n": int(n),
                       "box": L_box, "bins": "s 40 x mu 100 (LOS z)",
                       "precision": "FP32 separations, binary64 rescue near bin edges, int64 counts",
                       "parallelism": (f"block shards x{world} + one histogram sum"
                                       if args.shard else f"replicas x{world}")
                                      if world > 1 else "1 GPU",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "unit_of_work": "in-range pairs binned (each pair in exactly one bin)",
                       "structure": ("k-d tree (leaf capacity %d, list nodes %s), dual-tree "
                                     "traversal" % (args.n_leaf, list_cap or "auto"))
                                    if tree else "regular grid",
                       "cell_size": s0.cell_size, "ipt": opts.ipt, "priv": opts.priv,
                       "rescue": ("inline in the pair kernel" if opts.rescue_capacity < 0 else
                                  "queued for the rescue kernel"),
                       "tuning": tuning,
                       "tree": ({"node_pairs": int(s0.tree_pairs), "blocks": int(s0.blocks),
                                 "ms_build": statistics.mean(tree_ms[-args.steps:]),
                                 "ms_traverse": s0.ms_traverse,
                                 "largest_list_node_extent": s0.cell_size} if tree else None),
                       "in_range_pairs": int(counts.sum()),
                       "candidates_per_step": int(s0.candidates),
                       "pruned_per_step": int(s0.pruned)},
            "candidate_pairs_per_s": cand_all / (t_max * 1e-3),
            "rescued_fraction": s0.rescued / max(1, int(counts.sum())),
            "fp64_path": fp64,
            "kdtree_path": kd,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "roofline": roofline,
            "measured_peaks": {k: v for k, v in peaks.items() if k != "how"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
        if not emit:
            return line
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Many catalogues in one persistent launch (graph-replayed count)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2301_12557_gb300 as P
    from synth import catalogs as C
    from synth import workloads as W

    P.lib()
    w = W.WORKLOADS[args.workload]
    m = max(1, int(round(w.extra["m"] * args.volume_scale)))
    mocks = C.batch_mocks(m, w.extra["n_min"], w.extra["n_max"], 3.0, 8.0, w.L,
                          w.seed + 7919 * rank)
    dev = torch.device("cuda", local)
    X = [torch.from_numpy(x).to(dev) for x in mocks]
    n_tot = sum(x.shape[0] for x in mocks)
    bins = P.Bins(w.mode, w.los, w.edges_a, w.edges_b)
    box = P.make_box(w.L, True)
    stream = torch.cuda.current_stream()
    tuning = None
    tree = args.structure == "kdtree"
    list_cap = args.list_cap
    med = sorted(range(m), key=lambda k: X[k].shape[0])[m // 2]
    if tree and (args.list_cap > 0 or args.ipt > 0):
        opts = P.make_opts("f32", 0.0, args.ipt or 2)
        cell = 0.0
    elif tree:
        # measured list level and i-points per thread, on the mock of median size
        t0 = time.perf_counter()
        opts, list_cap, trials = P.pc_tune_tree(X[med], box=box, bins=bins, n_leaf=args.n_leaf,
                                                stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on_mock_n": int(X[med].shape[0]),
                  "trials": [{"list_cap": c, "ipt": i, "ms": round(ms, 3)} for c, i, ms in trials]}
        cell = 0.0
    elif args.cell_size > 0 or args.ipt > 0:
        cell = args.cell_size or P.pc_suggest_cell_size(n_tot // m, w.L ** 3, bins.r_max)
        opts = P.make_opts("f32", cell, args.ipt)
    else:
        # measured autotuning once, on the mock of median size; all mocks share it
        t0 = time.perf_counter()
        opts, trials = P.pc_tune(X[med], box=box, bins=bins, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on_mock_n": int(X[med].shape[0]),
                  "trials": [{"cell_size": round(c, 3), "ipt": i, "priv": pv, "ms": round(ms, 3)}
                             for c, i, pv, ms in trials]}
        cell = opts.cell_size
    opts.use_graph = 0 if tree else 1
    out = torch.zeros(m * bins.nbins, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    last_stats = []

    def step(xs=X, counts=out, batched=True, o=None):
        o = opts if o is None else o
        if tree:
            # every mock's k-d tree in one level loop
            ts = P.pc_build_tree_batch(xs, box=box, n_leaf=args.n_leaf, list_cap=list_cap,
                                       stream=stream)
        else:
            ts = [P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=o, stream=stream)
                  for x in xs]
        try:
            if batched:
                if tree:
                    _, _, st = P.pc_count_tree_batch(ts, bins, o, stream, counts=counts)
                else:
                    _, _, st = P.pc_count_batch(ts, bins, o, stream, counts=counts)
                last_stats.append(st)
                return st.candidates
            cand = 0
            for k, g in enumerate(ts):
                view = counts[k * bins.nbins:(k + 1) * bins.nbins]
                if tree:
                    _, _, st = P.pc_count_tree(g, None, bins, opts, stream, counts=view)
                else:
                    _, _, st = P.pc_count_auto(g, bins, opts, stream, counts=view)
                cand += st.candidates
            return cand
        finally:
            for g in ts:
                g.free()

    def timed(k_steps, **kw):
        ms, cand = [], 0
        for _ in range(k_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cand = step(**kw)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return ms, cand

    for _ in range(args.warmup):
        step()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = P.pc_launch_count()
    ms, cand = timed(args.steps)
    launches = P.pc_launch_count() - l0
    clocks = sampler.stop()
    t_local = torch.tensor([sum(ms)], dtype=torch.float64, device=dev)
    inr_step = float(out.sum().item())       # in-range pairs of all mocks, every step
    c_local = torch.tensor([inr_step * args.steps, float(cand) * args.steps],
                           dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(c_local, op=dist.ReduceOp.SUM)
    t_max = float(t_local.item())
    inr_all, cand_all = (float(v) for v in c_local.tolist())
    value = inr_all / (t_max * 1e-3)
    batched_counts = out.clone()
    loop_ms, _ = timed(1, batched=False)
    same = bool(torch.equal(out, batched_counts))
    e2e = None
    if args.e2e_steps > 0:
        Xh = [torch.from_numpy(x).pin_memory() for x in mocks]
        host = np.zeros(m * bins.nbins, dtype=np.int64)
        e_ms, _ = timed(args.e2e_steps, xs=Xh, counts=host)
        assert np.array_equal(host, batched_counts.cpu().numpy())
        e2e_t = max_over_ranks(statistics.mean(e_ms), dist, dev)
        e2e = {"value": inr_all / args.steps / (e2e_t * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(n_tot * 24), "d2h_bytes_per_step": int(m * bins.nbins * 8),
               "ms_per_step": e2e_t}
    peaks = measured_fp_peaks(P, stream, local)

    # ---- roofline of the batched pair kernel --------------------------------
    # The graph replay hides the pair kernel's own duration: one more batched
    # count launched directly gives the library's event-timed pair kernel
    # (the tree batch is never graph-replayed, so its timed steps give it).
    if tree:
        kst = last_stats[-1]
    else:
        import ctypes
        o_direct = P.pc_opts()
        ctypes.memmove(ctypes.byref(o_direct), ctypes.byref(opts), ctypes.sizeof(opts))
        o_direct.use_graph = 0
        kcounts = torch.zeros_like(out)
        step(counts=kcounts, o=o_direct)
        torch.cuda.synchronize()
        same = same and bool(torch.equal(kcounts, batched_counts))
        kst = last_stats[-1]
    roof = None
    if kst.ms_pairs > 0:
        fp32_peak = peaks["fp32_tflops"]
        achieved = FLOPS_PER_CANDIDATE * float(kst.candidates) / (kst.ms_pairs * 1e-3) / 1e12
        evaluated = kst.candidates - kst.pruned
        ach_ev = ((FLOPS_PER_CANDIDATE * float(evaluated) + FLOPS_PER_IN_RANGE * inr_step)
                  / (kst.ms_pairs * 1e-3) / 1e12)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "kernel": "k_pairs_f32<%s,LOS_%s>, one launch over all %d mocks"
                          % (w.mode.upper(), w.los.upper(), m),
                "kernel_ms": kst.ms_pairs,
                "kernel_share_of_step": kst.ms_pairs / (t_max / args.steps),
                "timed": ("the timed steps' batched launch" if tree else
                          "one batched launch outside the graph, same options and blocks"),
                "flops_per_launch": FLOPS_PER_CANDIDATE * float(kst.candidates),
                "flops_definition": "8 FP32 flops per candidate pair (%.4g per launch)"
                                    % float(kst.candidates),
                "achieved_evaluated": ach_ev, "frac_evaluated": ach_ev / fp32_peak,
                "evaluated_definition": "8 per pair evaluated one by one (%.4g) + 6 per in-range "
                                        "pair (%.4g)" % (float(evaluated), inr_step),
                "peak_source": "measured: " + peaks["how"] + " (" + peaks["profile"] + ")"}

    # ---- plain FP64 kernel on a subset of the mocks ---------------------------
    fp64 = None
    if args.fp64_steps > 0 and not tree and world == 1:
        k64 = min(m, max(1, args.fp64_mocks))
        n64 = sum(int(X[k].shape[0]) for k in range(k64))
        o64 = P.make_opts("f64", P.pc_suggest_cell_size(n64 // k64, w.L ** 3, bins.r_max), 1)
        o64.use_graph = 0
        out64 = torch.zeros(k64 * bins.nbins, dtype=torch.int64, device=dev)
        step(xs=X[:k64], counts=out64, o=o64)
        torch.cuda.synchronize()
        ms64 = []
        for _ in range(args.fp64_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(xs=X[:k64], counts=out64, o=o64)
            b.record(stream)
            torch.cuda.synchronize()
            ms64.append(a.elapsed_time(b))
        s64 = last_stats[-1]
        inr64 = float(out64.sum().item())
        fl64 = FLOPS_PER_CANDIDATE * float(s64.candidates) + FLOPS_PER_IN_RANGE * inr64
        k64_ms = s64.ms_pairs if s64.ms_pairs > 0 else statistics.mean(ms64)
        ach64 = fl64 / (k64_ms * 1e-3) / 1e12
        fp64 = {"value": inr64 / (statistics.mean(ms64) * 1e-3), "unit": UNIT,
                "mocks": f"the first {k64} of the {m} mocks ({n64} points), one batched launch",
                "cell_size": o64.cell_size, "ms_per_step": statistics.mean(ms64),
                "steps": args.fp64_steps,
                "counts_identical_to_fp32_rescue":
                    bool(torch.equal(out64, batched_counts[:k64 * bins.nbins])),
                "roofline": {"bound": "fp64", "achieved": ach64, "peak": peaks["fp64_tflops"],
                             "unit": "TFLOP/s", "frac": ach64 / peaks["fp64_tflops"],
                             "peak_source": "measured: DFMA loop (pc_fp_peak), " + peaks["profile"],
                             "kernel_ms": k64_ms}}

    # ---- the oracle on the host cores ----------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, dt, ms_, cores, evals = oracle_sample_rate(mocks[med], w, args.cpu_seconds, L=w.L)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{ms_} random points of the median mock x all its "
                         f"{mocks[med].shape[0]} points (brute force, binary64), {dt:.1f} s; "
                         f"in-range pairs found per second",
               "pair_evaluations_per_s": evals, "cpu_model": cpu_model()}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name if m == w.extra["m"] else f"{w.name} ({m} mocks)",
                       "mocks": m, "n_total": int(n_tot),
                       "structure": ("k-d trees (leaf capacity %d, list nodes %s) built in one "
                                     "batched level loop, dual-tree traversal per mock"
                                     % (args.n_leaf, list_cap or "auto"))
                                    if tree else "regular grid",
                       "cell_size": cell, "ipt": opts.ipt,
                       "priv": opts.priv, "tuning": tuning,
                       "unit_of_work": "in-range pairs binned (each pair in exactly one bin)",
                       "in_range_pairs": int(inr_step), "candidates_per_step": int(cand),
                       "bins": "s 40 x mu 100 (LOS z)",
                       "precision": "FP32 separations, binary64 rescue near bin edges, int64 counts",
                       "launch": ("one persistent pair-kernel launch over all mocks"
                                  if tree else "one persistent pair-kernel launch over all mocks, "
                                  "replayed as a CUDA graph"),
                       "l2": "flushed between timed steps (256 MiB write)"},
            "candidate_pairs_per_s": cand_all / (t_max * 1e-3),
            "count_call": ({"ms_total": kst.ms_total, "ms_pairs": kst.ms_pairs,
                            "ms_rescue": kst.ms_rescue,
                            "timed": roof["timed"] if roof else None}
                           if kst.ms_total > 0 else None),
            "loop_of_single_counts_ms": loop_ms[0],
            "batched_speedup_vs_loop": loop_ms[0] / (t_max / args.steps),
            "loop_counts_identical": same,
            "roofline": roof, "fp64_path": fp64, "cpu_baseline": cpu, "measured_peaks": peaks,
            "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def sets_inputs(w, f, seed_offset=0):
    """Catalogues of a weighted or multi-catalogue workload.  f < 1: the
    periodic cube keeps its number density and cluster shape in f times the
    volume (small cases for profiling); the survey shell keeps its shell with
    f times the points."""
    from synth import catalogs as C
    from synth import workloads as W
    if w.periodic:
        n = w.extra["n"] if f == 1.0 else int(round(w.extra["n"] * f))
        L = w.L * f ** (1.0 / 3.0)
        D = C.mixed_box(n, L, 0.5, 10.0, 5.0, w.seed + seed_offset)
        return {"D": D, "wD": C.lognormal_weights(n, 0.3, w.seed + 3 + seed_offset), "L": L}
    return W.make_inputs(w, scale=f)


def measured_fp_peaks(P, stream, sampler_gpu):
    """FP32 and FP64 FMA throughput of this GPU, measured now (pc_fp_peak):
    the FP32 peak is the faster of the scalar and packed FFMA loops, each
    the best of two runs; clocks sampled meanwhile."""
    smp = ClockSampler(sampler_gpu)
    smp.start()
    runs = {k: [P.pc_fp_peak(k, stream=stream) for _ in range(2)] for k in ("ffma", "ffma2", "dfma")}
    clk = smp.stop()
    best = {k: max(v, key=lambda t: t[0]) for k, v in runs.items()}
    fp32 = max(best["ffma"][0], best["ffma2"][0])
    return {"fp32_tflops": fp32, "fp64_tflops": best["dfma"][0],
            "ffma_tflops": best["ffma"][0], "ffma2_tflops": best["ffma2"][0],
            "how": "pc_fp_peak: 8 independent FMA chains per thread, every SM filled to its "
                   "thread limit, CUDA-event timed after one untimed launch (best of 2); "
                   "FP32 = faster of FFMA and packed FFMA2",
            "profile": "profiles/fp_peaks_gb300.md", "clocks": clk}


def run_sets(args, extra=None):
    """Workloads with weights and several pair kinds (the 100M-point weighted
    cube, the default line; the survey shell's DD, DR and RR): every step
    builds every catalogue's grid and runs every count, weighted sums in
    binary64."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2301_12557_gb300 as P
    from synth import workloads as W

    P.lib()
    w = W.WORKLOADS[args.workload]
    # replicas: every rank counts its own independent catalogue (periodic
    # cube: its own seed); block shards: every rank the same catalogue
    seed_off = 7919 * rank if (world > 1 and not args.shard) else 0
    inp = sets_inputs(w, args.volume_scale, seed_off)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    names = ["D"] + (["R"] if "R" in inp else [])
    host = {k: (inp[k], None if args.no_weights else inp.get("w" + k)) for k in names}
    weighted = any(wt is not None for _, wt in host.values())
    devc = {k: (torch.from_numpy(x).to(dev), torch.from_numpy(wt).to(dev) if wt is not None else None)
            for k, (x, wt) in host.items()}
    bins = P.Bins(w.mode, w.los, w.edges_a, w.edges_b)
    L_box = inp["L"]
    if w.periodic:
        box = P.make_box(L_box, True)
    else:
        lo = np.full(3, np.inf)
        hi = np.full(3, -np.inf)
        for k in names:
            a, b = P.pc_aabb(devc[k][0])
            lo, hi = np.minimum(lo, a), np.maximum(hi, b)
        box = P.make_box(None, False, lo, hi)
    big = max(names, key=lambda k: host[k][0].shape[0])
    tuning = None
    tree = args.structure == "kdtree"
    list_cap = args.list_cap
    if tree and args.shard:
        raise SystemExit("--shard is a grid-path option")
    if tree and (args.list_cap > 0 or args.ipt > 0):
        opts = P.make_opts("f32", 0.0, args.ipt or 2)
    elif tree:
        t0 = time.perf_counter()
        opts, list_cap, trials = P.pc_tune_tree(devc[big][0], devc[big][1], box=box, bins=bins,
                                                n_leaf=args.n_leaf, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on": big,
                  "trials": [{"list_cap": c, "ipt": i, "ms": round(ms, 3)} for c, i, ms in trials]}
    elif args.cell_size > 0 or args.ipt > 0:
        opts = P.make_opts("f32", args.cell_size, args.ipt, rescue_capacity=args.rescue_capacity)
    else:
        t0 = time.perf_counter()
        opts, trials = P.pc_tune(devc[big][0], devc[big][1], box=box, bins=bins, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on": big,
                  "trials": [{"cell_size": round(c, 3), "ipt": i, "priv": pv, "ms": round(ms, 3)}
                             for c, i, pv, ms in trials]}
    if args.shard and world > 1:
        from paper_2301_12557_gb300 import shard
        shard.shard_opts(opts, rank, world)
    kinds = list(w.pair_kinds)
    outs = {k: (torch.zeros(bins.nbins, dtype=torch.int64, device=dev),
                torch.zeros(bins.nbins, dtype=torch.float64, device=dev)) for k in kinds}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tree_ms = []

    def step(cats=devc, results=outs, o=opts, structure=args.structure):
        t_b = None
        if structure == "kdtree":
            a_ev = torch.cuda.Event(enable_timing=True)
            b_ev = torch.cuda.Event(enable_timing=True)
            a_ev.record(stream)
            gs = {k: P.pc_build_tree(x, wt, box=box, n_leaf=args.n_leaf, list_cap=list_cap,
                                     stream=stream)
                  for k, (x, wt) in cats.items()}
            b_ev.record(stream)
            t_b = (a_ev, b_ev)
        else:
            gs = {k: P.pc_build_grid(x, wt, box=box, r_max=bins.r_max, opts=o, stream=stream)
                  for k, (x, wt) in cats.items()}
        stats = {}
        try:
            for kind in kinds:
                a, b = gs[kind[0]], gs[kind[1]]
                c, wc = results[kind]
                if not weighted:
                    wc = None
                if structure == "kdtree":
                    _, _, st = P.pc_count_tree(a, None if kind[0] == kind[1] else b, bins, o,
                                               stream, counts=c, wcounts=wc)
                elif kind[0] == kind[1]:
                    _, _, st = P.pc_count_auto(a, bins, o, stream, counts=c, wcounts=wc)
                else:
                    _, _, st = P.pc_count_cross(a, b, bins, o, stream, counts=c, wcounts=wc)
                stats[kind] = st
        finally:
            for g in gs.values():
                g.free()
        if t_b is not None:
            tree_ms.append(t_b[0].elapsed_time(t_b[1]))
        return stats

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = P.pc_launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    all_stats = []
    for k in range(args.steps):
        flush.zero_()                        # evict L2 between timed steps
        ev[k][0].record(stream)
        all_stats.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = P.pc_launch_count() - l0
    clocks = sampler.stop()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stats = all_stats[-1]
    inr = {k: int(outs[k][0].sum().item()) for k in kinds}
    t_local = torch.tensor([sum(step_ms)], dtype=torch.float64, device=dev)
    work_local = torch.tensor([float(sum(inr.values())) * args.steps,
                               float(sum(st.candidates for s in all_stats for st in s.values()))],
                              dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
        dist.all_reduce(work_local, op=dist.ReduceOp.SUM)
    t_max = float(t_local.item())
    inr_all, cand_all = (float(v) for v in work_local.tolist())
    value = inr_all / (t_max * 1e-3)
    t_step = t_max / args.steps
    counts_local = {k: outs[k][0].cpu().numpy().copy() for k in kinds}
    if args.shard and dist is not None:
        from paper_2301_12557_gb300 import shard
        for k in kinds:
            outs[k] = (shard.sum_histograms(outs[k][0]), shard.sum_histograms(outs[k][1]))

    # ---- e2e: host buffers through the same ABI, copies inside the region --
    e2e = None
    if args.e2e_steps > 0:
        pinned = {k: (torch.from_numpy(x).pin_memory(),
                      torch.from_numpy(wt).pin_memory() if wt is not None else None)
                  for k, (x, wt) in host.items()}
        hout = {k: (np.zeros(bins.nbins, dtype=np.int64), np.zeros(bins.nbins, dtype=np.float64))
                for k in kinds}
        e_ms = []
        for _ in range(args.e2e_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(pinned, hout)
            b.record(stream)
            torch.cuda.synchronize()
            e_ms.append(a.elapsed_time(b))
        for k in kinds:
            assert np.array_equal(hout[k][0], counts_local[k]), k
        h2d = sum(x.nbytes + (wt.nbytes if wt is not None else 0) for x, wt in host.values())
        e2e_t = max_over_ranks(statistics.mean(e_ms), dist, dev)
        e2e = {"value": inr_all / args.steps / (e2e_t * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(len(kinds) * bins.nbins * 16),
               "ms_per_step": e2e_t}

    peaks = measured_fp_peaks(P, stream, local)

    # ---- plain FP64 path on the same GB300, on a block shard ----------------
    fp64 = None
    if args.fp64_steps > 0 and not tree and world == 1:
        n_big = host[big][0].shape[0]
        S = args.fp64_shards if args.fp64_shards > 0 else \
            (64 if n_big >= 50_000_000 else (16 if n_big >= 10_000_000 else 1))
        vol = float(np.prod(np.asarray(box.hi) - np.asarray(box.lo))) if not w.periodic \
            else float(L_box) ** 3
        cell64 = P.pc_suggest_cell_size(n_big, vol, bins.r_max)
        o64 = P.make_opts("f64", cell64, 1, shard_index=0, shard_count=S)
        # the FP32 + rescue path on the same blocks (same cell side, same shard)
        o32 = P.make_opts("f32", cell64, opts.ipt, rescue_capacity=opts.rescue_capacity,
                          shard_index=0, shard_count=S)
        r64 = {k: (torch.zeros_like(outs[k][0]), torch.zeros_like(outs[k][1])) for k in kinds}
        r32 = {k: (torch.zeros_like(outs[k][0]), torch.zeros_like(outs[k][1])) for k in kinds}
        step(results=r32, o=o32, structure="grid")
        s64 = step(results=r64, o=o64, structure="grid")     # warm-up (module load)
        torch.cuda.synchronize()
        ms64 = []
        for _ in range(args.fp64_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64 = step(results=r64, o=o64, structure="grid")
            b.record(stream)
            torch.cuda.synchronize()
            ms64.append(a.elapsed_time(b))
        exact = all(bool(torch.equal(r64[k][0], r32[k][0])) for k in kinds)
        wdiff = 0.0
        if weighted:
            for k in kinds:
                ref = r64[k][1].abs().clamp_min(1e-300)
                wdiff = max(wdiff, float(((r64[k][1] - r32[k][1]).abs() / ref).max().item()))
        inr64 = float(sum(r64[k][0].sum().item() for k in kinds))
        cand64 = float(sum(s64[k].candidates for k in kinds))
        k64_ms = sum(s64[k].ms_pairs for k in kinds)
        fl64 = FLOPS_PER_CANDIDATE * cand64 + FLOPS_PER_IN_RANGE * inr64
        ach64 = fl64 / (k64_ms * 1e-3) / 1e12
        fp64 = {"value": inr64 / (statistics.mean(ms64) * 1e-3), "unit": UNIT,
                "cell_size": cell64, "steps": args.fp64_steps,
                "blocks": (f"1/{S} of the i-blocks (shard 0 of {S}); the rate is measured on "
                           "them, the full-step time is extrapolated" if S > 1 else "all"),
                "ms_per_step": statistics.mean(ms64),
                "ms_per_full_step_extrapolated": statistics.mean(ms64) * S,
                "in_range_pairs": int(inr64),
                "counts_identical_to_fp32_rescue": exact,
                "weighted_max_rel_diff_vs_fp32_rescue": wdiff if weighted else None,
                "roofline": {"bound": "fp64", "achieved": ach64, "peak": peaks["fp64_tflops"],
                             "unit": "TFLOP/s", "frac": ach64 / peaks["fp64_tflops"],
                             "peak_source": "measured: DFMA loop (pc_fp_peak), "
                                            + peaks["profile"],
                             "kernel_ms": k64_ms,
                             "flops_definition": f"{FLOPS_PER_CANDIDATE} per candidate pair "
                                                 f"({cand64:.4g}) + {FLOPS_PER_IN_RANGE} per "
                                                 f"in-range pair ({inr64:.4g})"}}

    # ---- the k-d tree path on the same catalogues (grid line only) ----------
    kd = None
    if not tree and args.tree_steps > 0 and world == 1:
        t0 = time.perf_counter()
        o_kd, cap_kd, _ = P.pc_tune_tree(devc[big][0], devc[big][1], box=box, bins=bins,
                                         n_leaf=args.n_leaf, stream=stream)
        tune_s = time.perf_counter() - t0
        rkd = {k: (torch.zeros_like(outs[k][0]), torch.zeros_like(outs[k][1])) for k in kinds}
        list_cap_saved = list_cap
        list_cap = cap_kd
        step(results=rkd, o=o_kd, structure="kdtree")
        torch.cuda.synchronize()
        kd_ms = []
        nkd = min(args.tree_steps, 2)
        for _ in range(nkd):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(results=rkd, o=o_kd, structure="kdtree")
            b.record(stream)
            torch.cuda.synchronize()
            kd_ms.append(a.elapsed_time(b))
        list_cap = list_cap_saved
        same = all(bool(torch.equal(rkd[k][0], outs[k][0])) for k in kinds)
        kwd = 0.0
        if weighted:
            for k in kinds:
                ref = outs[k][1].abs().clamp_min(1e-300)
                kwd = max(kwd, float(((rkd[k][1] - outs[k][1]).abs() / ref).max().item()))
        kd = {"value": float(sum(rkd[k][0].sum().item() for k in kinds)) / (statistics.mean(kd_ms) * 1e-3),
              "unit": UNIT, "ms_per_step": statistics.mean(kd_ms), "steps": nkd,
              "ms_build": statistics.mean(tree_ms[-nkd:]),
              "step": "tree build + dual-tree traversal + pair kernel (weight products and near-edge "
                      "pairs as on the grid)",
              "list_cap": cap_kd or "auto", "ipt": o_kd.ipt, "n_leaf": args.n_leaf,
              "tuning_seconds": tune_s, "counts_identical_to_grid": same,
              "weighted_max_rel_diff_vs_grid": kwd if weighted else None}

    # ---- roofline of the dominant kernel -------------------------------------
    kdom = max(kinds, key=lambda k: stats[k].ms_pairs)
    sd = stats[kdom]
    ms_pairs = statistics.mean(s[kdom].ms_pairs for s in all_stats)
    inr_d = float(inr[kdom])
    flops = FLOPS_PER_CANDIDATE * float(sd.candidates)
    achieved = flops / (ms_pairs * 1e-3) / 1e12
    evaluated = float(sd.candidates - sd.pruned)
    flops_ev = FLOPS_PER_CANDIDATE * evaluated + FLOPS_PER_IN_RANGE * inr_d
    ach_ev = flops_ev / (ms_pairs * 1e-3) / 1e12
    fp32_peak = peaks["fp32_tflops"]
    trec = traffic_record(w.name, tree, opts.rescue_capacity < 0)
    kname = {"s": "S", "smu": "SMU", "sigpi": "SIGPI"}[w.mode]
    wkind = {0: "", 1: ", binary64 weight products", 2: ", integer weight products"}.get(sd.wsum, "")
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": trec["bytes_per_launch"] if trec else None,
                "traffic_source": trec.get("source") if trec else None,
                "kernel": f"k_pairs_f32<{kname},LOS_{w.los.upper()}>" + wkind +
                          (" (tree variant)" if tree else ""),
                "pair_kind": kdom,
                "flops_per_launch": flops,
                "flops_definition": (f"{FLOPS_PER_CANDIDATE} FP32 flops per candidate pair of the "
                                     f"cell stencil ({float(sd.candidates):.4g} per launch)"),
                "achieved_evaluated": ach_ev, "frac_evaluated": ach_ev / fp32_peak,
                "evaluated_definition": (f"{FLOPS_PER_CANDIDATE} per pair evaluated one by one "
                                         f"({evaluated:.4g}) + {FLOPS_PER_IN_RANGE} per in-range "
                                         f"pair ({inr_d:.4g}); the weight product is integer work"),
                "peak_source": "measured: " + peaks["how"] + " (" + peaks["profile"] + ")",
                "kernel_ms": ms_pairs,
                "kernel_share_of_step": ms_pairs / t_step}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        x, wt = host[big]
        r, dt, m, cores, evals = oracle_sample_rate(x, w, args.cpu_seconds, L=L_box, wt=wt)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{m} random {big} points x all {x.shape[0]} {big} points (brute force, "
                         f"binary64{', weighted' if wt is not None else ''}), {dt:.1f} s; "
                         f"in-range pairs found per second",
               "pair_evaluations_per_s": evals, "cpu_model": cpu_model()}
    if rank == 0:
        s0 = stats[kinds[0]]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "ms_per_step_trimmed": (statistics.mean(sorted(step_ms)[1:-1])
                                    if len(step_ms) >= 3 else None),
            "scaling": "strong" if (args.shard and world > 1) else "weak",
            "vs_baseline": None, "dtype": "f32+f64" if weighted else "f32",
            "data": "synthetic",
            "config": {"workload": w.name if args.volume_scale == 1.0 else
                       f"{w.name} at volume x{args.volume_scale}",
                       "catalogues": {k: int(host[k][0].shape[0]) for k in names},
                       "box": L_box if w.periodic else "survey shell bounds",
                       "bins": ("s 40 x 5 Mpc/h on [0, 200)" if w.mode == "s" else
                                "sigma 40 x pi 40 on [0, 200)^2 (midpoint LOS)"),
                       "pair_kinds": kinds, "weighted": weighted,
                       "precision": "FP32 separations, binary64 rescue near bin edges, int64 "
                                    "counts" + (", weighted sums in binary64 (per-pair products "
                                                "exact to 2^-34 or binary64)" if weighted else ""),
                       "parallelism": (f"block shards x{world} + one histogram sum"
                                       if args.shard else f"replicas x{world}")
                                      if world > 1 else "1 GPU",
                       "unit_of_work": "in-range pairs binned over all pair kinds",
                       "structure": ("k-d tree (leaf capacity %d, list nodes %s), dual-tree traversal"
                                     % (args.n_leaf, list_cap or "auto")) if tree else "regular grid",
                       "cell_size": s0.cell_size, "ipt": opts.ipt, "priv": opts.priv,
                       "rescue": ("inline in the pair kernel" if opts.rescue_capacity < 0 else
                                  "queued for the rescue kernel"),
                       "weight_sums": {0: "none", 1: "binary64 products",
                                       2: "exact integer products of binary32 significands",
                                       3: "integer products of the binary32 roundings of binary64 "
                                          "weights plus their remainders' terms"}.get(
                                           s0.wsum, str(s0.wsum)),
                       "tuning": tuning, "l2": "flushed between timed steps (256 MiB write)",
                       "in_range_pairs": int(sum(inr.values())),
                       "candidates_per_step": int(sum(st.candidates for st in stats.values())),
                       "pruned_per_step": int(sum(st.pruned for st in stats.values())),
                       "tree_build_ms": statistics.mean(tree_ms[-args.steps:]) if tree_ms else None},
            "candidate_pairs_per_s": cand_all / (t_max * 1e-3),
            "rescued_fraction": sum(st.rescued for st in stats.values()) / max(1, sum(inr.values())),
            "per_kind": {k: {"in_range_pairs": inr[k], "ms_pairs": stats[k].ms_pairs,
                             "ms_total": stats[k].ms_total, "candidates": stats[k].candidates,
                             "pruned": stats[k].pruned, "rescued": stats[k].rescued,
                             "node_pairs": stats[k].tree_pairs if tree else None,
                             "ms_traverse": stats[k].ms_traverse if tree else None,
                             "prec": "f32+rescue" if stats[k].prec == 0 else "f64"} for k in kinds},
            "fp64_path": fp64,
            "kdtree_path": kd,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "roofline": roofline,
            "measured_peaks": {k: v for k, v in peaks.items() if k != "how"},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        }
        if extra:
            line.update(extra())
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_micro_hist(args):
    """Histogram-update micro-benchmark (Sect. 3.2.4): 6.4e9 squared separations
    sampled as in App. C over [0, 200^2), linear bins on [0, 200) and
    logarithmic bins on [0.1, 200), 20 and 200 bins; binary search, reverse
    traversal, index mapping and the hybrid lookup table at several sizes."""
    import torch
    import paper_2301_12557_gb300 as P
    import synth
    import oracle

    P.lib()
    torch.cuda.set_device(0)
    R = 200.0
    n = 1 << 27
    total = 6.4e9
    repeat = int(np.ceil(total / n))
    host = synth.s2_samples(n, R, synth.SEED_BASE + 500)
    d = torch.from_numpy(host).cuda()
    configs = {"lin20": np.linspace(0.0, R, 21), "lin200": np.linspace(0.0, R, 201),
               "log20": np.geomspace(0.1, R, 21), "log200": np.geomspace(0.1, R, 201)}
    tables = [64, 256, 1024, 4096, 16384, 49152]
    sampler = ClockSampler(0)
    sampler.start()
    res = {}
    for name, edges in configs.items():
        mapm = "map_lin" if name.startswith("lin") else "map_log"
        methods = [("bsearch", 0), ("reverse", 0), (mapm, 0)] + [("lut", t) for t in tables]
        # parity on a slice against the oracle, then every method on the full stream
        want = oracle.hist_s2(host[: 1 << 22], edges)
        ref = None
        row = {}
        for m, t in methods:
            got, _ = P.pc_hist_s2(d[: 1 << 22], edges, m, table_size=t)
            assert np.array_equal(got, want), (name, m, t)
            full, ms = P.pc_hist_s2(d, edges, m, table_size=t, repeat=repeat)
            if ref is None:
                ref = full
            assert np.array_equal(full, ref), (name, m, t)
            key = m if m != "lut" else f"lut{t}"
            row[key] = {"ms": ms, "ns_per_sample": ms * 1e6 / (n * repeat),
                        "samples_per_s": n * repeat / (ms * 1e-3)}
        best = min((k for k in row if k.startswith("lut")), key=lambda k: row[k]["ms"])
        res[name] = {"methods": row, "best_table": best,
                     "in_range_fraction": float(ref.sum()) / (n * repeat)}
    clocks = sampler.stop()
    line = {"micro": "hist_s2", "metric": "histogram updates per second", "unit": "samples/s",
            "samples": n * repeat, "distinct_samples": n, "repeat": repeat,
            "sampler": "s2 = x^(2/3) R^2, x uniform in [0, 1), R = 200 (App. C), binary32",
            "edges": {"lin": "[0, 200)", "log": "[0.1, 200)"},
            "exact": "every method equals the oracle's histogram on 4M samples and the others on all",
            "results": res, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.micro == "hist":
        return run_micro_hist(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("mocks"):
        return run_batch(args)
    from synth import workloads as W
    w = W.WORKLOADS[args.workload]
    if w.weighted or len(w.pair_kinds) > 1:
        extra = None
        _, world, _ = dist_env()
        if (args.workload == DEFAULT_WORKLOAD and args.config2_steps > 0 and world == 1
                and args.volume_scale == 1.0 and args.structure == "grid"):
            def extra():
                # the 2M-point clustered (s, mu) benchmark, same GPU, same run
                a2 = argparse.Namespace(**vars(args))
                a2.workload = "ns_periodic_n2m_smu40x100"
                a2.steps, a2.warmup = args.config2_steps, 3
                a2.e2e_steps, a2.fp64_steps, a2.tree_steps = 1, 1, 1
                a2.cell_size, a2.ipt, a2.rescue_capacity = 0.0, 0, 0
                a2.no_cpu_baseline = True
                ln = run_ours(a2, emit=False)
                keep = ("value", "unit", "steps", "warmup", "ms_per_step", "config",
                        "candidate_pairs_per_s", "rescued_fraction", "fp64_path", "kdtree_path",
                        "speedup_vs_fp64", "roofline", "e2e", "clocks", "gpu_launches")
                return {a2.workload: {k: ln[k] for k in keep}}
        return run_sets(args, extra)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

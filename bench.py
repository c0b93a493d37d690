#!/usr/bin/env python
"""Benchmark of exact grid pair counting on GB300.

Default workload: 2,000,000 Neyman-Scott points (200,000 parents, Poisson(10)
children, sigma = 5 Mpc/h) in a periodic 1000 Mpc/h cube, auto counts in
(s, mu) bins (40 linear s bins on [0, 200) x 100 mu bins, line of sight z),
FP32 separations with binary64 rescue, int64 counts.

One step = one pass of the whole path over the catalogue already resident in
HBM: canonicalise + grid build (bounds, per-cell counts, scan, scatter),
i-block list, pair kernel (separation, bin lookup, shared histograms), the
binary64 re-evaluation of near-edge pairs (inside the pair kernel or by the
rescue kernel, as tuned), histogram read-back.  The value is in-range pairs
binned per second: the one unit every exact method shares, whatever its cell
size or pruning.

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
FP64_PEAK_NOMINAL = 1.25         # TFLOP/s, GB300 FP64 (non-tensor), nominal


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ns_periodic_n2m_smu40x100")
    ap.add_argument("--fp64-steps", type=int, default=1)
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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"sm_max_mhz": 2070.0}, "fallback"


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


def oracle_sample_rate(D, w, seconds, seed=0, L=None, threads=None):
    """Oracle throughput in in-range pairs binned per second: brute force over
    all pairs of a random sample of i-points against the whole catalogue (the
    cross form of the same pair set), self-pairs excluded.  Returns (rate,
    seconds, sample size, cores, pair evaluations per second)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    kw = dict(box=w.L if L is None else L, periodic=w.periodic, mode=w.mode, los=w.los,
              edges_a=w.edges_a, edges_b=w.edges_b)
    n = D.shape[0]
    m0, dt = 16, 0.0
    while True:      # calibrate on growing samples until one takes >= 1/8 of the budget
        S = np.ascontiguousarray(D[rng.choice(n, m0, replace=False)])
        t = time.perf_counter()
        oracle.count(S, D, threads=threads, **kw)
        dt = max(time.perf_counter() - t, 1e-6)
        if dt >= seconds / 8 or m0 >= n:
            break
        m0 = min(n, m0 * 4)
    m = int(max(1, min(n, m0 * seconds / dt)))
    S = np.ascontiguousarray(D[rng.choice(n, m, replace=False)])
    t = time.perf_counter()
    c, _ = oracle.count(S, D, threads=threads, **kw)
    dt = time.perf_counter() - t
    cores = threads or oracle.default_threads()
    in_range = int(c.sum()) - m        # each sampled point pairs with itself at s = 0
    return in_range / dt, dt, m, cores, m * n / dt


def traffic_record():
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if
    the kernel source is unchanged since it was captured."""
    p = os.path.join(ROOT, "profiles", "pairs_f32_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        rec = json.load(open(p))
        src = open(os.path.join(ROOT, "paper_2301_12557_gb300", "csrc", "pairs_impl.cuh"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec.get("source_sha256_16"):
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
    D = W.make_inputs(w)["D"]
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    samp = None
    for k in range(args.warmup + args.steps):
        r, dt, m, cores, _ = oracle_sample_rate(D, w, per_step, seed=k)
        if k >= args.warmup:
            rates.append((r, dt, m))
        samp = (m, cores)
    tot_pairs = sum(r * dt for r, dt, _ in rates)
    tot_t = sum(dt for _, dt, _ in rates)
    value = tot_pairs / tot_t
    sample = (f"{samp[0]} random i-points x all {D.shape[0]} points per step "
              f"(brute force, binary64); in-range pairs found per second")
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


def run_ours(args):
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
        # counts, against GB300's nominal FP64 (non-tensor) rate
        fl64 = FLOPS_PER_CANDIDATE * float(s64.candidates) + FLOPS_PER_IN_RANGE * inr64
        k64_ms = s64.ms_pairs if s64.ms_pairs > 0 else statistics.mean(ms64)
        ach64 = fl64 / (k64_ms * 1e-3) / 1e12
        fp64 = {"value": inr64 / (statistics.mean(ms64) * 1e-3), "unit": UNIT,
                "cell_size": o64.cell_size,
                "ms_per_step": statistics.mean(ms64), "steps": args.fp64_steps,
                "counts_identical_to_fp32_rescue": exact,
                "roofline": {"bound": "fp64", "achieved": ach64, "peak": FP64_PEAK_NOMINAL,
                             "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_NOMINAL,
                             "peak_source": "nominal GB300 FP64 rate (not measured)",
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
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    ms_pairs = statistics.mean(s.ms_pairs for s in stats)
    cand = stats[0].candidates
    evaluated = cand - stats[0].pruned       # pairs the kernel separated one by one
    flops = FLOPS_PER_CANDIDATE * evaluated + FLOPS_PER_IN_RANGE * inr_step
    achieved = flops / (ms_pairs * 1e-3) / 1e12
    trec = traffic_record()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                # the record holds for the grid kernel with the same rescue mode
                "traffic": (trec["bytes_per_launch"]
                            if trec and not tree and (trec.get("rescue") == "inline") ==
                            (opts.rescue_capacity < 0) else None),
                "kernel": "k_pairs_f32<SMU,LOS_Z>" + (" (tree variant)" if tree else ""),
                "flops_per_launch": flops,
                "flops_definition": (f"{FLOPS_PER_CANDIDATE} per pair evaluated one by one "
                                     f"({evaluated:.4g}) + {FLOPS_PER_IN_RANGE} per in-range "
                                     f"pair ({inr_step:.4g})"),
                "peak_source": (f"FP32 non-tensor: {props.multi_processor_count} SMs x "
                                f"{FP32_LANES_PER_SM} lanes x 2 flops x {sm_mhz:.0f} MHz "
                                f"({peak_src} sm_max_mhz)"),
                "kernel_ms": ms_pairs,
                "kernel_share_of_step": ms_pairs / (t_max / args.steps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
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
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
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

    def step(xs=X, counts=out, batched=True):
        if tree:
            ts = [P.pc_build_tree(x, box=box, n_leaf=args.n_leaf, list_cap=list_cap, stream=stream)
                  for x in xs]
        else:
            ts = [P.pc_build_grid(x, box=box, r_max=bins.r_max, opts=opts, stream=stream)
                  for x in xs]
        try:
            if batched:
                if tree:
                    _, _, st = P.pc_count_tree_batch(ts, bins, opts, stream, counts=counts)
                else:
                    _, _, st = P.pc_count_batch(ts, bins, opts, stream, counts=counts)
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
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name if m == w.extra["m"] else f"{w.name} ({m} mocks)",
                       "mocks": m, "n_total": int(n_tot),
                       "structure": ("k-d tree (leaf capacity %d, list nodes %s), dual-tree "
                                     "traversal per mock" % (args.n_leaf, list_cap or "auto"))
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
            "count_call": ({"ms_total": last_stats[-1].ms_total, "ms_pairs": last_stats[-1].ms_pairs,
                            "ms_rescue": last_stats[-1].ms_rescue}
                           if last_stats and last_stats[-1].ms_total > 0 else None),
            "loop_of_single_counts_ms": loop_ms[0],
            "batched_speedup_vs_loop": loop_ms[0] / (t_max / args.steps),
            "loop_counts_identical": same,
            "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_sets(args):
    """Workloads with weights and several pair kinds (the survey shell's DD,
    DR and RR; the 100M-point weighted cube): every step builds every
    catalogue's grid and runs every count, weighted sums in binary64."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    import paper_2301_12557_gb300 as P
    from synth import workloads as W

    P.lib()
    w = W.WORKLOADS[args.workload]
    inp = W.make_inputs(w, scale=args.volume_scale)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    names = ["D"] + (["R"] if "R" in inp else [])
    host = {k: (inp[k], inp.get("w" + k)) for k in names}
    devc = {k: (torch.from_numpy(x).to(dev), torch.from_numpy(wt).to(dev) if wt is not None else None)
            for k, (x, wt) in host.items()}
    bins = P.Bins(w.mode, w.los, w.edges_a, w.edges_b)
    if w.periodic:
        box = P.make_box(w.L, True)
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
    if tree and (args.list_cap > 0 or args.ipt > 0):
        opts = P.make_opts("f32", 0.0, args.ipt or 2)
    elif tree:
        t0 = time.perf_counter()
        opts, list_cap, trials = P.pc_tune_tree(devc[big][0], devc[big][1], box=box, bins=bins,
                                                n_leaf=args.n_leaf, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on": big,
                  "trials": [{"list_cap": c, "ipt": i, "ms": round(ms, 3)} for c, i, ms in trials]}
    elif args.cell_size > 0 or args.ipt > 0:
        opts = P.make_opts("f32", args.cell_size, args.ipt)
    else:
        t0 = time.perf_counter()
        opts, trials = P.pc_tune(devc[big][0], devc[big][1], box=box, bins=bins, stream=stream)
        tuning = {"seconds": time.perf_counter() - t0, "on": big,
                  "trials": [{"cell_size": round(c, 3), "ipt": i, "priv": pv, "ms": round(ms, 3)}
                             for c, i, pv, ms in trials]}
    kinds = list(w.pair_kinds)
    outs = {k: (torch.zeros(bins.nbins, dtype=torch.int64, device=dev),
                torch.zeros(bins.nbins, dtype=torch.float64, device=dev)) for k in kinds}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(cats=devc, results=outs):
        if tree:
            gs = {k: P.pc_build_tree(x, wt, box=box, n_leaf=args.n_leaf, list_cap=list_cap,
                                     stream=stream)
                  for k, (x, wt) in cats.items()}
        else:
            gs = {k: P.pc_build_grid(x, wt, box=box, r_max=bins.r_max, opts=opts, stream=stream)
                  for k, (x, wt) in cats.items()}
        stats = {}
        try:
            for kind in kinds:
                a, b = gs[kind[0]], gs[kind[1]]
                c, wc = results[kind]
                if tree:
                    _, _, st = P.pc_count_tree(a, None if kind[0] == kind[1] else b, bins, opts,
                                               stream, counts=c, wcounts=wc)
                elif kind[0] == kind[1]:
                    _, _, st = P.pc_count_auto(a, bins, opts, stream, counts=c, wcounts=wc)
                else:
                    _, _, st = P.pc_count_cross(a, b, bins, opts, stream, counts=c, wcounts=wc)
                stats[kind] = st
        finally:
            for g in gs.values():
                g.free()
        return stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = P.pc_launch_count()
    ms, stats = [], None
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        stats = step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    launches = P.pc_launch_count() - l0
    clocks = sampler.stop()
    t_step = statistics.mean(ms)
    inr = {k: int(outs[k][0].sum().item()) for k in kinds}
    value = sum(inr.values()) / (t_step * 1e-3)

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
            assert np.array_equal(hout[k][0], outs[k][0].cpu().numpy()), k
        h2d = sum(x.nbytes + (wt.nbytes if wt is not None else 0) for x, wt in host.values())
        e2e = {"value": sum(inr.values()) / (statistics.mean(e_ms) * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(len(kinds) * bins.nbins * 16),
               "ms_per_step": statistics.mean(e_ms)}

    cpu = None
    if not args.no_cpu_baseline:
        x, wt = host[big]
        r, dt, m, cores, evals = oracle_sample_rate(x, w, args.cpu_seconds, L=w.L)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{m} random {big} points x all {x.shape[0]} {big} points (brute force, "
                         f"binary64, unweighted), {dt:.1f} s; in-range pairs found per second",
               "pair_evaluations_per_s": evals}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name if args.volume_scale == 1.0 else
                   f"{w.name} at N x{args.volume_scale}",
                   "catalogues": {k: int(host[k][0].shape[0]) for k in names},
                   "pair_kinds": kinds, "weighted": bool(w.weighted),
                   "precision": "FP32 separations, binary64 rescue near bin edges, int64 counts, "
                                "binary64 weighted sums",
                   "unit_of_work": "in-range pairs binned over all pair kinds",
                   "structure": ("k-d tree (leaf capacity %d, list nodes %s), dual-tree traversal"
                                 % (args.n_leaf, list_cap or "auto")) if tree else "regular grid",
                   "cell_size": opts.cell_size, "ipt": opts.ipt, "priv": opts.priv,
                   "tuning": tuning, "l2": "flushed between timed steps (256 MiB write)"},
        "per_kind": {k: {"in_range_pairs": inr[k], "ms_pairs": stats[k].ms_pairs,
                         "ms_total": stats[k].ms_total, "candidates": stats[k].candidates,
                         "pruned": stats[k].pruned, "rescued": stats[k].rescued,
                         "node_pairs": stats[k].tree_pairs if tree else None,
                         "ms_traverse": stats[k].ms_traverse if tree else None,
                         "prec": "f32+rescue" if stats[k].prec == 0 else "f64"} for k in kinds},
        "roofline": None,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
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
        return run_sets(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

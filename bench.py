"""Benchmark: one exact mapper graph of the 1,000,000 x 256 clustered cloud.

A step is one complete mapper graph (lens, cover, per-element DBSCAN, nerve)
of the paper-scale workload (1M points x 256 dims, 32 Gaussian clusters plus
5 % uniform noise, L2 lens, 100 intervals at 20 % overlap, eps at the 1st
percentile of sampled distances, minPts 5). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16]
  python bench.py --impl reference      # the FP64 oracle on the host cores

Multi-GPU (torchrun): each rank computes its own graph (independent
replicas, weak scaling); value = graphs of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2011_03209_gb300 import synth  # noqa: E402

LENS_NAMES = {"l2": "L2", "ecc": "eccentricity (exponent 2)", "linf": "L-infinity norm",
              "density": "density (points within eps)", "eccinf": "L-infinity centrality (max distance)"}
METRIC = "mapper graph ms and eps-pair TFLOP/s at 1M\u00d7256, BF16-certified vs FP32, exact graph"
GPU_FP32_LANES = 128                 # FP32 lanes per SM (Blackwell)


def _traffic(st):
    """DRAM bytes of one count pass on the tensor cores (the pairs sent
    straight to three products and both phases of the rest), scaled from the
    ncu captures recorded in profiles/traffic.json by the tile pairs of each
    launch, or None when the kernel source changed since those captures or
    the pass ran in one phase."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2011_03209_gb300", "csrc", "k_tc.cu")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get("tc_kernel_count")
    if not rec or rec.get("source_sha1") != hashlib.sha1(open(src, "rb").read()).hexdigest():
        return None
    if not st.get("tile_pairs_screen1") or "bytes_per_tile_pair_first" not in rec:
        return None
    return (rec["bytes_per_tile_pair_first"] * st["tile_pairs_screen1"] +
            rec["bytes_per_tile_pair_second"] * st["tile_pairs_redo"] +
            rec.get("bytes_per_tile_pair_direct", 0.0) * st.get("tile_pairs_direct", 0))


def _bind_local_cpus(device: int):
    """Run on the CPUs local to the GPU (sysfs local_cpulist of its PCI
    device), so pinned host buffers land in the memory next to it and the
    end-to-end copies run at that link's rate. Returns the CPU list, or None
    when the topology is not readable."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (
            getattr(p, "pci_domain_id", 0), p.pci_bus_id, p.pci_device_id)
        cpus = set()
        for part in open(path).read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return sorted(cpus)
    except Exception:                            # no CUDA device, sysfs or attribute: leave placement alone
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def sampled_oracle(w, budget_s: float, seed: int, gpu_labels=None):
    """Time the FP64 oracle on a bounded sample of the workload: full lens
    and cover, then DBSCAN on cover elements drawn in a seeded order until
    `budget_s` seconds of DBSCAN have run. The full-graph time is
    extrapolated by the sampled share of sum n_i^2 (DBSCAN's brute-force cost
    is proportional to n_i^2 d). Returns (estimated ms, description,
    threads, exact) where exact compares sampled labels with gpu_labels."""
    import oracle
    t0 = time.perf_counter()
    f = oracle.lens(w.X, w.lens_kind, w.lens_arg)
    offs, pts = oracle.cover(f, w.n_intervals, w.overlap)
    t_front = time.perf_counter() - t0
    sizes = np.diff(offs).astype(np.float64)
    total = float((sizes ** 2).sum())
    order = np.random.default_rng(seed).permutation(np.nonzero(sizes)[0])
    spent, share, picked, exact = 0.0, 0.0, [], True
    for e in order:
        if spent >= budget_s:
            break
        if spent > 0 and (sizes[e] ** 2 / max(share, 1.0)) * spent > 4 * budget_s:
            continue                  # would overrun the budget several times over
        s, t = offs[e], offs[e + 1]
        t1 = time.perf_counter()
        _, _, lab, _ = oracle.dbscan(w.X, pts[s:t], w.eps, w.min_pts)
        spent += time.perf_counter() - t1
        share += sizes[e] ** 2
        picked.append(int(e))
        if gpu_labels is not None:
            exact &= bool(np.array_equal(gpu_labels[s:t], lab))
    est_s = t_front + spent * total / max(share, 1.0)
    desc = (f"lens+cover of all {w.n} points, DBSCAN of {len(picked)} of {len(order)} cover "
            f"elements ({100.0 * share / total:.2f}% of sum n_i^2), extrapolated by n_i^2")
    return est_s * 1e3, desc, oracle.num_threads(), exact


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = synth.clusters_1m_d256()
    vals = []
    for i in range(args.warmup + args.steps):
        ms, desc, cores, _ = sampled_oracle(w, args.ref_budget, seed=i)
        if i >= args.warmup:
            vals.append(ms)
    v = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "n": w.n, "d": w.d,
                                        "n_intervals": w.n_intervals[0], "overlap": w.overlap[0],
                                        "eps": w.eps, "min_pts": w.min_pts},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": v, "unit": "ms", "cores": cores, "kind": "oracle",
                         "sample": desc},
    }))


def _device_loop(ctx, stream, Xd, prm, steps, warmup, sampler=None, barrier=lambda: None):
    """Device-resident graphs: `warmup` untimed calls, then `steps` calls
    between two CUDA events on the context's stream. Returns (ms per graph,
    per-call stats)."""
    import torch
    import paper_2011_03209_gb300 as mg

    for _ in range(warmup):
        g = mg.mapper_graph(ctx, Xd, prm)
        g.numpy()
        del g
    torch.cuda.synchronize()
    stats = []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
        time.sleep(0.3)
    start.record(stream)
    for _ in range(steps):
        g = mg.mapper_graph(ctx, Xd, prm)
        stats.append(g.stats())
        del g
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    return start.elapsed_time(end) / steps, stats


def _e2e_loop(ctx, Xh, prm, steps, warmup, barrier=lambda: None):
    """End to end through the public API: host X in (pinned), graph back on
    the host, per call. Warm-up calls first (the first host-input call grows
    the context's memory pool by the device copy of X). Returns (ms per
    graph, bytes copied back per graph)."""
    import torch
    import paper_2011_03209_gb300 as mg

    for _ in range(warmup):
        g = mg.mapper_graph(ctx, Xh.numpy(), prm)
        g.numpy()
        del g
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(steps):
        g = mg.mapper_graph(ctx, Xh.numpy(), prm)
        out = g.numpy()
        d2h = sum(a.nbytes for a in out.values())
        del g
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3 / steps, d2h


def _roofline(prec, w, st, stats, n_sm):
    """Roofline of the dominant kernel: the count pass (tensor cores for the
    BF16 screens, CUDA cores for FP32), from its CUDA-event time in `stats`."""
    import paper_2011_03209_gb300 as mg

    kpairs = st["count_kernel_pairs"]
    kms = float(np.mean([s["ms_count_kernel"] for s in stats]))
    peaks, src = _peaks()
    if prec == mg.FP32:
        clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
        peak = n_sm * GPU_FP32_LANES * 2 * clk / 1e12      # FP32 FFMA peak, TFLOP/s
        achieved = 3.0 * w.d * kpairs / (kms * 1e-3) / 1e12
        return kms, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "simt_pass_kernel<1>: 3d FP32 flops (sub + FMA) per pair screened",
                     "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flops x {clk / 1e6:.0f} MHz (max clock)"}
    peak = peaks["bf16_tflops"]
    achieved = 2.0 * w.d * kpairs / (kms * 1e-3) / 1e12
    tp1 = st.get("tile_pairs_screen1", 0)
    # three products: the second phase's pairs and those sent straight to it
    tp3 = st["tile_pairs_tc"] if not tp1 else st.get("tile_pairs_redo", 0) + st.get("tile_pairs_direct", 0)
    ns = 1 if prec == mg.BF16X1 else 3
    kp = -(-w.d // 64) * 64 * 128.0 * 128.0 * 2.0
    first = 3 if prec == mg.FP8 else 1                 # products of the first phase
    executed = ((tp1 * first * kp + tp3 * 3 * kp) if tp1 else ns * kp * st["tile_pairs_tc"]) / (kms * 1e-3) / 1e12
    if prec == mg.FP8:
        desc = ("tc_kernel count pass (tcgen05): three FP8 E4M3 products per tile pair, then three BF16 "
                "products for the 32 x 32 blocks the first screen leaves open" if tp1 else
                "tc_kernel (tcgen05 FP8 E4M3 count pass): three products per pair")
    else:
        desc = ("tc_kernel count pass (tcgen05 BF16): one product per tile pair, three products for the "
                "32 x 32 blocks the first screen leaves open and for the tile pairs whose bin of the "
                "sampled first phase mostly deferred (phases and bins chosen per call from a sample of "
                "the first phase)" if tp1 else
                "tc_kernel<%d,1> (tcgen05 BF16 count pass): %d BF16 products per pair" % (ns, ns))
    return kms, {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak, "traffic": _traffic(st) if prec == mg.BF16 else None,
                 "kernel": desc + "; achieved counts 2d algorithmic flops per point pair screened",
                 "executed_tflops": executed,
                 "peak_source": f"{src} bf16_tflops (burst: the kernel's launches last a few ms)"}


def run_ours(args):
    import torch
    import paper_2011_03209_gb300 as mg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    prec = {"bf16": mg.BF16, "bf16x1": mg.BF16X1, "fp32": mg.FP32, "fp8": mg.FP8}[args.precision]
    w = synth.clusters_1m_d256(args.n)
    local_cpus = _bind_local_cpus(local)
    Xh = torch.from_numpy(w.X).pin_memory()
    Xd = Xh.to(f"cuda:{local}")
    stream = torch.cuda.Stream()
    ctx = mg.Context(local, stream=stream)
    ctx.set_timing(True)
    if args.pass1_tile_n:
        ctx.set_pass1_tile_n(args.pass1_tile_n)
    if args.screen:
        ctx.set_pass1_screen(args.screen)
    lens_kind = {"l2": w.lens_kind, "ecc": (mg.LENS_ECC,), "linf": (mg.LENS_LINF,),
                 "density": (mg.LENS_DENSITY,), "eccinf": (mg.LENS_ECC_INF,)}[args.lens]
    cover_kind = mg.COVER_BALANCED if args.cover == "balanced" else mg.COVER_UNIFORM

    def params(p):
        return mg.params(lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, p, cover_kind,
                         lens_param=(w.eps,))

    prm = params(prec)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- device-resident timed region
    sampler = ClockSampler(local)
    ms, stats = _device_loop(ctx, stream, Xd, prm, args.steps, args.warmup, sampler, barrier)
    clocks = sampler.stop()
    ms = max_over_ranks(ms)

    # ---- end to end through the public API: host X in, graph back on the host
    ctx.set_timing(False)
    e2e_ms, d2h = _e2e_loop(ctx, Xh, prm, args.steps, args.warmup, barrier)
    e2e_ms = max_over_ranks(e2e_ms)
    ctx.set_timing(True)

    st = stats[-1]
    pairs = st["pairs_screened"]                       # unordered pairs incl. self, pass 1
    eps_pair_flops = 2.0 * w.d * pairs
    pass1_ms = float(np.mean([s["ms_pass"][0] for s in stats]))
    kms, roof = _roofline(prec, w, st, stats, n_sm)

    line = {
        "metric": METRIC, "value": ms / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {mg.FP32: "f32+f64", mg.FP8: "fp8+bf16+f64"}.get(prec, "bf16+f64"),
        "data": "synthetic",
        "config": {"workload": w.name + ("" if args.lens == "l2" else "_" + args.lens)
                   + ("" if args.cover == "uniform" else "_balanced"), "n": w.n, "d": w.d,
                   "lens": LENS_NAMES[args.lens], "cover": args.cover,
                   "n_intervals": w.n_intervals[0], "overlap": w.overlap[0], "eps": w.eps,
                   "min_pts": w.min_pts, "precision": args.precision,
                   "l2_flush": (f"inputs larger than L2 ({w.X.nbytes / 1e9:.2f} GB point cloud read every step)"
                                if w.X.nbytes > 129e6 else
                                f"none: the {w.X.nbytes / 1e6:.0f} MB point cloud fits in L2 (profiling size)"),
                   "parallelism": f"replicas x{world}"},
        "eps_pair_tflops": eps_pair_flops / (pass1_ms * 1e-3) / 1e12,
        "count_kernel_ms": kms,
        "pass_ms": [float(np.mean([s["ms_pass"][i] for s in stats])) for i in range(3)],
        "stage_ms": {k: float(np.mean([s[k] for s in stats]))
                     for k in ("ms_lens", "ms_cover", "ms_cluster", "ms_nerve")},
        "counters": {k: st[k] for k in ("n_members", "n_rows", "n_groups", "sum_ni2", "tile_pairs",
                                        "tile_pairs_out", "tile_pairs_in", "tile_pairs_tc",
                                        "tile_pairs_simt", "union_pairs", "union_skipped", "pairs_screened",
                                        "band_pairs", "fp64_pairs", "near_ties", "n_core", "n_nodes", "n_edges",
                                        "pass1_tile_n", "tile_pairs_cross") + tuple(
                                            k for k in ("tile_pairs_screen1", "tile_pairs_redo", "redo_blocks", "redo_parts", "tile_pairs_direct") if k in st)},
        "ms_tiles": float(np.mean([s["ms_tiles"] for s in stats])),
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": int(sum(s["n_launches"] for s in stats)),
        "e2e": {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": int(w.X.nbytes),
                "d2h_bytes_per_step": int(d2h),
                "host": (f"pinned input, process bound to the {len(local_cpus)} CPUs local to the GPU"
                         if local_cpus else "pinned input, CPU placement left to the system")},
    }
    extras = (world == 1 and rank == 0 and not args.no_extras and args.lens == "l2" and args.cover == "uniform"
              and prec != mg.FP32 and args.n == 1_000_000)
    if extras:
        # the plain FP32 CUDA-core path of the same pipeline (the comparison
        # the metric names), device-resident and end to end
        f_steps = max(1, min(args.steps, 5))
        f_ms, f_stats = _device_loop(ctx, stream, Xd, params(mg.FP32), f_steps, 1)
        ctx.set_timing(False)
        f_e2e, _ = _e2e_loop(ctx, Xh, params(mg.FP32), f_steps, 1)
        ctx.set_timing(True)
        f_kms, f_roof = _roofline(mg.FP32, w, f_stats[-1], f_stats, n_sm)
        line["fp32"] = {"value": f_ms, "unit": "ms", "steps": f_steps,
                        "e2e": {"value": f_e2e, "unit": "ms"}, "count_kernel_ms": f_kms,
                        "roofline": f_roof, "nodes": int(f_stats[-1]["n_nodes"]),
                        "edges": int(f_stats[-1]["n_edges"])}
        line["speedup_vs_fp32"] = f_ms / ms
        line["e2e_speedup_vs_fp32"] = f_e2e / e2e_ms
        line["same_graph_size_as_fp32"] = (int(f_stats[-1]["n_nodes"]) == int(st["n_nodes"]) and
                                           int(f_stats[-1]["n_edges"]) == int(st["n_edges"]))
    if rank == 0 and not args.no_cpu_baseline and args.lens == "l2" and args.cover == "uniform":
        gl = None
        g = mg.mapper_graph(ctx, Xd, prm)
        offs, _ = g.cover().numpy()
        gl, _ = g.clusters().numpy(int(offs[-1]))
        del g
        cms, desc, cores, exact = sampled_oracle(w, args.ref_budget, seed=12345, gpu_labels=gl)
        line["cpu_baseline"] = {"value": cms, "unit": "ms", "cores": cores, "kind": "oracle",
                                "sample": desc}
        line["exact_on_sample"] = exact
    if extras:
        line["small_configs"] = measure_small_configs(ctx, 10)
        line["single_linkage"] = measure_single_linkage(ctx, 3)
    ctx.close()
    if extras:
        del Xd
        torch.cuda.empty_cache()
        line["sweep"] = measure_sweep(2, 1, prec, check_oracle=True)
        line["serving"] = measure_serving(args.requests, 8, args.rate, args.slots, prec, big_X=w.X)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def measure_serving(n_requests: int, warmup: int, rate: float, slots: int, prec, big_X=None) -> dict:
    """Serving mix: nine device-resident clouds, a seeded Poisson request
    stream (mean `rate` per second), requests admitted by device-memory
    footprint into `slots` concurrent slots. Returns graphs/s and the
    p50/p99 latency from submission to a finished graph. big_X: the
    1M x 256 cloud when the caller holds it already."""
    import torch
    import paper_2011_03209_gb300 as mg

    Xs = synth.serving_datasets(seed=4, big_X=big_X)
    samples = [synth.pair_sample(X, 4 + i) for i, X in enumerate(Xs)]
    reqs = synth.serving_requests(samples, n_requests + warmup, rate, seed=4)
    Xd = [torch.from_numpy(X).to("cuda:0") for X in Xs]

    def prm(r):
        return mg.params(r["lens_kind"], r["lens_arg"], r["n_intervals"], r["overlap"], r["eps"],
                         r["min_pts"], prec)

    with mg.Server(0, n_slots=slots) as srv:
        ids = [srv.add_dataset(X) for X in Xd]
        for r in reqs[:warmup]:                           # untimed: first calls, pool growth
            srv.wait(srv.submit(ids[r["dataset"]], prm(r)))
        timed = reqs[warmup:]
        t_base = timed[0]["t"]
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        tickets = []
        for r in timed:
            delay = (r["t"] - t_base) - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(ids[r["dataset"]], prm(r)))
        lat, runs, queued, nodes = [], [], [], 0
        for t in tickets:
            g, info = srv.wait(t)
            lat.append(info["latency_s"] * 1e3)
            runs.append(info["run_s"] * 1e3)
            queued.append(info["queue_s"] * 1e3)
            nodes += g.sizes()[0]
            del g
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
    del Xd
    lat = np.asarray(lat)
    return {"graphs_per_s": len(timed) / wall, "requests": len(timed), "rate_per_s": rate, "slots": slots,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_run_ms": float(np.mean(runs)), "mean_queue_ms": float(np.mean(queued)),
            "max_ms": float(lat.max()), "nodes": int(nodes), "wall_s": wall,
            "datasets": [list(X.shape) for X in Xs], "clocks": clocks}


def run_serving(args):
    """The serving mix as its own JSON line (graphs/s, p50/p99 latency)."""
    import torch
    import paper_2011_03209_gb300 as mg

    torch.cuda.set_device(0)
    prec = {"bf16": mg.BF16, "bf16x1": mg.BF16X1, "fp32": mg.FP32, "fp8": mg.FP8}[args.precision]
    r = measure_serving(args.requests, args.warmup, args.rate, args.slots, prec)
    print(json.dumps({
        "metric": "serving graphs/s (9 resident clouds, Poisson stream)", "value": r["graphs_per_s"],
        "unit": "graphs/s", "n_gpus": 1, "steps": r["requests"], "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f32+f64" if prec == mg.FP32 else "bf16+f64", "data": "synthetic",
        "config": {"workload": "serving_mix_9_clouds", "rate_per_s": args.rate, "slots": args.slots,
                   "datasets": r["datasets"], "precision": args.precision},
        **{k: r[k] for k in ("p50_ms", "p99_ms", "mean_run_ms", "mean_queue_ms", "max_ms", "nodes", "wall_s",
                             "clocks")},
    }))


def measure_sweep(steps: int, warmup: int, prec, check_oracle: bool = False) -> dict:
    """The 2D-lens sweep: 16 graphs (eps at 4 percentiles x 4 overlaps) of
    the 500,000 x 128 Zipf mixture with a (PC1, PC2) lens on a 30 x 30 grid,
    as one mapper_graph_sweep call; also timed as 16 mapper_graph calls.
    check_oracle: compare the cover of the first graph and the DBSCAN of one
    sampled element of every graph with the oracle."""
    import torch
    import paper_2011_03209_gb300 as mg

    w, eps, ov = synth.zipf_sweep()
    Xd = torch.from_numpy(w.X).to("cuda:0")
    stream = torch.cuda.Stream()
    exact = None
    with mg.Context(0, stream=stream) as ctx:
        base = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, eps[0], w.min_pts, prec)
        for _ in range(warmup):
            gs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
            del gs
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            gs = mg.mapper_graph_sweep(ctx, Xd, base, eps, ov)
            nodes = [g.sizes()[0] for g in gs]
            tile_n = gs[0].stats()["pass1_tile_n"]
            if _ < steps - 1:
                del gs
        end.record(stream)
        torch.cuda.synchronize()
        sweep_ms = start.elapsed_time(end) / steps
        if check_oracle:
            import oracle
            rng = np.random.default_rng(7)
            exact = True
            for k, (g, e, p) in enumerate(zip(gs, eps, ov)):
                offs, pts = g.cover().numpy()
                lab, core = g.clusters().numpy(len(pts))
                if k == 0:                      # the cover once (the others share its lens)
                    lens, _ = g.lens(w.n, 2)
                    ro, rp = oracle.cover(lens, w.n_intervals, (p, p))
                    exact &= bool(np.array_equal(ro, offs) and np.array_equal(rp, pts))
                sizes = np.diff(offs)
                cand = np.nonzero((sizes > 0) & (sizes <= 4000))[0]
                el = int(rng.choice(cand))
                s0, t0 = offs[el], offs[el + 1]
                _, rc, rl, _ = oracle.dbscan(w.X, pts[s0:t0], e, w.min_pts)
                exact &= bool(np.array_equal(rc, core[s0:t0]) and np.array_equal(rl, lab[s0:t0]))
        del gs
        start.record(stream)
        for _ in range(steps):
            for e, p in zip(eps, ov):
                g = mg.mapper_graph(ctx, Xd, mg.params(w.lens_kind, w.lens_arg, w.n_intervals, (p, p), e,
                                                       w.min_pts, prec))
                del g
        end.record(stream)
        torch.cuda.synchronize()
        single_ms = start.elapsed_time(end) / steps
    return {"workload": w.name + "_sweep16", "n": w.n, "d": w.d, "lens": "(PC1, PC2)", "grid": [30, 30],
            "eps": eps, "overlap": ov, "min_pts": w.min_pts, "sweep_ms": sweep_ms,
            "ms_per_graph": sweep_ms / len(eps), "single_calls_ms": single_ms,
            "sweep_speedup": single_ms / sweep_ms, "pass1_tile_n": tile_n, "nodes": nodes,
            "exact_on_sample": exact}


def run_sweep(args):
    """The 2D-lens sweep as its own JSON line."""
    import torch
    import paper_2011_03209_gb300 as mg

    torch.cuda.set_device(0)
    prec = {"bf16": mg.BF16, "bf16x1": mg.BF16X1, "fp32": mg.FP32, "fp8": mg.FP8}[args.precision]
    sampler = ClockSampler(0)
    sampler.start()
    r = measure_sweep(args.steps, args.warmup, prec)
    clocks = sampler.stop()
    print(json.dumps({
        "metric": "sweep ms (16 graphs, 500k x 128, 2D lens, 30 x 30 grid)", "value": r["sweep_ms"], "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "dtype": "f32+f64" if prec == mg.FP32 else "bf16+f64", "data": "synthetic",
        "config": {k: r[k] for k in ("workload", "n", "d", "lens", "grid", "eps", "overlap", "min_pts")}
        | {"precision": args.precision},
        **{k: r[k] for k in ("ms_per_graph", "single_calls_ms", "sweep_speedup", "pass1_tile_n", "nodes")},
        "clocks": clocks,
    }))


def measure_single_linkage(ctx, steps: int) -> dict:
    """Single linkage (the minimum spanning forests of the cover elements'
    eps-graphs) of the 100,000 x 64 mixture with its PC1 cover: device time
    of mapper_single_linkage on the given cover, and its forests of the
    smallest, median and largest elements against the oracle's Kruskal."""
    import torch
    import oracle
    import paper_2011_03209_gb300 as mg

    w = synth.mixture_100k()
    Xd = torch.from_numpy(w.X).to(f"cuda:{ctx.device}")
    lens, _ = mg.mapper_lens(ctx, Xd, w.lens_kind, w.lens_arg)
    cover = mg.mapper_cover(ctx, lens, w.n_intervals, w.overlap)
    for _ in range(2):
        f = mg.mapper_single_linkage(ctx, Xd, cover, w.eps)
        del f
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        f = mg.mapper_single_linkage(ctx, Xd, cover, w.eps)
        k = f.size()
        if _ < steps - 1:
            del f
    ms = (time.perf_counter() - t0) * 1e3 / steps
    got = f.numpy()
    offs, pts = cover.numpy()
    sizes = np.diff(offs)
    ne = np.nonzero(sizes)[0]
    exact = True
    for e in (int(ne[np.argmin(sizes[ne])]), int(ne[np.argsort(sizes[ne])[len(ne) // 2]]), int(np.argmax(sizes))):
        u, v, d2 = oracle.msf(w.X, pts[offs[e]:offs[e + 1]], w.eps)
        mine = got["elem"] == e
        exact &= bool(np.array_equal(got["u"][mine], u) and np.array_equal(got["v"][mine], v) and
                      np.array_equal(got["d2"][mine], d2))
    return {"workload": w.name, "eps": w.eps, "ms": ms, "forest_edges": int(k), "exact_on_sample": exact,
            "timing": "host wall clock around mapper_single_linkage (the call syncs), mean of %d" % steps}


def measure_small_configs(ctx, steps: int) -> dict:
    """The two configurations the oracle finishes in full: 5,000 x 8 (blobs
    and a circle, L2 lens) and 100,000 x 64 (16 anisotropic Gaussians, PC1
    lens). Per configuration: the device-resident graph time, the oracle's
    whole graph (lens, cover, DBSCAN of every element, nerve) timed on the
    host cores, and whether the two graphs are equal."""
    import torch
    import oracle
    import paper_2011_03209_gb300 as mg

    out = {}
    for w in (synth.blobs_circle_5k(), synth.mixture_100k()):
        Xd = torch.from_numpy(w.X).to(f"cuda:{ctx.device}")
        prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, mg.BF16)
        for _ in range(3):
            g = mg.mapper_graph(ctx, Xd, prm)
            del g
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            g = mg.mapper_graph(ctx, Xd, prm)
            got = g.numpy()
            if _ < steps - 1:
                del g
        gpu_ms = (time.perf_counter() - t0) * 1e3 / steps
        lens, pca = g.lens(w.n, len(w.lens_kind))
        del g
        t0 = time.perf_counter()
        f = oracle.lens(w.X, w.lens_kind, w.lens_arg)
        ref_own = oracle.mapper_graph(w.X, f, w.n_intervals, w.overlap, w.eps, w.min_pts)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        ref = oracle.mapper_graph(w.X, lens, w.n_intervals, w.overlap, w.eps, w.min_pts)
        exact = all(np.array_equal(got[k], ref[k]) for k in ("node_offsets", "node_members", "node_elem", "edges"))
        out[w.name] = {"gpu_ms": gpu_ms, "oracle_ms": cpu_ms, "oracle_cores": oracle.num_threads(),
                       "exact": bool(exact), "near_ties": int(ref["near_ties"]),
                       "nodes": int(len(got["node_elem"])), "edges": int(len(got["edges"])),
                       "oracle_nodes_own_lens": int(len(ref_own["node_elem"])),
                       "timing": "host wall clock around mapper_graph + copy-out, mean of %d" % steps}
    return out


def run_knn(args):
    """k-th nearest-neighbour distances (k = 5, as in the paper's module for
    choosing eps) of a seeded sample of query rows against the whole 1M x 256
    cloud; the oracle's brute force on a few of the same queries beside it."""
    import torch
    import paper_2011_03209_gb300 as mg

    torch.cuda.set_device(0)
    w = synth.clusters_1m_d256(args.n)
    Xd = torch.from_numpy(w.X).to("cuda:0")
    rng = np.random.default_rng(5)
    q = np.sort(rng.choice(w.n, size=min(args.queries, w.n), replace=False)).astype(np.int32)
    k = 5
    stream = torch.cuda.Stream()
    with mg.Context(0, stream=stream) as ctx:
        for _ in range(args.warmup):
            mg.mapper_knn_distance(ctx, Xd, q, k)
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(args.steps):
            kd = mg.mapper_knn_distance(ctx, Xd, q, k)
        end.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        path = ctx.knn_info()
    ms = start.elapsed_time(end) / args.steps
    # tensor-core screen: 2 d algorithmic flops per (query, point) pair (one
    # product; the kernel executes three BF16 products), over the whole call
    # (operands, screen, FP64 merge and the CUDA-core screen of the queries the
    # lists do not settle)
    peaks, src = _peaks()
    algo = 2.0 * w.d * float(q.size) * w.n
    tflops = algo / (ms * 1e-3) / 1e12
    peak = peaks["bf16_tflops_sustained"]
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sub = q[:4]
        t0 = time.perf_counter()
        ref = oracle.knn_distance(w.X, sub, k)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        assert np.array_equal(ref, kd[:4])
        cpu = {"value": cpu_ms / sub.size * q.size, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{sub.size} of the {q.size} queries, scaled by queries; equal to the GPU values"}
    print(json.dumps({
        "metric": f"k-distance ms ({q.size} queries, k = {k}, {w.n // 1000}k x {w.d})", "value": ms, "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "dtype": "f32+f64",
        "data": "synthetic", "config": {"workload": f"clusters_{w.n // 1000}k_d{w.d}_knn", "queries": int(q.size),
                                        "k": k},
        "queries_per_s": q.size / (ms * 1e-3),
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                     "traffic": None, "executed_tflops": 3.0 * tflops,
                     "kernel": "tc_kernel<3,3,2> (tcgen05 BF16 k-distance screen: a sample of the point tiles "
                               "gives each query a threshold, the full screen keeps the keys below it): 2d "
                               "algorithmic flops per (query, point) pair over the whole call",
                     "peak_source": f"{src} bf16_tflops_sustained"},
        "path": path, "cpu_baseline": cpu, "clocks": clocks,
    }))


def run_sharded(args):
    """One 1M x 256 graph per step with its cover elements split over the
    ranks (longest processing time by n_i^2 d), each rank clustering its
    share; the ranks exchange their nodes (one all-gather) and every rank
    builds the nerve of the merged nodes. Strong scaling: the value is the
    time of one whole graph."""
    import torch
    import paper_2011_03209_gb300 as mg
    from paper_2011_03209_gb300 import sharded

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"bf16": mg.BF16, "bf16x1": mg.BF16X1, "fp32": mg.FP32, "fp8": mg.FP8}[args.precision]
    w = synth.clusters_1m_d256(args.n)
    Xd = torch.from_numpy(w.X).to(f"cuda:{local}")
    stream = torch.cuda.Stream()
    ctx = mg.Context(local, stream=stream)
    prm = mg.params(w.lens_kind, w.lens_arg, w.n_intervals, w.overlap, w.eps, w.min_pts, prec)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            g, _ = sharded.sharded_graph(ctx, Xd, prm)
            del g
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        sampler = ClockSampler(local)
        sampler.start()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(args.steps):
            g, mine = sharded.sharded_graph(ctx, Xd, prm)
            sizes = g.sizes()
            del g
        end.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop()
    ms = start.elapsed_time(end) / args.steps
    if dist is not None:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "strong",
            "vs_baseline": None, "dtype": "bf16+f64" if prec != mg.FP32 else "f32+f64", "data": "synthetic",
            "config": {"workload": f"clusters_{w.n // 1000}k_d{w.d}_sharded", "n": w.n, "d": w.d,
                       "parallelism": f"elements over {world} ranks, one node all-gather",
                       "l2_flush": "inputs larger than L2 (1 GB point cloud read every step)"},
            "elements_rank0": int(mine.size), "nodes": int(sizes[0]), "edges": int(sizes[2]), "clocks": clocks,
        }))
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "bf16x1", "fp32", "fp8"])
    ap.add_argument("--ref-budget", type=float, default=12.0,
                    help="seconds of oracle DBSCAN per reference sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="clusters workload: skip the FP32 arm, the small configurations, the sweep and the "
                         "serving sub-objects (profiling runs)")
    ap.add_argument("--screen", type=int, default=0, choices=[0, 1, 2, 3],
                    help="clusters workload, BF16: pass-1 screen (0: the library default, 1: one product "
                         "first and three products for the tile pairs whose band is not empty, 2: three "
                         "products everywhere, 3: as 1, the first phase deferring every block its rows' "
                         "extremes do not decide)")
    ap.add_argument("--workload", default="clusters", choices=["clusters", "serving", "sweep", "sharded", "knn"],
                    help="clusters: the 1M x 256 graph (default; N ranks = N replicas); serving: the "
                         "request mix; sweep: 16 graphs of the 500k x 128 2D-lens cloud; sharded: the "
                         "1M x 256 graph with its elements split over the ranks")
    ap.add_argument("--requests", type=int, default=200, help="serving: timed requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent slots")
    ap.add_argument("--queries", type=int, default=8192, help="knn: query rows")
    ap.add_argument("--lens", default="l2", choices=sorted(LENS_NAMES),
                    help="clusters workload filter: L2 norm (default), eccentricity (exponent 2), "
                         "L-infinity norm, or density (points within eps); the oracle sample needs "
                         "the L2 filter")
    ap.add_argument("--cover", default="uniform", choices=["uniform", "balanced"],
                    help="clusters workload cover: uniform intervals (default) or balanced (equal counts)")
    ap.add_argument("--pass1-tile-n", type=int, default=0, choices=[0, 128, 256],
                    help="clusters workload: fix the pass-1 tensor-core product shape (0: the context's "
                         "autotuner picks; a fixed shape keeps profiler runs on the same kernel)")
    ap.add_argument("--n", type=int, default=1_000_000,
                    help="points of the clustered cloud (smaller only for profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "sharded":
        run_sharded(args)
    elif args.workload == "knn":
        run_knn(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

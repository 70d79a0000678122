#!/usr/bin/env python
"""Throughput benchmark of the edge-sampled, degree-partitioned triangle count.

Default workload: the largest graph, R-MAT scale 26, edge factor 16,
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 1: the library canonicalises
the 2^30 raw draws (pinned host memory) into m = 1,051,928,416 undirected
edges.  One step counts the graph at p = 1.0 and p = 0.05 (seed = step
index + 1 each): sampling, degree partition, degree-oriented CSR, light and
heavy class counts and the rescaled estimate, all on the GPU.

Metric: input edges processed by the sampler per second (sampled edges/s),
whole job.  The graph (8 GiB of keys in rank order, plus their original
keys) is far larger than L2, so no L2 flush is needed between steps.

The default single-GPU run also measures, as extra keys of the same line,
the batched form (10,000 uneven graphs in one launch against one call per
graph: "batched") and the served form (a Poisson request stream against one
blocking call per request: "served"); --no-extras skips them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat26|chung_lu|dense_core|batch|serve]

Other workloads: chung_lu is the 2^22-vertex, 2^26-edge power-law graph
(p = 1, 0.1, 0.01 per step); dense_core stresses the tensor-core heavy
block; batch and serve time the batched and served forms alone.

With N > 1 (torchrun, one process per GPU) every rank counts its own replica
of the workload (no data-path collective); time is the max over ranks.
--impl reference times the CPU oracle (one thread) on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the headline workload: power-law graph shaped like the paper's social networks
    "chung_lu": {"workload": "chung_lu_n4M_m64M_gamma2.1", "kind": "chung_lu", "n": 1 << 22, "m": 1 << 26,
                 "gamma": 2.1, "wmax": 1e5, "graph_seed": 1, "p_sweep": [1.0, 0.1, 0.01]},
    # the largest graph: R-MAT scale 26, edge factor 16; the library gets the
    # 2^30 raw draws and canonicalises them itself (about 10^9 distinct edges)
    "rmat26": {"workload": "rmat_s26_ef16", "kind": "rmat", "n": 1 << 26, "scale": 26, "edge_factor": 16,
               "abc": (0.57, 0.19, 0.19), "graph_seed": 1, "p_sweep": [1.0, 0.05], "oracle_draws": 1 << 26},
    # heavy-block stress: 16384-vertex core at pair density 0.7 (all heavy) in a
    # sparse 2^20-vertex graph; measures the tensor-core contraction
    "dense_core": {"workload": "dense_core_n1M_core16384_q0.7", "kind": "dense_core", "n": 1 << 20,
                   "core": 16384, "q": 0.7, "m_rest": 4 << 20, "graph_seed": 1, "p_sweep": [1.0]},
    # batched counting: 10000 small uneven graphs, each with its own p and seed
    "batch": {"workload": "batch_10000_er_chunglu2.3", "kind": "batch", "graphs": 10000, "graph_seed": 1},
    # served counting: Poisson request stream over a pool of resident graphs
    # drawn like the batched workload plus 1% requests on Chung-Lu m = 2^23
    "serve": {"workload": "serve_poisson2000_pool2000_plus_chunglu_m8M", "kind": "serve", "rate": 2000.0,
              "small_graphs": 2000, "large": {"n": 1 << 20, "m": 1 << 23, "gamma": 2.1, "wmax": 35000.0},
              "large_graphs": 4, "large_frac": 0.01, "budget": 120 * 10 ** 9, "slots": 3,
              "slot_edges": 1 << 25, "slot_vertices": 1 << 24, "slot_requests": 4096,
              "saturation_requests": 30000, "graph_seed": 2},
}
DEFAULT_WORKLOAD = "rmat26"
WORKLOAD = WORKLOADS[DEFAULT_WORKLOAD]
METRIC = "sampled edges/s"
UNIT = "edges/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of Poisson arrivals")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served comparisons of the default single-GPU run")
    ap.add_argument("--extras-serve-duration", type=float, default=10.0,
                    help="seconds of Poisson arrivals of the served comparison inside the default run")
    ap.add_argument("--rmat-scale", type=int, default=None,
                    help="rmat26: another R-MAT scale (e.g. a smaller case for profiling)")
    ap.add_argument("--no-plain", action="store_true",
                    help="batch: only the batched counts (no autotune, no one-count-per-graph comparison), "
                         "e.g. for a launch list")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_ms(ms: float, ws: int, device) -> float:
    """Max over the ranks of a per-rank time: the job ends with its slowest
    replica (one collective; ws == 1 returns ms)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, steps: int, counts_per_step: int, m: int, elapsed_ms: float) -> float:
    """Whole-job input edges per second: every replica counts its own copy of
    the workload (weak scaling), all within elapsed_ms."""
    return ws * steps * counts_per_step * m / (elapsed_ms / 1000.0)


def make_graph(out=None, count=None):
    """The workload's input pairs: a canonical edge list, or for R-MAT the raw
    draws (written into out when given, e.g. a pinned host array; only the
    first `count` draws when count is given)."""
    import gen
    w = WORKLOAD
    if w["kind"] == "rmat":
        return gen.rmat_draws(w["scale"], w["edge_factor"], *w["abc"], seed=w["graph_seed"], out=out, count=count)
    if w["kind"] == "dense_core":
        return gen.cached("planted_core", gen.planted_core, w["n"], w["core"], w["q"], w["m_rest"], w["graph_seed"])
    return gen.cached("chung_lu", gen.chung_lu, w["n"], w["m"], w["gamma"], w["wmax"], w["graph_seed"])


def recorded_traffic(workload, kernel, algorithmic_bytes=None):
    """DRAM bytes per launch of the roofline kernel on this workload from the
    committed ncu capture (profiles/traffic.json), or None when there is no
    record or a source it depends on has changed (sha1 of the listed files,
    concatenated in order).  A record captured on a smaller case of the same
    graph family (scale_by_algorithmic_bytes) gives its ratio of DRAM bytes
    to algorithmic bytes times this launch's algorithmic_bytes."""
    import hashlib
    try:
        recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["records"]
        for rec in recs:
            if rec["workload"] != workload or rec["kernel"] != kernel:
                continue
            src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in rec["sources"])
            if hashlib.sha1(src).hexdigest()[:12] != rec["sources_sha1_12"]:
                return None
            if rec.get("scale_by_algorithmic_bytes"):
                if not algorithmic_bytes:
                    return None
                return float(rec["dram_bytes"]) / float(rec["algorithmic_bytes"]) * float(algorithmic_bytes)
            return float(rec["dram_bytes"])
    except Exception:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(edges, n):
    """The oracle's bounded sample of the workload: (canonical edges, p, what
    it is).  R-MAT: the subgraph of the first oracle_draws raw draws,
    canonicalised by the oracle, at the sweep's smallest p (the whole graph
    takes hours single-threaded); otherwise the whole graph at p = 0.1."""
    import oracle
    oracle.build()
    w = WORKLOAD
    if w["kind"] == "rmat":
        k = w["oracle_draws"]
        canon = oracle.canonicalize(edges[:k], n)
        p = min(w["p_sweep"])
        return canon, p, ("the subgraph of the first %d of the %d raw draws (%d distinct edges, canonicalised "
                          "by the oracle), p=%g" % (k, w["edge_factor"] << w["scale"], len(canon), p))
    return edges, 0.1, "the full graph at p=0.1 (one of the sweep legs; the p=1 leg takes minutes)"


def cpu_baseline(edges, n):
    """The oracle (one thread) on its bounded sample of the workload, seed 1."""
    import oracle
    canon, p, what = oracle_sample(edges, n)
    t0 = time.perf_counter()
    oracle.run(canon, n, p, 1)
    dt = time.perf_counter() - t0
    return {"value": len(canon) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "CPU oracle, 1 thread, %s: %s, seed 1: %.2f s for %d input edges" %
                      (WORKLOAD["workload"], what, dt, len(canon))}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n = WORKLOAD["n"]
    count = WORKLOAD.get("oracle_draws") if WORKLOAD["kind"] == "rmat" else None
    edges, p, what = oracle_sample(make_graph(count=count), n)
    import oracle
    for i in range(args.warmup):
        oracle.run(edges, n, p, i + 1)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(edges, n, p, k + 1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * len(edges) / total
    sample = ("CPU oracle, 1 thread: each step is %s (seed = step + 1) of the %s workload"
              % (what, WORKLOAD["workload"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD["workload"], "n": n, "m": len(edges),
                                            "p_sweep": [p]},
            "same_config": False,
            "note": ("the oracle takes hours on the whole graph at every p of the sweep, so each step is a "
                     "bounded sample: %s; the GPU arm counts the whole graph at p in %s"
                     % (what, WORKLOAD["p_sweep"])),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def our_arm(args):
    import numpy as np
    import torch
    from paper_1011_0468_gb300 import tc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    tc.lib()
    tc.use_torch_allocator(True)

    n, ps = WORKLOAD["n"], WORKLOAD["p_sweep"]
    if WORKLOAD["kind"] == "rmat":  # raw draws straight into pinned memory
        w = WORKLOAD
        host = torch.empty((w["edge_factor"] << w["scale"], 2), dtype=torch.int32, pin_memory=True)
        edges = make_graph(out=host.numpy().view(np.uint32))
    else:
        edges = make_graph()
        host = torch.from_numpy(edges).pin_memory()
    m_in = len(edges)
    stream = torch.cuda.Stream()
    res_buf = torch.zeros((len(ps), ctypes.sizeof(tc.tc_result)), dtype=torch.uint8, pin_memory=True)

    g = tc.Graph.from_address(host.data_ptr(), m_in, n, on_device=False, stream=stream)
    m = g.m  # distinct undirected edges: the unit of the metric
    assert WORKLOAD["kind"] == "rmat" or m == m_in

    def step(k):
        for j, p in enumerate(ps):
            g.count_async(p, k + 1, res_buf[j].data_ptr())

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for k in range(args.warmup):
        step(k)
    g.sync()
    # ---- timed region: device time of K steps on the graph's stream
    g.set_timing(True)
    g.timing_drain()
    l0 = tc.tc_launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clocks:
        e0.record(stream)
        for k in range(args.steps):
            step(k)
        e1.record(stream)
        g.sync()
        torch.cuda.synchronize()
    launches = tc.tc_launch_count() - l0
    elapsed_ms = e0.elapsed_time(e1)
    phases = g.timing_drain(4 * len(ps) * max(args.steps, 1))
    g.set_timing(False)
    results = [tc.tc_result.from_address(res_buf[j].data_ptr()).as_dict() for j in range(len(ps))]
    barrier()
    elapsed_ms = reduce_max_ms(elapsed_ms, ws, "cuda")
    value = job_throughput(ws, args.steps, len(ps), m, elapsed_ms)

    # ---- roofline of the dominant launch group: the intersection kernels
    # (k_probe_warp + k_probe_block) of the p = 1 count, timed live per count
    # with CUDA events on the graph's stream
    peaks, peak_src = measured_peaks()
    ph = np.asarray(phases, dtype=np.float64) if len(phases) else np.zeros((len(ps), 8))
    per_leg = {p: ph[j::len(ps)].mean(axis=0) for j, p in enumerate(ps)}
    j1 = ps.index(1.0)
    t_isect = float(per_leg[1.0][2]) / 1000.0
    b_isect = 4.0 * (results[j1]["src_elems"] + results[j1]["nbr_elems"])
    achieved = b_isect / t_isect / 1e9 if t_isect > 0 else 0.0
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = recorded_traffic(WORKLOAD["workload"], "k_probe_warp+k_probe_block", b_isect)
    roofline = {"bound": "hbm", "kernel": "k_probe_warp+k_probe_block (p=1 count)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src, "traffic": traffic,
                "algorithmic_bytes_per_launch": b_isect, "launch_ms": t_isect * 1000.0,
                "phase_ms": {str(p): {"sample": float(per_leg[p][0]), "csr": float(per_leg[p][1]),
                                      "intersect": float(per_leg[p][2]), "heavy": float(per_leg[p][3])}
                             for p in ps}}
    if traffic:
        roofline["traffic_gbs"] = traffic / t_isect / 1e9
    if WORKLOAD["kind"] == "dense_core":
        # the heavy block dominates: tensor-core roofline of k_heavy_tc
        t_heavy = float(per_leg[1.0][3]) / 1000.0
        flops = float(results[j1]["heavy_mma_flops"])
        h = float(results[j1]["n_heavy"])
        # fp8 e4m3 operands: the measured bf16 burst peak times the nominal
        # fp8 / bf16 dense ratio (4.5 / 2.25 PFLOP/s)
        tf = 2.0 * float(peaks.get("bf16_tflops", 1900.0))
        roofline = {"bound": "tensor", "kernel": "k_heavy_tc (p=1 count)",
                    "achieved": flops / t_heavy / 1e12 if t_heavy > 0 else 0.0, "peak": tf,
                    "unit": "TFLOP/s", "frac": (flops / t_heavy / 1e12) / tf if t_heavy > 0 else 0.0,
                    "peak_source": peak_src + " bf16 burst x 2 (fp8 e4m3 operands; kernel of a few ms inside one count)",
                    "traffic": recorded_traffic(WORKLOAD["workload"], "k_heavy_tc"),
                    "executed_flops_per_launch": flops,
                    "useful_flops_per_launch": h * (h - 1) * (h - 2) / 3.0, "launch_ms": t_heavy * 1000.0,
                    "phase_ms": {str(p): {"sample": float(per_leg[p][0]), "csr": float(per_leg[p][1]),
                                          "intersect": float(per_leg[p][2]), "heavy": float(per_leg[p][3])}
                                 for p in ps}}
        if roofline["traffic"] and t_heavy > 0:
            roofline["traffic_gbs"] = roofline["traffic"] / t_heavy / 1e9

    # ---- end to end through the C ABI from pinned host memory
    e2e_steps = max(1, min(5, args.steps))
    out_host = torch.zeros((len(ps), ctypes.sizeof(tc.tc_result)), dtype=torch.uint8, pin_memory=True)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        h = tc.Graph.from_address(host.data_ptr(), m_in, n, on_device=False, stream=stream)
        for j, p in enumerate(ps):
            h.count_async(p, k + 1, out_host[j].data_ptr())
        h.sync()
        h.close()
    e2e_s = reduce_max_ms(1000.0 * (time.perf_counter() - t0), ws, "cuda") / 1000.0
    e2e_value = job_throughput(ws, e2e_steps, len(ps), m, 1000.0 * e2e_s)

    g.close()
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline and WORKLOAD["kind"] in ("chung_lu", "rmat"):
            cpu = cpu_baseline(edges, n)
        extras = {}
        if ws == 1 and not args.no_extras and WORKLOAD["kind"] in ("chung_lu", "rmat"):
            # the batched and served forms against the plain path, on the same
            # GPU, after the single graph's memory is returned
            del edges, host
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            tc.release_cached_memory()
            extras["batched"] = run_batch(WORKLOADS["batch"], steps=max(1, min(5, args.steps)), warmup=2)
            torch.cuda.empty_cache()
            tc.release_cached_memory()
            extras["served"] = run_serve(WORKLOADS["serve"], args.extras_serve_duration)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD["workload"], "n": n, "m": m, "m_input_pairs": m_in, "p_sweep": ps,
                           "counts_per_step": len(ps), "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (%d MiB edge list)" % (8 * m >> 20)},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(8 * m_in),
                        "d2h_bytes_per_step": int(len(ps) * ctypes.sizeof(tc.tc_result)),
                        "steps": e2e_steps, "includes": "tc_graph_create from pinned host pairs + %d counts "
                                                        "+ result copies + destroy" % len(ps)},
                "gpu_launches": int(launches), "clocks": clocks.summary(),
                "results": [{k: r[k] for k in ("m_sampled", "n_heavy", "t_light", "t_heavy", "estimate")}
                            for r in results],
                "kept_edges_per_s": ws * args.steps * sum(r["m_sampled"] for r in results) / (elapsed_ms / 1e3)}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def make_batch_graphs(count: int, seed: int = 1):
    """The batched workload: `count` graphs, n log-uniform in [100, 50000],
    average degree uniform in [4, 64], alternating Erdos-Renyi and Chung-Lu
    (exponent 2.3), p from {0.1, 0.5, 1.0}, sampling seed = index + 1."""
    from concurrent.futures import ThreadPoolExecutor
    import gen
    specs = gen.batch_specs(count, seed=seed)
    with ThreadPoolExecutor(max(4, os.cpu_count() or 4)) as ex:
        graphs = list(ex.map(gen.batch_graph, specs))
    return specs, graphs


def run_batch(w, steps: int, warmup: int, plain_steps: int = 3, compare: bool = True) -> dict:
    """Batched counting (tc_batch_*) against the plain one-count-per-graph
    path on the same GPU, same graphs, same (p, seed): the result line (a
    dict) of workload w (WORKLOADS["batch"]).  compare=False: the batched
    counts alone, under the default schedule."""
    import numpy as np
    import torch
    from paper_1011_0468_gb300 import tc

    tc.lib()
    specs, graphs = make_batch_graphs(w["graphs"], w["graph_seed"])
    k = len(graphs)
    p = np.array([s["p"] for s in specs], dtype=np.float64)
    seeds = np.array([s["seed"] for s in specs], dtype=np.uint64)
    batch = tc.Batch([(g, s["n"]) for g, s in zip(graphs, specs)])
    m_total = batch.m
    schedule = batch.autotune(p, seeds) if compare else "default"
    for i in range(warmup):
        batch.count(p, seeds + np.uint64(i))
    l0 = tc.tc_launch_count()
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            res = batch.count(p, seeds + np.uint64(i))
        t_batch = time.perf_counter() - t0
    launches = tc.tc_launch_count() - l0
    batch.close()
    if not compare:
        return {"metric": "batched graphs/s", "value": steps * k / t_batch, "unit": "graphs/s", "n_gpus": 1,
                "steps": steps, "warmup": warmup, "ms_per_step": 1000 * t_batch / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": w["workload"], "graphs": k, "m_total": int(m_total), "schedule": schedule},
                "gpu_launches": int(launches), "clocks": clocks.summary()}

    # plain path: the same graphs resident one per object, one count per call
    tc.use_torch_allocator(True)
    objs = [tc.Graph(g, s["n"]) for g, s in zip(graphs, specs)]
    buf = torch.zeros((k, ctypes.sizeof(tc.tc_result)), dtype=torch.uint8, pin_memory=True)
    for i in range(1):
        for j, o in enumerate(objs):
            o.count_async(float(p[j]), int(seeds[j]), buf[j].data_ptr())
        for o in objs:
            o.sync()
    plain_steps = max(1, min(steps, plain_steps))
    t0 = time.perf_counter()
    for i in range(plain_steps):
        for j, o in enumerate(objs):
            o.count_async(float(p[j]), int(seeds[j]) + i, buf[j].data_ptr())
        for o in objs:
            o.sync()
    t_plain = time.perf_counter() - t0
    plain = np.frombuffer(buf.numpy().tobytes(), dtype=tc.RESULT_DTYPE)
    # the last plain step used seed + (plain_steps - 1); compare with a batch
    # count at the same seeds
    with tc.Batch([(g, s["n"]) for g, s in zip(graphs, specs)]) as b2:
        ref = b2.count(p, seeds + np.uint64(plain_steps - 1))
    identical = bool(all(np.array_equal(ref[f], plain[f]) for f in ("m_sampled", "n_heavy", "t_light", "t_heavy",
                                                                      "estimate")))
    for o in objs:
        o.close()

    value = steps * k / t_batch
    plain_value = plain_steps * k / t_plain
    line = {"metric": "batched graphs/s", "value": value, "unit": "graphs/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1000 * t_batch / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w["workload"], "graphs": k, "m_total": int(m_total),
                       "n_total": int(sum(s["n"] for s in specs)), "schedule": schedule},
            "edges_per_s": steps * m_total / t_batch,
            "plain": {"value": plain_value, "unit": "graphs/s", "ms_per_step": 1000 * t_plain / plain_steps,
                      "path": "one tc_count_async per graph, graphs resident"},
            "speedup_vs_plain": value / plain_value, "identical_to_plain": identical,
            "gpu_launches": int(launches), "clocks": clocks.summary(),
            "t_total_estimate_sum": float(np.sum(res["estimate"]))}
    return line


def batch_arm(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(run_batch(WORKLOAD, args.steps, args.warmup, compare=not args.no_plain)), flush=True)


def serve_requests(w, n_small, duration, seed=7):
    """The request stream: Poisson arrivals at w["rate"] per second for
    `duration` seconds; each request names a graph (a large one with
    probability w["large_frac"], else a uniform small one), p from
    {0.1, 0.5, 1.0} and a seed."""
    import numpy as np
    rng = np.random.default_rng(seed)
    k = int(rng.poisson(w["rate"] * duration))
    t = np.sort(rng.uniform(0.0, duration, size=k))
    large = rng.random(k) < w["large_frac"]
    gid = np.where(large, n_small + rng.integers(0, w["large_graphs"], size=k), rng.integers(0, n_small, size=k))
    p = rng.choice([0.1, 0.5, 1.0], size=k)
    sd = rng.integers(1, 2 ** 63, size=k, dtype=np.uint64)
    return t, gid, p, sd


def _sleep_until(t_abs):
    while True:
        dt = t_abs - time.perf_counter()
        if dt <= 0:
            return
        if dt > 3e-4:
            time.sleep(dt - 2e-4)


def _pct(x, q):
    import numpy as np
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def run_serve(w, duration: float) -> dict:
    """Served counting (tc_server_*) under a Poisson request stream of
    `duration` seconds, against the plain path (one blocking tc_count per
    request, in arrival order) on the same stream; then both at saturation.
    Returns the result line (a dict) of workload w (WORKLOADS["serve"])."""
    import queue
    import threading
    import numpy as np
    import torch
    import gen
    from paper_1011_0468_gb300 import tc

    tc.lib()
    specs, small = make_batch_graphs(w["small_graphs"], w["graph_seed"])
    L = w["large"]
    large = [gen.cached("chung_lu", gen.chung_lu, L["n"], L["m"], L["gamma"], L["wmax"], 100 + i)
             for i in range(w["large_graphs"])]
    pool = [(g, s["n"]) for g, s in zip(small, specs)] + [(g, L["n"]) for g in large]
    t_arr, gid, p, sd = serve_requests(w, len(small), duration)
    R = len(t_arr)
    KEYS = ("m_sampled", "n_heavy", "t_light", "t_heavy", "estimate")

    srv = tc.Server(w["budget"], slots=w["slots"], slot_edges=w["slot_edges"], slot_vertices=w["slot_vertices"],
                    slot_requests=w["slot_requests"])
    t0 = time.perf_counter()
    for e, n in pool:
        srv.add_graph(e, n)
    t_add = time.perf_counter() - t0
    # warm-up: every large graph and a few small ones once
    for t in [srv.submit(len(small) + i, 1.0, 1) for i in range(len(large))] + \
             [srv.submit(i, 0.5, 1) for i in range(0, len(small), 50)]:
        srv.wait(t)

    # ---- served: Poisson arrivals, a collector thread waits in ticket order
    tickets = queue.Queue()
    served = [None] * R

    def collect():
        for i in range(R):
            served[i] = srv.wait(tickets.get(), 600000)

    col = threading.Thread(target=collect)
    col.start()
    l0 = tc.tc_launch_count()
    s0 = srv.stats()
    with ClockSampler(0) as clocks:
        base = time.perf_counter() + 0.05
        for i in range(R):
            _sleep_until(base + t_arr[i])
            tickets.put(srv.submit(int(gid[i]), float(p[i]), int(sd[i])))
        col.join()
    launches = tc.tc_launch_count() - l0
    st = srv.stats()
    lat = np.array([(r["t_done_us"] - r["t_submit_us"]) / 1000.0 for r in served])
    qwait = np.array([(r["t_admit_us"] - r["t_submit_us"]) / 1000.0 for r in served])
    span = (max(r["t_done_us"] for r in served) - min(r["t_submit_us"] for r in served)) / 1e6
    waves = st["waves"] - s0["waves"]

    # ---- plain: one blocking tc_count per request in arrival order
    objs = [tc.Graph(e, n) for e, n in pool]
    for o in objs[len(small):]:
        o.count(1.0, 1)
    plain_lat = np.zeros(R)
    plain_res = [None] * R
    base = time.perf_counter() + 0.05
    for i in range(R):
        arr = base + t_arr[i]
        _sleep_until(arr)
        plain_res[i] = objs[gid[i]].count(float(p[i]), int(sd[i]))
        plain_lat[i] = (time.perf_counter() - arr) * 1000.0
    plain_span = time.perf_counter() - base
    identical = all(served[i]["status"] == 0 and all(served[i][k] == plain_res[i][k] for k in KEYS)
                    for i in range(R))

    # ---- saturation: the first S requests all at once
    S = min(R, w["saturation_requests"])
    t0 = time.perf_counter()
    tk = [srv.submit(int(gid[i]), float(p[i]), int(sd[i])) for i in range(S)]
    sat = [srv.wait(t, 600000) for t in tk]
    t_sat = time.perf_counter() - t0
    sat_identical = all(sat[i][k] == served[i][k] for i in range(S) for k in KEYS)
    buf = torch.zeros((S, ctypes.sizeof(tc.tc_result)), dtype=torch.uint8, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(S):
        objs[gid[i]].count_async(float(p[i]), int(sd[i]), buf[i].data_ptr())
    for o in objs:
        o.sync()
    t_plain_sat = time.perf_counter() - t0
    for o in objs:
        o.close()
    srv.close()

    edges = np.array([len(e) for e, _ in pool], dtype=np.float64)
    line = {"metric": "served requests/s", "value": R / span, "unit": "requests/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1000.0 * span, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w["workload"], "requests": R, "rate_per_s": w["rate"],
                       "duration_s": duration, "pool_graphs": len(pool),
                       "pool_input_edges": int(edges.sum()), "large_frac": w["large_frac"],
                       "budget_bytes": w["budget"], "slots": w["slots"], "slot_edges": w["slot_edges"],
                       "slot_requests": w["slot_requests"]},
            "latency_ms": {"p50": _pct(lat, 50), "p99": _pct(lat, 99), "mean": float(lat.mean()),
                           "max": float(lat.max()), "queue_p50": _pct(qwait, 50), "queue_p99": _pct(qwait, 99)},
            "plain": {"latency_ms": {"p50": _pct(plain_lat, 50), "p99": _pct(plain_lat, 99),
                                     "mean": float(plain_lat.mean()), "max": float(plain_lat.max())},
                      "value": R / plain_span, "path": "one blocking tc_count per request, arrival order"},
            "identical_to_plain": bool(identical),
            "saturation": {"requests": S, "served_per_s": S / t_sat, "plain_per_s": S / t_plain_sat,
                           "speedup_vs_plain": t_plain_sat / t_sat, "identical": bool(sat_identical),
                           "plain_path": "one tc_count_async per request, graphs resident"},
            "server": {"waves": waves, "mean_wave": R / max(waves, 1), "max_wave": st["max_wave"],
                       "resident_bytes": st["resident_bytes"], "slot_bytes": st["slot_bytes"],
                       "uploads": st["uploads"], "evictions": st["evictions"], "add_graph_s": t_add},
            "gpu_launches": int(launches), "clocks": clocks.summary()}
    return line


def serve_arm(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(run_serve(WORKLOAD, args.duration)), flush=True)


def select_workload(name: str, rmat_scale=None) -> dict:
    """A copy of WORKLOADS[name]; for R-MAT, rmat_scale (if given) replaces the
    scale, the vertex count, the name and caps the oracle's sample."""
    w = dict(WORKLOADS[name])
    if rmat_scale is not None and w["kind"] == "rmat":
        sc = int(rmat_scale)
        w.update(scale=sc, n=1 << sc, workload="rmat_s%d_ef%d" % (sc, w["edge_factor"]),
                 oracle_draws=min(w["oracle_draws"], w["edge_factor"] << sc))
    return w


def main():
    global WORKLOAD
    args = parse_args()
    WORKLOAD = select_workload(args.workload, args.rmat_scale)
    if WORKLOAD["kind"] == "serve":
        if args.impl == "ours":
            serve_arm(args)
        return
    if WORKLOAD["kind"] == "batch":
        if args.impl == "ours":
            batch_arm(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()

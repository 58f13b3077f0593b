#!/usr/bin/env python
"""Benchmark: Dupin batch peeling (Algorithm 2) on one GB300, and replicas on N.

Default workload (the largest single-GPU configuration): an undirected R-MAT
graph of scale 24 (16,777,216 vertices, 16 * 2^24 draws with a = 0.57,
b = c = 0.19, self-loops dropped and pairs merged: 260,377,346 edges) with
Fraudar weights c = 1/ln(d_obj + 5) in Q32.32, peeled with the FD and the DG
metric at the threshold (1 + eps) g(S) (k_mult = 1, eps = 1/10).  One step =
the two peels of the whole hot path (initial weights, grid-wide rounds, tail
sub-graph, tail rounds on one CTA or a thread-block cluster) in one batched
call.  Beside it (not the headline): the same graph at k_mult = 2 and the DW
metric (c uniform in 1..100, a uniform in 0..10) at k_mult = 1.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]

value     edges peeled per second over all ranks (2 * m per step per rank),
          graph resident in HBM, results left in device memory;
e2e       the same metric through the C ABI with host buffers: each step
          loads the graph from pinned host memory, validates it, peels it
          with both metrics and copies every result (peel rounds, best mask,
          trace) back;
roofline  the dominant kernel's algorithmic bytes per launch / its CUDA-event
          time, against the measured HBM copy bandwidth;
cpu_baseline  the single-threaded C oracle on one of the step's peels of the
          full graph.
Multi-GPU: replicas only (every rank peels its own copy; no collective on
the data path), so scaling is weak.
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

from typing import Optional

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# name -> the graph, the peels of one step (metric, eps) and k_mult.  A batched
# call runs its peels' grid-wide stages in the order given, each tail beside
# the later peels' grid-wide stages, so the step lists the peel with the
# longest tail first (FD: its weights rarely tie, so the minimum rule removes
# few vertices per round; DG's integer degrees tie often).
WORKLOADS = {
    "rmat24": dict(graph="rmat24_fd", peels=[("fd", (1, 10)), ("dg", (1, 10))], k=1),
    "rmat24_dw": dict(graph="rmat24_dw", peels=[("dw", (1, 10))], k=1),
    # R-MAT scale 22 (4.2M vertices, 64M edges): the profiling case of the R-MAT runs
    "rmat22": dict(graph="rmat22_fd", peels=[("fd", (1, 10)), ("dg", (1, 10))], k=1),
    "fd_2Mx1M_40M": dict(graph="fd_2Mx1M_40M", peels=[("fd", (0, 1)), ("fd", (1, 20)), ("fd", (1, 5))], k=1),
    "dg_block_10kx5k": dict(graph="dg_block_10kx5k", peels=[("dg", (1, 10))], k=1),
    # the FD generator at a quarter of the size: a profiling case (arcs still exceed L2)
    "fd_500kx250k_8M": dict(graph="fd_500kx250k_8M", peels=[("fd", (0, 1)), ("fd", (1, 20)), ("fd", (1, 5))], k=1),
}
# the reference arm's per-step sample of each workload (the oracle on the full
# R-MAT-24 graph takes tens of seconds per peel): the same generator at scale 22
REFERENCE_SAMPLE = {"rmat24": "rmat22_fd", "rmat24_dw": "rmat22_dw"}


def make_graph(name: str):
    from paper_2504_09311_gb300 import synth

    if name == "fd_2Mx1M_40M":
        return synth.fd_camouflage(seed=1)
    if name.startswith("rmat"):
        scale, metric = name[len("rmat"):].split("_")
        return synth.rmat_weighted(int(scale), 16, metric, seed=1)
    if name == "dg_block_10kx5k":
        return synth.dg_planted_block(seed=1)
    if name == "fd_500kx250k_8M":
        return synth.fd_camouflage(seed=1, nU=500_000, nI=250_000, m_bg=8_000_000)
    raise ValueError(name)


def dw_copy(g):
    """The same topology with DW weights (c uniform in 1..100, a in 0..10)."""
    from paper_2504_09311_gb300 import synth

    h = synth.SynthGraph(g.n_left, g.n_right, g.eu, g.ev)
    synth.with_weights(h, "dw", 1, a_range=(0, 10), c_range=(1, 100))
    return h


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def algorithmic_bytes(g, pr, trace_size, n_bulk, metric):
    """Bytes the method must move, per phase (see the design notes).

    init: read c (8 B/arc; DG: none, w from the row offsets) + a, w, offsets;
    bulk rounds 1..n_bulk: live scan 12 B per live vertex per round, 52 B per
    peeled vertex (round mark, offsets, staging, frontier), 16 B per arc of a
    peeled vertex (col 4, c 8, neighbour round 4; DG 8 B), 16 B per decrement;
    tail (rounds > n_bulk): the live sub-graph build reads the arcs of the
    live vertices (16 B/arc) and writes the live arcs (12 B), then the same
    per-arc / per-decrement bytes over the sub-graph.
    """
    ptr, idx, _ = g.symmetric_csr()
    deg = np.diff(ptr)
    A = int(ptr[-1])
    n = g.n
    arc_b = 8 if metric == "dg" else 16
    init_b = (0 if metric == "dg" else 8 * A) + 32 * n
    bulk_v = pr <= n_bulk
    u, v = g.global_edges()
    pu, pv = pr[u], pr[v]
    lo = np.minimum(pu, pv)
    dec = (pu != pv)
    bulk_arcs = int(deg[bulk_v].sum())
    bulk_dec = int((dec & (lo <= n_bulk)).sum())
    scan_bulk = int(np.sum(trace_size[:n_bulk]))
    bulk_b = 12 * scan_bulk + 52 * int(bulk_v.sum()) + arc_b * bulk_arcs + 16 * bulk_dec
    tail_v = ~bulk_v
    tail_arcs_full = int(deg[tail_v].sum())
    both_tail = (pu > n_bulk) & (pv > n_bulk)
    tail_live_arcs = 2 * int(both_tail.sum())
    build_b = 16 * tail_arcs_full + 12 * tail_live_arcs
    tail_dec = int((dec & (lo > n_bulk)).sum())
    tail_b = arc_b * tail_live_arcs + 16 * tail_dec + 8 * int(tail_v.sum())
    return {"init": init_b, "bulk": bulk_b, "build": build_b, "tail": tail_b,
            "bulk_arcs": bulk_arcs, "tail_live_arcs": tail_live_arcs}


def bench_batched(dupin, stream, args):
    """4,096 transaction windows (edges log-uniform in 1k..500k, FD, eps=1/10, k=1) peeled by one
    dupin_peel_batch call vs one dupin_peel per graph; results must be identical."""
    import torch

    from paper_2504_09311_gb300 import synth

    t0 = time.perf_counter()
    gs = synth.transaction_windows(args.windows, seed=1)
    tgen = time.perf_counter() - t0
    dgs = [dupin.Graph.from_synth(g) for g in gs]
    ps = [dupin.make_params("fd", 1, (1, 10)) for _ in gs]
    cta_threads = dupin.batch_tune(dgs, ps, stream=stream)  # the autotuner picks the launch shape
    # page-locked peel-round buffers, allocated once and reused by every call (a service's result pool)
    bufs = dupin.BatchBuffers.for_graphs(dgs, want_rounds=True, pinned=True)
    for _ in range(2):
        dupin.peel_batch(dgs, ps, stream=stream, buffers=bufs)
    torch.cuda.synchronize()
    reps = 3
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        outs = dupin.peel_batch(dgs, ps, want_rounds=True, stream=stream, buffers=bufs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    tb = sum(times) / reps
    t0 = time.perf_counter()
    singles = [dupin.peel(dg, "fd", 1, (1, 10), want_mask=False, want_trace=False, stream=stream) for dg in dgs]
    torch.cuda.synchronize()
    tl = time.perf_counter() - t0
    same = all(np.array_equal(a.peel_round, b.peel_round) and a.best_round == b.best_round and a.best_f == b.best_f
               for a, b in zip(outs, singles))
    # a seeded sample of the windows against the CPU oracle
    import oracle

    sample = list(range(0, len(gs), max(1, len(gs) // 64)))[:64]
    bad = 0
    for j in sample:
        og = oracle.Graph.from_synth(gs[j], "fd")
        r = oracle.peel_batch(og, 1, (1, 10))
        og.close()
        o = outs[j]
        bad += 0 if (np.array_equal(o.peel_round, r.peel_round) and o.best_round == r.best_round and
                     o.best_f == r.best_f and o.n_rounds == r.n_rounds) else 1
    edges = int(sum(g.m for g in gs))
    for dg in dgs:
        dg.free()
    return {"workload": f"{args.windows} bipartite windows, edges log-uniform 1k..500k (total {edges}), FD, "
                        "eps=1/10, k=1", "graphs_per_s": args.windows / tb, "edges_per_s": edges / tb,
            "ms": tb * 1e3, "ms_best": min(times) * 1e3, "calls": reps,
            "one_launch_per_graph_graphs_per_s": args.windows / tl, "speedup": tl / tb,
            "identical_to_single": bool(same), "oracle_checked": len(sample), "oracle_mismatches": bad,
            "oracle_sample": "every (count/64)-th window, peel rounds, rounds, best round and best f",
            "generation_s": round(tgen, 1),
            "cta_threads": cta_threads, "one_cta_max_vertices": dupin.BATCH_CTA_MAX_N,
            "result_buffers": "peel rounds copied every call into page-locked host buffers allocated once"}


def bench_serving(dupin, args, requests=2000, rate=2000.0):
    """Poisson stream (mean 2,000 req/s) of FD peels over resident graphs: the window mix plus
    1% of requests on a few R-MAT scale-21 graphs (edge factor 10); p50/p99 from the server.
    Then the same requests submitted all at once (saturation graphs/s), and every distinct
    graph's result against the CPU oracle."""
    import oracle
    from paper_2504_09311_gb300 import synth

    pool = synth.transaction_windows(256, seed=7)
    big = [synth.rmat_weighted(21, 10, "fd", seed=s) for s in (1, 2)]
    gpool = [dupin.Graph.from_synth(g) for g in pool]
    gbig = [dupin.Graph.from_synth(g) for g in big]
    p = dupin.make_params("fd", 1, (1, 10))
    arrivals = synth.poisson_arrivals(requests, rate, seed=3)
    pick = synth.uniform_ints(requests, 1_000_000, seed=4)
    which = [("big", int(pick[j] // 100) % len(gbig)) if pick[j] % 100 == 0 else ("pool", int(pick[j]) % len(gpool))
             for j in range(requests)]
    graph_of = lambda w: gbig[w[1]] if w[0] == "big" else gpool[w[1]]

    def run(paced: bool):
        """Submit every request (at its Poisson arrival time when paced); the
        client polls its outstanding tickets between submissions, so each
        request's latency as the client sees it is recorded too."""
        srv = dupin.Server(memory_budget=16 << 30, max_slots=8)
        pend, outs, lat = {}, [None] * requests, [0.0] * requests

        def sweep():
            for t, (j, ts) in list(pend.items()):
                if srv.poll(t)[0]:
                    lat[j] = (time.perf_counter() - ts) * 1e3
                    outs[j] = (which[j], srv.wait(t))
                    del pend[t]

        t0 = time.perf_counter()
        for j in range(requests):
            while paced and arrivals[j] > time.perf_counter() - t0:
                sweep()
            pend[srv.submit(graph_of(which[j]), p, want_rounds=True)] = (j, time.perf_counter())
        while pend:
            sweep()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return outs, wall, st, lat

    def by_class(lat):
        out = {}
        for cls in ("pool", "big"):
            x = np.array([lat[j] for j in range(requests) if which[j][0] == cls])
            out["windows" if cls == "pool" else "rmat21"] = {
                "requests": int(x.size), "p50_ms": float(np.percentile(x, 50)), "p99_ms": float(np.percentile(x, 99))}
        return out

    outs, wall, st, lat = run(True)
    outs_sat, wall_sat, st_sat, lat_sat = run(False)
    # every result equals the graph's own peel alone, and each distinct graph's equals the oracle's
    ref, orc = {}, {}
    mismatch = omis = 0
    for w, o in outs + outs_sat:
        if w not in ref:
            ref[w] = dupin.peel(graph_of(w), "fd", 1, (1, 10), want_mask=False, want_trace=False)
            sg = big[w[1]] if w[0] == "big" else pool[w[1]]
            og = oracle.Graph.from_synth(sg, "fd")
            orc[w] = oracle.peel_batch(og, 1, (1, 10))
            og.close()
        r, q = ref[w], orc[w]
        mismatch += 0 if (np.array_equal(o.peel_round, r.peel_round) and o.best_f == r.best_f) else 1
        omis += 0 if (np.array_equal(o.peel_round, q.peel_round) and o.best_f == q.best_f and
                      o.best_round == q.best_round) else 1
    for g in gpool + gbig:
        g.free()
    return {"workload": f"{requests} requests, Poisson {rate:.0f}/s, 256 windows + 1% on 2 R-MAT-21 (ef 10) graphs",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "graphs_per_s": requests / wall,
            "client_latency_by_class": by_class(lat),
            "completed": st["completed"], "mismatches_vs_alone": mismatch, "oracle_mismatches": omis,
            "oracle_graphs_checked": len(orc),
            "saturation": {"graphs_per_s": requests / wall_sat, "p50_ms": st_sat["p50_ms"], "p99_ms": st_sat["p99_ms"],
                           "client_latency_by_class": by_class(lat_sat), "how": "the same requests submitted at once"}}


def cpu_baseline(g, metric, eps, k):
    import oracle

    t0 = time.perf_counter()
    og = oracle.Graph.from_synth(g, metric)
    t1 = time.perf_counter()
    oracle.peel_batch(og, k, eps)
    t2 = time.perf_counter()
    og.close()
    return {"value": g.m / (t2 - t1), "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"one of the step's peels ({metric.upper()}, eps={eps[0]}/{eps[1]}, k={k}) of the full graph, "
                      f"single-threaded C oracle; {t2 - t1:.2f} s peel + {t1 - t0:.2f} s adjacency build (not counted)",
            "seconds": t2 - t1}


TAIL_KERNEL_BEGIN = "template <bool NARROW>\n__device__ __forceinline__ void peel_tail_body("
TAIL_KERNEL_END = "// best_mask[u] = (peel_round[u] > best_round) for a best round known on the host"


def tail_kernel_source_hash() -> Optional[str]:
    """sha256 of k_peel_tail's definition and the two device headers it uses."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2504_09311_gb300", "csrc")
    try:
        peel = open(os.path.join(csrc, "peel.cu")).read()
        a, b = peel.index(TAIL_KERNEL_BEGIN), peel.index(TAIL_KERNEL_END)
        text = peel[a:b] + open(os.path.join(csrc, "peel_device.cuh")).read() + \
            open(os.path.join(csrc, "dupin_common.cuh")).read()
    except (OSError, ValueError):
        return None
    return hashlib.sha256(text.encode()).hexdigest()


def measured_traffic(kernel: str) -> Optional[float]:
    """DRAM bytes per launch that ncu measured for the kernel on this workload
    (profiles/dram_traffic.json), or None once its sources have changed."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if kernel != "k_peel_tail" or not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("source_sha256") != tail_kernel_source_hash():
        return None
    return float(d["bytes_per_launch"])


# Latencies measured on a GB300 (one thread, dependent chains): a global load
# that hits L2 and a 64-bit shared-memory atomic add with its result used.
L2_HIT_CYCLES = 311
SMEM_ATOMIC64_CYCLES = 130


def round_latency(tail_ms: float, tail_rounds: float, sm_mhz: float) -> Optional[dict]:
    """The one-CTA tail's time per round against the latency every round pays
    in sequence: the removed vertices' arcs are read from L2 and their
    neighbours' weights updated by shared atomics whose results decide the
    next round, so a round cannot take less than one L2 hit plus one
    dependent shared atomic."""
    if tail_rounds <= 0 or tail_ms <= 0 or sm_mhz <= 0:
        return None
    us = tail_ms * 1e3 / tail_rounds
    floor_us = (L2_HIT_CYCLES + SMEM_ATOMIC64_CYCLES) / sm_mhz
    return {"tail_rounds_per_peel": round(tail_rounds, 1), "us_per_round": round(us, 3),
            "floor_us": round(floor_us, 3), "frac": round(floor_us / us, 3),
            "floor": f"L2 hit {L2_HIT_CYCLES} + dependent 64-bit shared atomic {SMEM_ATOMIC64_CYCLES} cycles "
                     f"at {sm_mhz:.0f} MHz"}


# the cluster tail's result exchange: every CTA's asynchronous stores into
# every inbox and the wait on its own mbarrier (measured in the kernel with
# clock64 on R-MAT-24: 0.3 us at 2,070 MHz)
CLUSTER_EXCHANGE_CYCLES = 620


def cluster_round_latency(tail_ms: float, tail_rounds: float, sm_mhz: float) -> Optional[dict]:
    """The cluster tail's time per round against the latency every round pays
    in sequence: the removed vertices' arc groups are read from L2, their
    heads' weights updated by shared atomics whose results decide the next
    round's minimum, and the CTAs' results exchanged before the next round."""
    if tail_rounds <= 0 or tail_ms <= 0 or sm_mhz <= 0:
        return None
    us = tail_ms * 1e3 / tail_rounds
    floor_us = (L2_HIT_CYCLES + SMEM_ATOMIC64_CYCLES + CLUSTER_EXCHANGE_CYCLES) / sm_mhz
    return {"tail_rounds_per_step": round(tail_rounds, 1), "us_per_round": round(us, 3),
            "floor_us": round(floor_us, 3), "frac": round(floor_us / us, 3),
            "floor": f"L2 hit {L2_HIT_CYCLES} + dependent 64-bit shared atomic {SMEM_ATOMIC64_CYCLES} + result "
                     f"exchange {CLUSTER_EXCHANGE_CYCLES} cycles at {sm_mhz:.0f} MHz"}


def max_over_ranks(ms: float, dist) -> float:
    """The step time every rank reports is the slowest rank's (host tensors, so
    the gloo process group carries it)."""
    if not dist:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_parallel_baseline(g, metric, eps, k):
    """The multi-threaded CPU Algorithm 2 (the paper's own design) on all host
    cores, one peel of the full graph (its results equal the oracle's)."""
    import cpu_baseline

    cg = cpu_baseline.Graph(g, metric)
    threads = os.cpu_count() or 1
    cpu_baseline.peel(cg, k, eps, 0, threads)  # warm-up
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        cpu_baseline.peel(cg, k, eps, 0, threads)
    dt = (time.perf_counter() - t0) / reps
    return {"value": g.m / dt, "unit": "edges/s", "cores": threads, "kind": "parallel C, Algorithm 2 with "
            "parallel_for over live vertices and removed vertices' arcs (Sec. 4.1), exact integers",
            "sample": f"one peel (eps={eps[0]}/{eps[1]}, k={k}) of the full graph, mean of {reps}", "seconds": dt}


def run_reference(args, wl, rank, world):
    """The oracle as it stands, single-threaded, on this arm's workload: each
    step peels the step's (metric, eps) list once.  For the R-MAT-24 workloads
    a step peels the scale-22 graph of the same generator (a quarter of the
    vertices and edges), so that 20 + 5 steps end within minutes."""
    if rank != 0:
        return
    import oracle

    sample_graph = REFERENCE_SAMPLE.get(args.workload, wl["graph"])
    g = make_graph(sample_graph)
    ogs = {}
    for metric, _ in wl["peels"]:
        if metric not in ogs:
            ogs[metric] = oracle.Graph.from_synth(g, metric)

    def step():
        for metric, eps in wl["peels"]:
            oracle.peel_batch(ogs[metric], wl["k"], eps)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = g.m * len(wl["peels"]) / dt
    peels = ", ".join(f"{m.upper()} eps={e[0]}/{e[1]}" for m, e in wl["peels"])
    sample = (f"each step peels the {sample_graph} graph ({g.n} vertices, {g.m} edges) once per ({peels}), "
              f"k={wl['k']}" + ("; the same R-MAT generator at scale 22 stands in for scale 24" if
                                sample_graph != wl["graph"] else ""))
    line = {"impl": "reference", "metric": "edges peeled/s", "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": args.workload, "k_mult": wl["k"],
                       "peels": [f"{m}:{e[0]}/{e[1]}" for m, e in wl["peels"]], "sample": sample},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    for og in ogs.values():
        og.close()
    print(json.dumps(line), flush=True)


def kernel_of(phase: str, tail_ctas: int) -> str:
    return {"init": "k_init_vertex+k_init_arcs+k_init_reduce", "bulk": "k_peel_bulk",
            "build": "k_tail_prep+k_tail_scan+k_tail_arcs+k_tail_rowcnt+k_tail_grp",
            "tail": "k_peel_cluster" if tail_ctas > 1 else "k_peel_tail"}[phase]


def side_runs(dupin, g, dg, stream, wl, reps=3):
    """Beside the headline: the same graph at k_mult = 2, and the DW metric at
    k_mult = 1 on the same topology (its own weights): per-peel device time."""
    import torch

    out = {}

    def time_peel(graph, metric, k, eps):
        dupin.peel(graph, metric, k, eps, want_rounds=False, want_mask=False, want_trace=False, stream=stream)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o = dupin.peel(graph, metric, k, eps, flags=dupin.TIMING, want_rounds=False, want_mask=False,
                           want_trace=False, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = float(np.median(ms))
        return {"ms_per_peel": round(t, 3), "edges_per_s": g.m / (t / 1e3), "rounds": int(o.n_rounds),
                "bulk_rounds": int(o.n_bulk_rounds), "tail_ctas": int(o.tail_ctas),
                "phase_ms": [round(float(x), 3) for x in o.phase_ms]}

    for metric, eps in wl["peels"]:
        out[f"{metric}_k2"] = time_peel(dg, metric, 2, eps)
    gw = dw_copy(g)
    dw = dupin.Graph.from_synth(gw, stream=stream)
    out["dw_k1"] = time_peel(dw, "dw", 1, (1, 10))
    out["dw_k1"]["weights"] = "c uniform 1..100, a uniform 0..10 (Q32.32), same topology"
    dw.free()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dupin", choices=["dupin", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=list(WORKLOADS))
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-side", action="store_true")
    ap.add_argument("--windows", type=int, default=4096)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.k is not None:
        wl["k"] = args.k
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch

    from paper_2504_09311_gb300 import dupin

    torch.cuda.set_device(local)
    dupin.lib()  # the CUDA library must be present: no fallback
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    g = make_graph(wl["graph"])
    gen_s = time.perf_counter() - t0
    peels, k = wl["peels"], wl["k"]
    dg = dupin.Graph.from_synth(g)
    params = [dupin.make_params(metric, k, e, flags=dupin.TIMING) for metric, e in peels]
    # one output pair per peel: the step's peels run together (grid-wide
    # stages in turn, tails side by side) through dupin_peel_batch
    prs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in peels]
    mks = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for _ in peels]
    # a peel whose (graph, metric) came earlier in the step copies that peel's initial weights
    follower = [any(peels[q][0] == peels[j][0] for q in range(j)) for j in range(len(peels))]

    def step(record=None):
        R = dupin.peel_batch_device([dg] * len(params), params, prs, mks, stream=stream)
        if record is not None:
            for j in range(len(params)):
                record.append((j, R[j].n_rounds, R[j].n_bulk_rounds, list(R[j].phase_ms), R[j].tail_ctas))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    rec = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(rec)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    edges_per_step = g.m * len(params)
    value = world * edges_per_step / (ms / 1e3)
    sm_mhz = clocks.summary().get("sm_mhz") or 2070.0

    # per peel: phase times (mean over the timed steps) and algorithmic bytes
    # from the peel's own output
    names = ["init", "bulk", "build", "tail"]
    per_peel = []
    for j, (metric, e) in enumerate(peels):
        ph = np.mean(np.array([r[3] for r in rec if r[0] == j], np.float64), axis=0)
        nb = [r[2] for r in rec if r[0] == j][0]
        tc = [r[4] for r in rec if r[0] == j][0]
        out = dupin.peel(dg, metric, k, e, flags=dupin.TIMING)
        b = algorithmic_bytes(g, out.peel_round, np.asarray(out.trace_size), nb, metric)
        if follower[j]:  # its initial weights are a copy (w, round, live list: 24 B per vertex)
            b["init"] = 24 * g.n
        per_peel.append({"metric": metric, "eps": f"{e[0]}/{e[1]}", "rounds": int(out.n_rounds), "bulk_rounds": int(nb),
                         "tail_ctas": int(tc), "init_copied": bool(follower[j]),
                         "ms": {names[q]: round(float(ph[q]), 4) for q in range(4)},
                         "algorithmic_bytes": {kk: int(b[kk]) for kk in names}})
    # the dominant kernel: the largest total device time over the step's peels
    # (a follower's copied initial weights are another kernel and left out)
    tot = {}
    for p in per_peel:
        for q in names:
            if q == "init" and p["init_copied"]:
                continue
            key = kernel_of(q, p["tail_ctas"])
            t_, b_ = tot.get(key, (0.0, 0))
            tot[key] = (t_ + p["ms"][q], b_ + p["algorithmic_bytes"][q])
    kernel = max(tot, key=lambda kk: tot[kk][0])
    t_dom, b_dom = tot[kernel]
    launches = sum(1 for p in per_peel for q in names if kernel_of(q, p["tail_ctas"]) == kernel and
                   not (q == "init" and p["init_copied"]))
    peak, peak_kind = measured_peaks()
    achieved = b_dom / (t_dom / 1e3) / 1e9 if t_dom > 0 else 0.0
    traffic = measured_traffic(kernel) if args.workload == "fd_2Mx1M_40M" else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kernel,
                "launches_per_step": launches, "ms_per_step": round(t_dom, 4),
                "algorithmic_bytes_per_step": int(b_dom),
                "peak_source": f"{peak_kind} hbm_gbs", "per_peel": per_peel}
    # the whole step against the same roofline: every phase's algorithmic bytes over the step time
    step_bytes = sum(p["algorithmic_bytes"][q] for p in per_peel for q in names)
    roofline["step"] = {"algorithmic_bytes": int(step_bytes), "achieved": round(step_bytes / (ms / 1e3) / 1e9, 2),
                        "frac": round(step_bytes / (ms / 1e3) / 1e9 / peak, 4)}
    one_cta = [(p["ms"]["tail"], p["rounds"] - p["bulk_rounds"]) for p in per_peel if p["tail_ctas"] == 1]
    if one_cta:
        lat = round_latency(sum(t for t, _ in one_cta), sum(r for _, r in one_cta), sm_mhz)
        if lat is not None:
            roofline["round_latency"] = lat
    cl = [(p["ms"]["tail"], p["rounds"] - p["bulk_rounds"]) for p in per_peel if p["tail_ctas"] > 1]
    if cl and sum(r for _, r in cl) > 0:
        roofline["cluster_tail_us_per_round"] = round(sum(t for t, _ in cl) * 1e3 / sum(r for _, r in cl), 3)
        lat = cluster_round_latency(sum(t for t, _ in cl), sum(r for _, r in cl), sm_mhz)
        if lat is not None:
            roofline["cluster_round_latency"] = lat

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        csr = g.bipartite_csr() if g.bipartite else g.symmetric_csr()
        pinned = []
        for a in csr:
            if a is None:
                pinned.append(None)
                continue
            t = torch.empty(a.shape, dtype={np.dtype(np.int64): torch.int64, np.dtype(np.int32): torch.int32}[a.dtype],
                            pin_memory=True)
            t.numpy()[:] = a
            pinned.append(t.numpy())
        del csr
        h2d = sum(a.nbytes for a in pinned if a is not None)
        d2h = 0
        # the results land in page-locked host buffers (allocated once)
        res_bufs = [dupin.result_buffers(g.n, True, True, True, pinned=True) for _ in peels]

        def e2e_step():
            nonlocal d2h
            if g.bipartite:
                gg = dupin.Graph.load_bipartite(g.n_left, g.n_right, *pinned, g.a, stream=stream)
            else:
                gg = dupin.Graph.load_symmetric(g.n, *pinned, g.a, stream=stream)
            d2h = 0
            ps = [dupin.make_params(metric, k, e) for metric, e in peels]
            for o in dupin.peel_batch([gg] * len(ps), ps, want_rounds=True, want_trace=True, want_mask=True,
                                      stream=stream, buffers=res_bufs):
                d2h += o.peel_round.nbytes + o.best_mask.nbytes + 32 * (o.n_rounds + 1)
            gg.free()

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 3))
        for _ in range(ksteps):
            e2e_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / ksteps
        e2e = {"value": world * edges_per_step / dt, "unit": "edges/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3,
               "includes": "graph load from pinned host memory + validation + one batched call of the step's peels "
                           "(peel workspaces from the cache of freed graphs' workspaces) + result copies + free"}
        del pinned

    side = None if args.no_side or not args.workload.startswith("rmat") else side_runs(dupin, g, dg, stream, wl)
    batched = None if args.no_batch else bench_batched(dupin, stream, args)
    serving = None if args.no_serve else bench_serving(dupin, args)

    cpu = cpu_par = None
    if rank == 0 and not args.no_cpu_baseline:
        # the step's longest peel (its first weighted one), else its middle one
        metric_b, eps_b = next((pe for pe in peels if pe[0] != "dg"), peels[len(peels) // 2])
        if len(peels) >= 3:
            metric_b, eps_b = peels[1]
        cpu = cpu_baseline(g, metric_b, eps_b, k)
        cpu_par = cpu_parallel_baseline(g, metric_b, eps_b, k)

    # kernels per peel: control reset, initial weights (DG: one kernel; FD/DW: three), the
    # set-up's finish, the grid-wide rounds, the tail build (prep, two scans, two arc passes,
    # row counts and owner groups), the one-CTA tail and the cluster tail (one of the two
    # returns at once), and the final mask
    launches_per_peel = {"dg": 14, "fd": 16, "dw": 16}
    line = {
        "metric": "edges peeled/s", "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "graph": wl["graph"], "k_mult": k,
                   "peels": [f"{m}:{e[0]}/{e[1]}" for m, e in peels], "n": g.n, "m": g.m, "arcs": 2 * g.m,
                   "rounds": [p["rounds"] for p in per_peel], "bulk_rounds": [p["bulk_rounds"] for p in per_peel],
                   "tail_ctas": [p["tail_ctas"] for p in per_peel], "generation_s": round(gen_s, 1),
                   "l2": "inputs larger than L2 (graph arrays several GB vs 129 MB L2)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_parallel_baseline": cpu_par,
        "e2e": e2e,
        # (+ one note per pair of the call's large peels: an earlier peel's tail kind for a later one)
        "gpu_launches": (sum(launches_per_peel[m] for m, _ in peels) + len(peels) * (len(peels) - 1) // 2) * args.steps,
        "clocks": clocks.summary(),
        "side": side,
        "batched": batched,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dg.free()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

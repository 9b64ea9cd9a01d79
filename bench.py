#!/usr/bin/env python
"""Benchmark of the SKIM hot path on one GB300 (or N replicas).

One step = one pass over the whole hot path on R-MAT scale 20 (edge factor
16), weighted cascade, l = k = 64:
  live-edge instances -> rank order of the n*l pairs -> all combined sketches
  (Algorithm 2) -> 50 SKIM seeds with residual updates (Algorithm 1) -> a
  batch of influence-oracle queries (Eq. unionest).

value: edge-instance traversals per second, the traversal count being the
oracle's sequential count for the step (stored next to the tests), so work
the GPU does twice is not credited.  Also reported: seconds to 50 seeds,
sketch-build seconds, live-edge and coin rates, oracle QPS and single-query
p50/p99 latency, the roofline of the dominant kernel (with the random-gather
ceiling measured in the same run), the same step with coins hashed in the
searches, the influence oracle served over R-MAT scale 22 sketches (plain
one-query form against continuous batching), 256 graphs built in one batch
against one at a time, and R-MAT scale 24 (uniform p = 0.01): all sketches
and 200 seeds.

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own replica (independent problems, no
collective on the data path: weak scaling).
"""
from __future__ import annotations

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
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SKIM edge-instance traversals/s & s-to-50-seeds; oracle QPS, p50/p99 latency"
UNIT = "edge-instance traversals/s"
GOLDEN = os.path.join(ROOT, "tests", "golden")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# integer operations per live-edge coin on a 32-bit datapath, from the
# SplitMix64 definition: 3 xor-shifts x 4 + 2 64-bit multiplies x 3 = 18 per
# output function; + 5 for the stream offset (64-bit multiply-add), + 2 for
# the 64-bit compare, + 2 to set the lane bit = 27.
OPS_PER_COIN = 27
INT32_OPS_PER_SM_CLK = 64
SMS = 152


def workload_desc(w: synth.Workload, g) -> str:
    model = {0: f"uniform p={w.p}", 1: "weighted cascade", 2: "trivalency"}[w.prob_model]
    return (f"{w.name}: R-MAT scale {w.n_or_scale} edge factor {w.m_or_ef} ({g.m} edges after dedup), "
            f"{model}, l={w.l}, k={w.k}; live-edge instances + rank order + all sketches + {w.seeds} SKIM seeds "
            "+ queries")


def step_traversals(gold: dict) -> int:
    """Oracle's sequential edge-instance traversals for one step."""
    t = gold["sketches"]["counters"]["rev_edge_scans"]
    t += gold["skim"]["counters"]["rev_edge_scans"] + gold["skim"]["counters"]["fwd_edge_scans"]
    return int(t)


def query_sets(w, n, count):
    ks = w.keys()
    sizes = synth.query_sizes(count, ks.query ^ 0x1234)
    return [synth.uniform_seed_set(n, int(s), ks.query ^ 0x1234, q) for q, s in enumerate(sizes)]


class Clocks:
    """nvidia-smi samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch of a kernel group on a workload, from the
    committed ncu summaries (profiles/traffic.json), if the kernels' source
    has not changed since they were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    for rec in json.load(open(path)).get("records", []):
        if rec.get("kernel") != kernel or rec.get("workload") != workload:
            continue
        src = os.path.join(ROOT, "paper_1408_6282_gb300", "csrc", rec["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
            return None
        return rec
    return None


def kernel_roofline(kname, kt, gold, m, l, steps, sm_max, hbm_peak, total_ms, workload, gather=None):
    """Roofline of one kernel group of the step, from its CUDA-event time and
    the algorithmic work of one step (the oracle's counts, so redundant GPU
    work is not credited).

    rev_search  (memory): every candidate visit -- a batch's source lane or a
                live in-edge walked -- reads a 4 B node or pair id, the 8 B
                bounds of the live row of (v, i) (which carry Algorithm 2's
                pruning flag) and reads and writes its 8 B visited word (16 B);
                every expansion also writes its 12 B visit record.  Sources are
                taken inside the search kernel, so their lanes count here.
    fwd_search  (memory): 16 B per forward expansion (the two row bounds of
                (v, i)) + 20 B per live out-edge (4 B neighbour id, covered word
                read and write) + 8 B per index entry erased (node id, size).
    instances   (integer ALU): 2 m l coins (both CSR orders) x 27 int32 ops.
    """
    ms, launches = kt[kname]
    sec = ms / 1000.0 / steps
    sk, sm = gold["sketches"]["counters"], gold["skim"]["counters"]
    common = {"kernel": kname, "avg_launch_ms": ms / max(1, launches), "launches_per_step": launches / steps,
              "share_of_kernel_time": ms / total_ms if total_ms else None}
    if kname == "instances":
        ops = 2 * m * l * OPS_PER_COIN
        peak = SMS * INT32_OPS_PER_SM_CLK * sm_max * 1e6 / 1e12
        achieved = ops / sec / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (int32)", "frac": achieved / peak,
                "traffic": None, "peak_note": "derived: 152 SMs x 64 int32 ops/clk x max SM clock",
                "algorithmic_units": f"2 x {m} edges x {l} instances coins x {OPS_PER_COIN} ops", **common}
    extra = {}
    if kname == "rev_search":
        lanes = sk["ranks_consumed"] + sm["ranks_consumed"]
        E = sk["rev_expansions"] + sm["rev_expansions"]
        L = sk.get("rev_live_edges", 0) + sm.get("rev_live_edges", 0)
        cand = lanes + L
        byts = 28 * cand + 12 * E
        units = (f"{cand} candidate visits ({lanes} source lanes + {L} live in-edges) x 28 B + {E} expansions "
                 "x 12 B per step")
        key = "rev_search"
        if gather:
            # each candidate costs at least two independent random accesses
            # (its row entry and its visited slot) and each live in-edge's id
            # is a third: the count a random-access ceiling applies to
            acc = 2 * cand + L
            extra["random_access"] = {"achieved": acc / sec / 1e9, "peak": gather / 1e9, "unit": "G accesses/s",
                                      "frac": acc / sec / gather,
                                      "basis": "2 random accesses per candidate visit + 1 per live in-edge; peak = "
                                               "random 8-byte gathers over a 4 GiB array (torch index_select) "
                                               "timed in this run"}
    else:
        E, L, X = sm["fwd_expansions"], sm.get("fwd_live_edges", 0), sm["index_erased"]
        byts = 16 * E + 20 * L + 8 * X
        units = f"{E} forward expansions x 16 B + {L} live out-edges x 20 B + {X} index entries x 8 B per step"
        key = "fwd_search"
    achieved = byts / sec / 1e9
    trb = traffic_record(key, workload)
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": trb["dram_bytes_per_launch"] if trb else None,
            "traffic_note": (f"DRAM bytes per launch ({trb['launch']}), from profiles/traffic.json") if trb
            else "no capture of the current source",
            "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "algorithmic_units": units, **common, **extra}


def gather_peak(device: str = "cuda") -> float:
    """Random 8-byte loads per second over a 4 GiB array (the ceiling of a
    kernel whose every access is an independent random one)."""
    import torch
    n = 1 << 29
    a = torch.arange(n, dtype=torch.int64, device=device)
    idx = torch.randint(0, n, (1 << 26,), device=device, dtype=torch.int64)
    out = torch.empty(1 << 26, dtype=torch.int64, device=device)
    for _ in range(3):
        torch.index_select(a, 0, idx, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        torch.index_select(a, 0, idx, out=out)
    e1.record()
    torch.cuda.synchronize()
    rate = 5 * idx.shape[0] / (e0.elapsed_time(e1) / 1000.0)
    del a, idx, out
    torch.cuda.empty_cache()
    return rate


def max_over_ranks(elapsed: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the job's time); identity on one process."""
    if dist is None:
        return elapsed
    import torch
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, units_per_step: float, elapsed: float) -> float:
    """Whole-job throughput: every rank processed `units_per_step` per step."""
    return world * steps * units_per_step / elapsed


def cpu_baseline(w, g, instances: int):
    """The oracle's Algorithm 2 as it stands, on `instances` of the l instances
    of the same graph (single thread, host cores)."""
    import oracle
    ks = w.keys()
    pb = oracle.Problem(g.n, g.src, g.dst, instances, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob)
    t0 = time.perf_counter()
    _, _, cnt = oracle.build_sketches(pb)
    dt = time.perf_counter() - t0
    return cnt["rev_edge_scans"] / dt, dt, cnt["rev_edge_scans"]


def config5_object(pkg, stream, local):
    """Large plain SKIM (R-MAT scale 24, uniform p = 0.01, l = k = 64): every
    sketch (Algorithm 2) and 200 seeds (Algorithm 1) on the device-resident
    graph, each timed with CUDA events, plus the reverse search's roofline."""
    import torch
    w = synth.WORKLOADS["rmat24_p01"]
    gold = json.load(open(os.path.join(GOLDEN, f"{w.name}.json")))
    a = time.perf_counter()
    g = w.graph(device=f"cuda:{local}")
    gen_s = time.perf_counter() - a
    assert g.digest() == gold["graph_sha256"], "generated graph differs from the one the oracle counted"
    ks = w.keys()
    src_d = torch.from_numpy(g.src.view(np.int32)).cuda()
    dst_d = torch.from_numpy(g.dst.view(np.int32)).cuda()
    m = g.m
    del g
    torch.cuda.synchronize()
    a = time.perf_counter()
    sk = pkg.Skim(1 << w.n_or_scale, src_d, dst_d, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob,
                  stream=stream.cuda_stream)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - a
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    sk.set_timing(True)
    sk.kernel_times(reset=True)
    ev[0].record(stream)
    sk.build_sketches()
    ev[1].record(stream)
    seeds, cov = sk.greedy(w.seeds)
    ev[2].record(stream)
    torch.cuda.synchronize()
    kt = sk.kernel_times(reset=True)
    build_s, greedy_s = ev[0].elapsed_time(ev[1]) / 1000.0, ev[1].elapsed_time(ev[2]) / 1000.0
    ok = seeds.tolist() == gold["skim"]["seeds"] and [int(c) for c in cov] == gold["skim"]["cov"]
    live_pairs, _ = sk.instance_stats()
    out = {"workload": f"rmat24_p01: R-MAT scale 24 edge factor 16 ({m} edges after dedup), uniform p=0.01, "
                       f"l={w.l}, k={w.k}, {w.seeds} seeds",
           "graph_generation_s": gen_s, "context_s": create_s, "sketch_build_s": build_s,
           "s_to_200_seeds": greedy_s, "build_plus_200_seeds_s": build_s + greedy_s, "seeds_match_oracle": ok,
           "live_pairs": live_pairs, "kernel_ms": {k2: round(v[0], 3) for k2, v in kt.items()}}
    sm = gold["skim"]["counters"]
    skim_t = sm["rev_edge_scans"] + sm["fwd_edge_scans"]
    out["skim_traversals_per_s"] = skim_t / greedy_s
    if "sketches" in gold:
        t_alg = gold["sketches"]["counters"]["rev_edge_scans"] + skim_t
        out["traversals"] = t_alg
        out["edge_instance_traversals_per_s"] = t_alg / (build_s + greedy_s)
        out["oracle_seconds"] = gold["sketches"]["oracle_seconds"] + gold["skim"]["oracle_seconds"]
        peak = json.load(open(PEAKS)).get("hbm_gbs", 6800.0) if os.path.exists(PEAKS) else 6800.0
        total_ms = sum(v[0] for v in kt.values())
        out["roofline"] = kernel_roofline("rev_search", kt, gold, m, w.l, 1, 2070.0, peak, total_ms, w.name)
    else:
        out["oracle_seconds"] = gold["skim"]["oracle_seconds"]
    sk.close()
    del src_d, dst_d
    torch.cuda.empty_cache()
    pkg.skim_release_memory()
    return out


def serving_config4_object(pkg, stream, local, args):
    """The influence oracle served on R-MAT scale 22 (weighted cascade, l = k =
    64) sketches resident on the device: the plain one-query form (one C-ABI
    call per query, host seeds and result), one batched call, and Poisson
    streams at swept rates through the continuous-batching server."""
    import torch
    w = synth.WORKLOADS["rmat22_wc"]
    gold = json.load(open(os.path.join(GOLDEN, f"{w.name}.json")))
    g = w.graph(device=f"cuda:{local}")
    assert g.digest() == gold["graph_sha256"]
    ks = w.keys()
    src_d = torch.from_numpy(g.src.view(np.int32)).cuda()
    dst_d = torch.from_numpy(g.dst.view(np.int32)).cuda()
    out = {"workload": f"rmat22_wc: R-MAT scale 22 edge factor 16 ({g.m} edges after dedup), weighted cascade, "
                       f"l={w.l}, k={w.k}; |S| = floor(10^(3U)) in 1..1000, seeds uniform"}
    with pkg.Skim(g.n, src_d, dst_d, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob,
                  stream=stream.cuda_stream) as sk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sk.build_sketches()
        e1.record(stream)
        torch.cuda.synchronize()
        out["sketch_build_s"] = e0.elapsed_time(e1) / 1000.0
        est = sk.query_batch([q["seeds"] for q in gold["queries"]])
        out["estimates_match_oracle"] = bool(all(abs(float(e) - q["estimate"]) <= 1e-12 * abs(q["estimate"])
                                                 for q, e in zip(gold["queries"], est)))
        qs = query_sets(w, g.n, args.queries)
        # plain one-query form: one call per query, host seeds to host estimate
        lat = []
        for q in qs[: args.latency_queries]:
            a = time.perf_counter()
            sk.query(q)
            lat.append((time.perf_counter() - a) * 1000.0)
        lat.sort()
        out["plain"] = {"qps": 1000.0 / (sum(lat) / len(lat)), "p50_ms": lat[len(lat) // 2],
                        "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "queries": len(lat)}
        a = time.perf_counter()
        sk.query_batch(qs)
        out["one_batch_call_qps"] = len(qs) / (time.perf_counter() - a)
        serving = []
        with sk.server(max_inflight=4096, scratch_slots=1 << 24, streams=4) as srv:
            for rate in args.serve_rates:
                arr = synth.poisson_arrivals(len(qs), rate, ks.query + int(rate))
                g0, q0 = srv.stats()
                t_a = time.perf_counter()
                slat, sest = srv.replay(arr, qs)
                wall = time.perf_counter() - t_a
                g1, q1 = srv.stats()
                slat = np.sort(slat) * 1000.0
                serving.append({"offered_qps": rate, "qps": len(qs) / wall, "p50_ms": float(slat[len(slat) // 2]),
                                "p99_ms": float(slat[min(len(slat) - 1, int(0.99 * len(slat)))]),
                                "mean_group": (q1 - q0) / max(1, g1 - g0)})
        out["served"] = serving
    del src_d, dst_d
    torch.cuda.empty_cache()
    return out


def batched_object(pkg, stream, local, count):
    """The batched form against one graph at a time on the same GPU, both
    timed like for like: builds only (contexts created before the clock
    starts), and everything (create, build, destroy)."""
    import torch
    specs = synth.batched_graph_specs(count)
    gl = [synth.rmat(sc, ef, key, device=f"cuda:{local}") for sc, ef, key in specs]
    gk = [synth.Keys.from_seed(key) for _, _, key in specs]
    bl, bk = 64, 32
    build_one = 0.0
    torch.cuda.synchronize()
    t_a = time.perf_counter()
    for gr, kk in zip(gl, gk):
        with pkg.Skim(gr.n, gr.src, gr.dst, bl, bk, 2, 0.0, kk.coin, kk.rank, kk.prob,
                      stream=stream.cuda_stream) as one:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one.build_sketches()
            e1.record(stream)
            e1.synchronize()
            build_one += e0.elapsed_time(e1) / 1000.0
    torch.cuda.synchronize()
    total_one = time.perf_counter() - t_a
    t_a = time.perf_counter()
    many = pkg.Skim.batch([(gr.n, gr.src, gr.dst) for gr in gl], bl, bk, [2] * len(gl), [0.0] * len(gl),
                          [kk.coin for kk in gk], [kk.rank for kk in gk], [kk.prob for kk in gk],
                          stream=stream.cuda_stream)
    torch.cuda.synchronize()
    create_many = time.perf_counter() - t_a
    with many:
        grid = [(lanes, ring, 4) for lanes in (1 << 20, 1 << 21, 1 << 22) for ring in (0.0, 8.0)]
        bi, secs = many.autotune_settings(grid)
        best = many.tuning()
        many.build_sketches()  # warm, with the tuned settings
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        many.build_sketches()
        e1.record(stream)
        torch.cuda.synchronize()
        build_many = e0.elapsed_time(e1) / 1000.0
        bstats = many.stats()
        t_a = time.perf_counter()
    t_close = time.perf_counter() - t_a
    return {"graphs": len(gl), "nodes": int(sum(gr.n for gr in gl)), "edges": int(sum(gr.m for gr in gl)),
            "l": bl, "k": bk, "prob_model": "trivalency",
            "builds_only": {"batched_s": build_many, "one_graph_at_a_time_s": build_one,
                            "speedup": build_one / build_many},
            "create_build_destroy": {"batched_s": create_many + build_many + t_close,
                                     "one_graph_at_a_time_s": total_one,
                                     "speedup": total_one / (create_many + build_many + t_close)},
            "autotuned": best, "autotune_grid": grid, "autotune_s": [float(x) for x in secs],
            "batches": bstats["batches"], "retries": bstats["retries"]}


def coins_on_the_fly_object(sk, w, gold, stream):
    """The same step's sketch build and SKIM seeds with no instance stored:
    every search hashes the coins of the edges its lanes reach (Section 2's
    coins evaluated on the fly), against the materialised live rows."""
    import torch
    sk.set_live_rows(False)
    try:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        sk.build_sketches()
        ev[1].record(stream)
        st = sk.stats()
        seeds, cov = sk.greedy(w.seeds)
        ev[2].record(stream)
        torch.cuda.synchronize()
        st2 = sk.stats()
        b, gr = ev[0].elapsed_time(ev[1]) / 1000.0, ev[1].elapsed_time(ev[2]) / 1000.0
        ok = seeds.tolist() == gold["skim"]["seeds"]
        return {"sketch_build_s": b, "s_to_50_seeds": gr, "seeds_match_oracle": ok,
                "build_coins": st["rev_coins"], "build_coins_per_s": st["rev_coins"] / b,
                "skim_coins": st2["rev_coins"] + st2["fwd_coins"]}
    finally:
        sk.set_live_rows(True)



def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on a bounded sample of the workload."""
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    g = w.graph()
    vals = []
    for s in range(args.warmup + args.steps):
        v, dt, trav = cpu_baseline(w, g, 1)
        if s >= args.warmup:
            vals.append((v, dt))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(dt for _, dt in vals) * 1000
    sample = (f"oracle Algorithm 2 on 1 of the {w.l} instances of {w.name} (k={w.k}), "
              "single thread; rate = oracle edge-instance traversals / wall time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_desc(w, g), "parallelism": "none (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="rmat20_wc")
    ap.add_argument("--queries", type=int, default=1000)
    ap.add_argument("--latency-queries", type=int, default=300)
    ap.add_argument("--cpu-instances", type=int, default=2)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[50000.0, 200000.0, 500000.0, 1000000.0])
    ap.add_argument("--batched-graphs", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--neighborhood-queries", type=int, default=300)
    ap.add_argument("--no-rank-modes", action="store_true")
    ap.add_argument("--no-config5", dest="config5", action="store_false")
    ap.add_argument("--no-on-the-fly", dest="on_the_fly", action="store_false")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_1408_6282_gb300 as pkg
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = synth.WORKLOADS[args.workload]
    gold = json.load(open(os.path.join(GOLDEN, f"{w.name}.json")))
    ks = w.keys()
    g = w.graph(device=f"cuda:{local}")
    assert g.digest() == gold["graph_sha256"], "generated graph differs from the one the oracle counted"
    t_alg = step_traversals(gold)
    src_d = torch.from_numpy(g.src.view(np.int32)).cuda()
    dst_d = torch.from_numpy(g.dst.view(np.int32)).cuda()
    src_h = torch.from_numpy(g.src.view(np.int32)).pin_memory()
    dst_h = torch.from_numpy(g.dst.view(np.int32)).pin_memory()
    qs = query_sets(w, g.n, args.queries)
    q_off = np.zeros(len(qs) + 1, np.uint64)
    q_off[1:] = np.cumsum([len(q) for q in qs])
    q_flat_h = torch.from_numpy(np.concatenate(qs).view(np.int32)).pin_memory()
    q_flat_d = q_flat_h.cuda()
    q_out_d = torch.zeros(len(qs), dtype=torch.float64, device="cuda")
    q_out_h = torch.zeros(len(qs), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    sk = pkg.Skim(g.n, src_d, dst_d, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob,
                  stream=stream.cuda_stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    part = {"instances": [], "ranks": [], "build": [], "greedy": [], "query": []}

    def step(record):
        e = [ev() for _ in range(6)]
        e[0].record(stream)
        sk.instances()
        e[1].record(stream)
        sk.rank_order()
        e[2].record(stream)
        sk.build_sketches()
        e[3].record(stream)
        seeds, cov = sk.greedy(w.seeds)
        e[4].record(stream)
        pkg.skim_oracle_query_batch(sk.ctx, q_off, len(qs), q_flat_d, q_out_d, 1)
        e[5].record(stream)
        if record:
            stream.synchronize()
            for key, a, b in (("instances", 0, 1), ("ranks", 1, 2), ("build", 2, 3), ("greedy", 3, 4),
                              ("query", 4, 5)):
                part[key].append(e[a].elapsed_time(e[b]) / 1000.0)
        return seeds, cov

    for i in range(args.warmup):
        seeds, cov = step(False)
        if i == 0:  # the timed path is the verified one
            assert seeds.tolist() == gold["skim"]["seeds"] and [int(c) for c in cov] == gold["skim"]["cov"]
    torch.cuda.synchronize()
    sk.set_timing(True)
    sk.kernel_times(reset=True)
    clocks = Clocks(local)
    clocks.start()
    launches0 = pkg.skim_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = ev(), ev()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = pkg.skim_kernel_launches() - launches0
    clk = clocks.stop()
    kt = sk.kernel_times(reset=True)
    sk.set_timing(False)
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1000.0, dist, device="cuda")
    value = job_value(world, args.steps, t_alg, elapsed)

    # single-query latency: submit (host seeds) to result (host estimate)
    lat = []
    for q in qs[: args.latency_queries]:
        a = time.perf_counter()
        sk.query(q)
        lat.append((time.perf_counter() - a) * 1000.0)
    lat.sort()

    # adaptive error estimation (Section 4.3.2) for the step's seed set: the
    # same SKIM run with each selection's threshold rank and k' recorded
    # (untimed), then the confidence bound on the summed discrepancy
    sk.greedy_reset()
    a = time.perf_counter()
    sseeds, scov, stau, skp = sk.greedy_stops(w.seeds)
    t_stops = time.perf_counter() - a
    assert sseeds.tolist() == gold["skim"]["seeds"]
    if "tau" in gold["skim"]:
        assert [str(int(t)) for t in stau] == gold["skim"]["tau"]
        assert [int(x) for x in skp] == gold["skim"]["kprime"]
    tot = float(scov.sum())
    conf = [0.5, 0.9, 0.99]
    a = time.perf_counter()
    bnd, _ = pkg.discrepancy_bound(scov, stau, skp, tot / 1024, 4096, conf)
    adaptive = {"seed_set_pairs": int(tot), "confidence": conf,
                "discrepancy_bound_pairs": [float(b) for b in bnd],
                "relative_to_seed_set": [float(b) / tot for b in bnd],
                "exact_selections": int((skp < 0).sum()), "greedy_with_records_s": t_stops,
                "bound_host_s": time.perf_counter() - a}

    # the second query distribution of Section 6.2: neighbourhood seed sets
    # (degree-proportional root, smallest ball with |S| nodes), one device batch
    nb = synth.Neighborhoods(g.n, g.src, g.dst)
    nsizes = synth.query_sizes(args.neighborhood_queries, ks.query ^ 0x4E42)
    nqs = [nb.draw(int(z), ks.query ^ 0x4E42, q)[0] for q, z in enumerate(nsizes)]
    n_off = np.zeros(len(nqs) + 1, np.uint64)
    n_off[1:] = np.cumsum([len(q) for q in nqs])
    n_flat_d = torch.from_numpy(np.concatenate(nqs).view(np.int32)).cuda()
    n_out_d = torch.zeros(len(nqs), dtype=torch.float64, device="cuda")
    nt = []
    for i in range(4):
        e0, e1 = ev(), ev()
        e0.record(stream)
        pkg.skim_oracle_query_batch(sk.ctx, n_off, len(nqs), n_flat_d, n_out_d, 1)
        e1.record(stream)
        stream.synchronize()
        if i:
            nt.append(e0.elapsed_time(e1) / 1000.0)
    neighborhood = {"queries": len(nqs), "seeds": int(n_off[-1]), "qps": len(nqs) / statistics.median(nt)}

    # the other rank readings of the same workload (untimed, once each):
    # structured permutation ranks (Section 3.1) with SKIM, and IC-model
    # sketches (Section 3.2, l -> infinity, k*n positions, unpruned searches)
    rank_modes = {}
    if not args.no_rank_modes:
        for name, mode, lm in (("permutation", pkg.RANKS_PERMUTATION, w.l), ("ic_model", pkg.RANKS_IC_MODEL, 1)):
            with pkg.Skim(g.n, src_d, dst_d, lm, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob,
                          stream=stream.cuda_stream, rank_mode=mode) as s3:
                torch.cuda.synchronize()
                a = time.perf_counter()
                s3.build_sketches()
                torch.cuda.synchronize()
                tb = time.perf_counter() - a
                st = s3.stats()
                rec = {"l": lm, "k": w.k, "build_s": tb, "positions": st["ranks"], "coins": st["rev_coins"],
                       "coins_per_s": st["rev_coins"] / tb}
                if mode == pkg.RANKS_PERMUTATION:
                    a = time.perf_counter()
                    s3.greedy(w.seeds)
                    torch.cuda.synchronize()
                    rec["s_to_50_seeds"] = time.perf_counter() - a
                rank_modes[name] = rec

    # the same step with no instance stored (coins hashed in the searches)
    on_the_fly = coins_on_the_fly_object(sk, w, gold, stream) if args.on_the_fly else None

    # serving (config 4): the influence oracle over R-MAT 22 sketches, plain
    # one-query form vs continuous batching
    serving = serving_config4_object(pkg, stream, local, args) if args.serve_rates else None

    # batched form: many independent graphs in one context and one pass,
    # against one graph at a time on the same GPU
    batched = batched_object(pkg, stream, local, args.batched_graphs) if args.batched_graphs else None

    # end to end through the C ABI with host buffers
    e2e_times = []
    h2d = 8 * g.m + 4 * int(q_off[-1]) + 8 * (len(qs) + 1)
    d2h = 12 * w.seeds + 8 * len(qs)
    for s in range(args.steps + 1):
        torch.cuda.synchronize()
        a = time.perf_counter()
        with pkg.Skim(g.n, src_h.numpy().view(np.uint32), dst_h.numpy().view(np.uint32), w.l, w.k,
                      w.prob_model, w.p, ks.coin, ks.rank, ks.prob, stream=stream.cuda_stream) as s2:
            s2.build_sketches()
            s2.greedy(w.seeds)
            pkg.skim_oracle_query_batch(s2.ctx, q_off, len(qs), q_flat_h.numpy().view(np.uint32),
                                        q_out_h.numpy(), 0)
        torch.cuda.synchronize()
        if s > 0:
            e2e_times.append(time.perf_counter() - a)
    e2e_t = max_over_ranks(statistics.median(e2e_times), dist, device="cuda")
    e2e_value = job_value(world, 1, t_alg, e2e_t)

    sk.close()
    # large plain SKIM (config 5) on the same GPU, after the step's context is gone
    config5 = config5_object(pkg, stream, local) if args.config5 else None
    gather = gather_peak() if rank == 0 else None

    # roofline of the dominant kernel group (largest device time per step)
    sm_max = (clk or {}).get("sm_max_mhz")
    if not sm_max:
        sm_max = json.load(open(PEAKS)).get("sm_max_mhz", 2070.0) if os.path.exists(PEAKS) else 2070.0
    hbm_peak = json.load(open(PEAKS)).get("hbm_gbs", 6800.0) if os.path.exists(PEAKS) else 6800.0
    total_ms = sum(v[0] for v in kt.values())
    dominant = max(("rev_search", "fwd_search", "instances"), key=lambda kname: kt[kname][0])
    roofline = kernel_roofline(dominant, kt, gold, g.m, w.l, args.steps, sm_max, hbm_peak, total_ms, w.name,
                               gather)
    sk_c, sm_c = gold["sketches"]["counters"], gold["skim"]["counters"]
    step_s = elapsed / args.steps

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_desc(w, g), "parallelism": f"replicas x{world}" if world > 1 else "none",
                       "queries_per_step": len(qs), "traversals_per_step": t_alg,
                       "l2": "no flush: the step's working set (ranks 0.8 GB, sketches 0.5 GB, graph 0.13 GB) "
                             "exceeds the 129 MB L2"},
            "s_to_50_seeds": statistics.median(part["greedy"]),
            "sketch_build_s": statistics.median(part["build"]),
            "rank_order_s": statistics.median(part["ranks"]),
            "instances_s": statistics.median(part["instances"]),
            "oracle_qps": len(qs) / statistics.median(part["query"]),
            "query_p50_ms": lat[len(lat) // 2], "query_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "single_query_qps": 1000.0 / (sum(lat) / len(lat)),
            "rates": {"live_edge_traversals_per_s": (sk_c["rev_live_edges"] + sm_c["rev_live_edges"]
                                                     + sm_c["fwd_live_edges"]) / step_s,
                      "reverse_expansions_per_s": (sk_c["rev_expansions"] + sm_c["rev_expansions"]) / step_s,
                      "instance_coins_per_s": 2 * g.m * w.l / statistics.median(part["instances"]),
                      "note": "live edges and expansions are the oracle's counts for the step; coins = 2 m l "
                              "(both CSR orders) per instance generation"},
            "coins_on_the_fly": on_the_fly,
            "serving_config4": serving,
            "batched": batched,
            "config5": config5,
            "adaptive_error": adaptive,
            "neighborhood_queries": neighborhood,
            "rank_modes": rank_modes,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "kernel_ms": {k2: round(v[0], 3) for k2, v in kt.items()},
            "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, trav = cpu_baseline(w, g, args.cpu_instances)
        full = gold["sketches"]["oracle_seconds"] + gold["skim"]["oracle_seconds"]
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"oracle Algorithm 2 on {args.cpu_instances} of the {w.l} instances of "
                                          f"{w.name} ({trav} traversals in {dt:.1f} s), single thread of the "
                                          f"host's {os.cpu_count()} cores",
                                "full_step_oracle_s": full, "full_step_oracle_value": t_alg / full,
                                "full_step_note": "the oracle's whole step (all sketches + 50 seeds), single "
                                                  "thread, as stored by tests/golden/make_golden.py on the "
                                                  "development host"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

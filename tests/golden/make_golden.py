"""Write full-size expected values from the CPU oracle (oracle/ only).

For a named workload this runs the oracle once and stores, in
``tests/golden/<workload>.json``:
  - the sha256 of the generated graph (so a changed generator is caught),
  - the sha256 of all combined sketches (Algorithm 2) and a few sampled rows,
  - the SKIM seed sequence and integer marginal coverages (Algorithm 1), with
    each selection's threshold rank and k' (Section 4.3.2),
  - influence-oracle estimates (Eq. unionest) for seeded uniform query sets,
  - the oracle's sequential work counters (edge-instance traversals).
No value here comes from the GPU path.

usage: python tests/golden/make_golden.py WORKLOAD [--skip-sketches] [--skip-skim]
       python tests/golden/make_golden.py batched256 [--jobs J]

``batched256`` is the many-graph workload: 256 R-MAT graphs (scale uniform in
10..16, edge factor uniform in 8..32), trivalency probabilities, l = 64,
k = 32, every graph with keys of its own.  For each graph the oracle builds its
sketches alone and the file stores the graph's digest, the sketch digest and
the oracle's counters (``batched256_trivalency.json``).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def sketch_digest(x: np.ndarray, ln: np.ndarray) -> str:
    """sha256 of len[n] (uint32 LE) followed by X[n,k] (uint64 LE, row-major,
    slots at or beyond len[v] zeroed)."""
    x = np.array(x, dtype=np.uint64, copy=True)
    k = x.shape[1]
    x[np.arange(k)[None, :] >= ln[:, None].astype(np.int64)] = 0
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ln, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(x, dtype="<u8").tobytes())
    return h.hexdigest()


def query_sets(w: synth.Workload, n: int, count: int = 24):
    ks = w.keys()
    sizes = synth.query_sizes(count, ks.query)
    return [synth.uniform_seed_set(n, int(s), ks.query, q).tolist() for q, s in enumerate(sizes)]


BATCHED_L, BATCHED_K, BATCHED_MODEL = 64, 32, 2


def _batched_one(spec):
    scale, ef, key = spec
    g = synth.rmat(scale, ef, key)
    ks = synth.Keys.from_seed(key)
    pb = oracle.Problem(g.n, g.src, g.dst, BATCHED_L, BATCHED_K, BATCHED_MODEL, 0.0, ks.coin, ks.rank, ks.prob)
    t = time.time()
    x, ln, cnt = oracle.build_sketches(pb)
    return {"scale": scale, "edge_factor": ef, "key": str(key), "n": g.n, "m": g.m, "graph_sha256": g.digest(),
            "sketch_sha256": sketch_digest(x, ln), "counters": cnt, "oracle_seconds": time.time() - t}


def batched_main(jobs: int):
    import multiprocessing as mp
    specs = synth.batched_graph_specs(256)
    t0 = time.time()
    with mp.get_context("spawn").Pool(jobs) as pool:
        graphs = pool.map(_batched_one, specs, chunksize=1)
    res = {"workload": "batched256_trivalency", "graphs": len(specs), "l": BATCHED_L, "k": BATCHED_K,
           "prob_model": BATCHED_MODEL, "spec": "synth.batched_graph_specs(256); keys synth.Keys.from_seed(key)",
           "per_graph": graphs, "oracle_seconds": sum(g["oracle_seconds"] for g in graphs)}
    out_path = os.path.join(HERE, "batched256_trivalency.json")
    json.dump(res, open(out_path + ".tmp", "w"), indent=1)
    os.replace(out_path + ".tmp", out_path)
    print(f"[batched256] wrote {out_path} ({time.time() - t0:.1f}s wall)", flush=True)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "batched256":
        ap = argparse.ArgumentParser()
        ap.add_argument("workload")
        ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
        batched_main(ap.parse_args().jobs)
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--skip-sketches", action="store_true")
    ap.add_argument("--skip-skim", action="store_true")
    ap.add_argument("--seeds", type=int, default=None)
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    out_path = os.path.join(HERE, f"{w.name}.json")
    res = json.load(open(out_path)) if os.path.exists(out_path) else {}
    t0 = time.time()
    g = w.graph()
    ks = w.keys()
    res.update({"workload": w.name, "n": g.n, "m": g.m, "graph_sha256": g.digest(),
                "l": w.l, "k": w.k, "prob_model": w.prob_model, "p": w.p})
    print(f"[{w.name}] graph n={g.n} m={g.m} ({time.time() - t0:.1f}s)", flush=True)
    pb = oracle.Problem(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob)
    if not args.skip_sketches:
        t = time.time()
        x, ln, cnt = oracle.build_sketches(pb)
        dt = time.time() - t
        rows = [0, 1, g.n // 3, g.n // 2, g.n - 1]
        qs = query_sets(w, g.n)
        res["sketches"] = {
            "sha256": sketch_digest(x, ln),
            "full_nodes": int((ln == w.k).sum()),
            "sample_rows": {str(v): [str(int(r)) for r in x[v, : ln[v]]] for v in rows},
            "counters": cnt,
            "oracle_seconds": dt,
        }
        res["queries"] = [{"seeds": q, "estimate": oracle.union_estimate(x, ln, w.l, q)} for q in qs]
        print(f"[{w.name}] sketches {dt:.1f}s {cnt}", flush=True)
        del x, ln
    if not args.skip_skim:
        s = args.seeds if args.seeds is not None else w.seeds
        if s:
            t = time.time()
            seeds, cov, tau, kp, cnt = oracle.skim_stops(pb, s)
            dt = time.time() - t
            res["skim"] = {"n_seeds": s, "seeds": seeds.tolist(), "cov": [int(c) for c in cov],
                           "tau": [str(int(x)) for x in tau], "kprime": [int(x) for x in kp],
                           "counters": cnt, "oracle_seconds": dt}
            print(f"[{w.name}] skim {s} seeds {dt:.1f}s {cnt}", flush=True)
    json.dump(res, open(out_path + ".tmp", "w"), indent=1)
    os.replace(out_path + ".tmp", out_path)
    print(f"[{w.name}] wrote {out_path}", flush=True)


if __name__ == "__main__":
    main()

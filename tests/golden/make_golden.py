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


def main():
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

"""GPU path vs the CPU oracle, through the C ABI.

Sketches, seed sequences and coverage counts must match bit for bit;
influence estimates within 1e-12 relative (the GPU sums exactly and rounds
once, the oracle sums in double in its own order).
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import paper_1408_6282_gb300 as p
    from paper_1408_6282_gb300 import build as b
    b.build()
    p.load()
    return p


def _both(pkg, g, l, k, model, p, seed, batch_lanes=0):
    ks = synth.Keys.from_seed(seed)
    pb = oracle.Problem(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob)
    sk = pkg.Skim(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob, batch_lanes=batch_lanes)
    return pb, sk


def _close(a, b):
    return abs(a - b) <= REL * max(abs(a), abs(b)) or (a == 0 and b == 0)


SMALL = [
    ("chain", lambda: synth.chain(40)),
    ("star", lambda: synth.star_out(50)),
    ("cycle", lambda: synth.cycle(33)),
    ("clique", lambda: synth.clique(9)),
    ("empty", lambda: synth.empty_graph(17)),
    ("single", lambda: synth.empty_graph(1)),
    ("er_sparse", lambda: synth.random_small_graph(300, 900, 3)),
    ("er_dense", lambda: synth.random_small_graph(120, 3000, 4)),
    ("rmat10", lambda: synth.rmat(10, 8, 99)),
]
CONF = [  # l, k, model, p, batch_lanes
    (1, 2, 0, 0.5, 0),
    (3, 4, 0, 0.3, 64),
    (16, 16, 0, 0.1, 0),
    (64, 8, 1, 0.0, 0),
    (64, 64, 1, 0.0, 128),
    (7, 5, 2, 0.0, 0),
    (64, 3, 0, 1.0, 256),
]


@pytest.mark.parametrize("name,mk", SMALL)
@pytest.mark.parametrize("l,k,model,p,bl", CONF)
def test_small_graphs_sketches_skim_queries(pkg, name, mk, l, k, model, p, bl):
    g = mk()
    pb, sk = _both(pkg, g, l, k, model, p, 11, bl)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_sketches(pb)
        assert np.array_equal(ln, oln)
        assert np.array_equal(x, ox)
        s = min(g.n, 25)
        seeds, cov, tau, kp = sk.greedy_stops(s)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, s)
        assert np.array_equal(seeds, os_), (seeds, os_)
        assert np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)  # Section 4.3.2 records
        rng = np.random.default_rng(5)
        sets = [[], [0], list(seeds[:3]), rng.integers(0, g.n, 10).tolist(), list(range(g.n))]
        single = [sk.query(q) for q in sets]
        batch = sk.query_batch(sets)
        for q, a, b in zip(sets, single, batch):
            assert a == b  # bitwise: same result alone and in a batch
            assert _close(a, oracle.union_estimate(ox, oln, l, q))


@pytest.mark.parametrize("name,mk", SMALL)
@pytest.mark.parametrize("l,k,model,p,bl", [CONF[1], CONF[3], CONF[5], CONF[6]])
def test_small_graphs_coins_hashed_in_the_search(pkg, name, mk, l, k, model, p, bl):
    """No instance stored: every search hashes the coins of the edges its lanes
    reach (Section 2's coins, evaluated on the fly).  Bit-exact as above, and
    switching the live rows back on gives the same results."""
    g = mk()
    pb, sk = _both(pkg, g, l, k, model, p, 11, bl)
    with sk:
        ox, oln, _ = oracle.build_sketches(pb)
        s = min(g.n, 25)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, s)
        for rows in (False, True):
            sk.set_live_rows(rows)
            sk.build_sketches()
            x, ln = sk.sketches()
            assert np.array_equal(ln, oln) and np.array_equal(x, ox), rows
            seeds, cov, tau, kp = sk.greedy_stops(s)
            assert np.array_equal(seeds, os_) and np.array_equal(cov, oc), rows
            assert np.array_equal(tau, otau) and np.array_equal(kp, okp), rows
            if not rows:
                st = sk.stats()
                assert st["rev_coins"] > 0 or g.m == 0  # the coins were drawn in the search
            assert sk.instance_stats()[1] == (rows and True)


@pytest.mark.parametrize("items", [512, 8192])
@pytest.mark.parametrize("ring", [0.0, 8.0])
@pytest.mark.parametrize("name,mk,conf", [("rmat10", SMALL[-1][1], CONF[3]), ("er_dense", SMALL[7][1], CONF[2]),
                                          ("chain", SMALL[0][1], CONF[6])])
def test_queue_overflow_parks_and_requeues(pkg, monkeypatch, items, ring, name, mk, conf):
    """A work queue far too small for the searches (SKIM_QUEUE_ITEMS): pushes
    past its end park their work in the pending masks, which are queued again
    once it drains, in reverse and residual searches, with stored instances
    and with coins hashed in the search.  Results stay the oracle's."""
    monkeypatch.setenv("SKIM_QUEUE_ITEMS", str(items))
    g = mk()
    l, k, model, p, bl = conf
    pb, sk = _both(pkg, g, l, k, model, p, 17, bl)
    monkeypatch.delenv("SKIM_QUEUE_ITEMS")
    ox, oln, _ = oracle.build_sketches(pb)
    s = min(g.n, 20)
    os_, oc, otau, okp, _ = oracle.skim_stops(pb, s)
    with sk:
        sk.set_tuning(bl, ring, 4)
        for rows in (True, False):
            sk.set_live_rows(rows)
            sk.build_sketches()
            requeued = sk.stats()["requeues"]
            x, ln = sk.sketches()
            assert np.array_equal(ln, oln) and np.array_equal(x, ox), rows
            sk.greedy_reset()
            seeds, cov, tau, kp = sk.greedy_stops(s)
            requeued += sk.stats()["requeues"]
            assert requeued > 0 or items > 512, rows  # the small queue did overflow
            assert np.array_equal(seeds, os_) and np.array_equal(cov, oc), rows
            assert np.array_equal(tau, otau) and np.array_equal(kp, okp), rows


@pytest.mark.parametrize("name,mk,conf,records", [("er_sparse", SMALL[6][1], CONF[2], 2048)])
def test_table_overflow_reruns_batches(pkg, monkeypatch, name, mk, conf, records):
    """Record and visited tables far too small for the default batches
    (SKIM_RECORD_ITEMS): overflowing build and SKIM batches stop early and are
    re-run with fewer lanes.  Results stay the oracle's."""
    monkeypatch.setenv("SKIM_RECORD_ITEMS", str(records))
    g = mk()
    l, k, model, p, bl = conf
    pb, sk = _both(pkg, g, l, k, model, p, 19, 1 << 16)
    monkeypatch.delenv("SKIM_RECORD_ITEMS")
    ox, oln, _ = oracle.build_sketches(pb)
    s = min(g.n, 20)
    os_, oc, otau, okp, _ = oracle.skim_stops(pb, s)
    with sk:
        sk.build_sketches()
        retried = sk.stats()["retries"]
        x, ln = sk.sketches()
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov, tau, kp = sk.greedy_stops(s)
        retried += sk.stats()["retries"]
        assert retried > 0  # the small tables did overflow
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)


@pytest.mark.parametrize("ring", [0.0, 1e9])
@pytest.mark.parametrize("name,mk,conf", [("rmat10", SMALL[-1][1], CONF[4]), ("er_dense", SMALL[7][1], (16, 16, 0, 0.1, 64)),
                                          ("rmat12", lambda: synth.rmat(12, 16, 77), (64, 32, 1, 0.0, 2048))])
def test_search_kernels_each_alone(pkg, ring, name, mk, conf):
    """Every batch of reverse searches on the global queue (ring = 0), or every
    batch whose records per lane are known on the per-warp queues (ring =
    1e9), with records radix sorted (density 0) or placed by node buckets:
    each setting gives the oracle's sketches and seeds."""
    g = mk()
    l, k, model, p, bl = conf
    pb, sk = _both(pkg, g, l, k, model, p, 13, bl)
    ox, oln, _ = oracle.build_sketches(pb)
    os_, oc, otau, okp, _ = oracle.skim_stops(pb, min(g.n, 20))
    with sk:
        for density in (0, 1, 1 << 30):
            sk.set_tuning(bl, ring, density)
            assert sk.tuning() == {"batch_lanes": bl, "ring_records_per_lane": ring, "node_sort_density": density}
            sk.build_sketches()
            x, ln = sk.sketches()
            assert np.array_equal(ln, oln) and np.array_equal(x, ox), density
            sk.greedy_reset()
            seeds, cov, tau, kp = sk.greedy_stops(min(g.n, 20))
            assert np.array_equal(seeds, os_) and np.array_equal(cov, oc), density
            assert np.array_equal(tau, otau) and np.array_equal(kp, okp), density


@pytest.mark.parametrize("density", [0, 4])
def test_record_order_hub_in_sparse_batches(pkg, density):
    """A star of 100000 leaves with every edge live and k = 200: every lane's
    reverse search reaches the centre until its local sketches fill, so the
    second batch (8192 lanes) gives the centre a record in each of its 128 words
    (the block pass of the record order) while the batch's records are sparse
    over the nodes (placement by buckets of nodes, density 4) -- and the same
    with the radix sort (density 0).  Sketches and seeds match the oracle."""
    g = synth.star_out(100000)
    l, k = 4, 200
    pb, sk = _both(pkg, g, l, k, 0, 1.0, 21, 8192)
    ox, oln, _ = oracle.build_sketches(pb)
    os_, oc, otau, okp, _ = oracle.skim_stops(pb, 20)
    with sk:
        sk.set_tuning(8192, 8.0, density)
        sk.build_sketches()
        x, ln = sk.sketches()
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov, tau, kp = sk.greedy_stops(20)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)


@pytest.mark.parametrize("bl", [0, 64, 1024])
def test_skim_full_permutation_and_resume(pkg, bl):
    g = synth.random_small_graph(200, 1200, 8)
    pb, sk = _both(pkg, g, 8, 6, 1, 0.0, 21, bl)
    with sk:
        a, ca = sk.greedy(7)
        b, cb, tb, kb = sk.greedy_stops(g.n - 7)  # continues the sequence to exhaustion
        seeds = np.concatenate([a, b])
        cov = np.concatenate([ca, cb])
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, g.n)
        assert np.array_equal(seeds, os_)
        assert np.array_equal(cov, oc)
        assert np.array_equal(tb, otau[7:]) and np.array_equal(kb, okp[7:])
        assert okp[-1] == -1  # the tail comes from exact residual counts
        assert sorted(seeds.tolist()) == list(range(g.n))
        sk.greedy_reset()
        c, cc = sk.greedy(10)
        assert np.array_equal(c, os_[:10]) and np.array_equal(cc, oc[:10])


def test_er4096_workload(pkg):
    w = synth.WORKLOADS["er4096"]
    g = w.graph()
    pb, sk = _both(pkg, g, w.l, w.k, w.prob_model, w.p, w.seed)
    gold = json.load(open(os.path.join(GOLDEN, "er4096.json")))
    assert g.digest() == gold["graph_sha256"]
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        assert _digest(x, ln) == gold["sketches"]["sha256"]
        _check_skim(sk, gold["skim"], w.seeds)
        for q in gold["queries"]:
            assert _close(sk.query(q["seeds"]), q["estimate"])


@pytest.mark.parametrize("scale,model,p", [(12, 1, 0.0), (13, 0, 0.02), (12, 2, 0.0)])
def test_rmat_midsize(pkg, scale, model, p):
    ks = synth.Keys.from_seed(40 + scale)
    g = synth.rmat(scale, 16, ks.graph)
    pb, sk = _both(pkg, g, 64, 32, model, p, 40 + scale)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_sketches(pb)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov, tau, kp = sk.greedy_stops(40)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, 40)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)
        pre = oracle.exact_coverage(pb, seeds)
        assert np.array_equal(np.cumsum(cov), pre)


def _digest(x, ln):
    x = np.array(x, dtype=np.uint64, copy=True)
    k = x.shape[1]
    x[np.arange(k)[None, :] >= ln[:, None].astype(np.int64)] = 0
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ln, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(x, dtype="<u8").tobytes())
    return h.hexdigest()


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    return json.load(open(path))


@pytest.mark.parametrize("name", ["rmat18_wc", "rmat20_wc", "rmat20_p01"])
def test_rmat_wc_full_size(pkg, name):
    """R-MAT scale 18 and 20 with weighted cascade, and scale 20 with uniform
    p = 0.01 (hub-heavy searches, as at scale 24), l = k = 64: every sketch, 50
    SKIM seeds and the query set against stored oracle values."""
    gold = _golden(name)
    w = synth.WORKLOADS[name]
    g = w.graph(device="cuda")
    assert g.digest() == gold["graph_sha256"]
    ks = w.keys()
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        for v, row in gold["sketches"]["sample_rows"].items():
            assert [str(int(r)) for r in x[int(v), : ln[int(v)]]] == row
        assert _digest(x, ln) == gold["sketches"]["sha256"]
        est = sk.query_batch([q["seeds"] for q in gold["queries"]])
        for q, e in zip(gold["queries"], est):
            assert _close(float(e), q["estimate"])
        _check_skim(sk, gold["skim"], w.seeds)


def test_contexts_on_pooled_memory(pkg):
    """Contexts created one after another reuse the pooled blocks of the
    destroyed ones (stale contents included) and after a release take fresh
    ones: the sketches match the stored oracle values every time."""
    gold = _golden("er4096")
    w = synth.WORKLOADS["er4096"]
    g = w.graph()
    ks = w.keys()
    for rep in range(3):
        if rep == 2:
            pkg.skim_release_memory()
        with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
            sk.build_sketches()
            x, ln = sk.sketches()
            assert _digest(x, ln) == gold["sketches"]["sha256"]
            _check_skim(sk, gold["skim"], w.seeds)


def test_rmat18_wc_coins_hashed_in_the_search(pkg):
    """R-MAT scale 18, weighted cascade, l = k = 64 with no instance stored:
    the searches hash every reached edge's coins; sketches, 50 seeds, their
    thresholds and k' against the stored oracle values."""
    gold = _golden("rmat18_wc")
    w = synth.WORKLOADS["rmat18_wc"]
    g = w.graph(device="cuda")
    ks = w.keys()
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
        sk.set_live_rows(False)
        sk.build_sketches()
        x, ln = sk.sketches()
        assert _digest(x, ln) == gold["sketches"]["sha256"]
        _check_skim(sk, gold["skim"], w.seeds)


def test_rmat18_wc_sketches_large_batches(pkg):
    """Batches of up to 2^24 lanes (the record table holds them to about 8M
    here: 17 word bits, so 32 KB of shared memory per block for a node's word
    bitmap and its prefix counts, four times the default run's): the sketches
    must still match the stored oracle values."""
    gold = _golden("rmat18_wc")
    w = synth.WORKLOADS["rmat18_wc"]
    g = w.graph(device="cuda")
    ks = w.keys()
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob,
                  batch_lanes=1 << 24) as sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        assert _digest(x, ln) == gold["sketches"]["sha256"]


def _check_skim(sk, gs, s):
    """Seeds and coverages, and the Section 4.3.2 records where stored."""
    seeds, cov, tau, kp = sk.greedy_stops(s)
    assert seeds.tolist() == gs["seeds"]
    assert [int(c) for c in cov] == gs["cov"]
    if "tau" in gs:
        assert [str(int(t)) for t in tau] == gs["tau"]
        assert [int(x) for x in kp] == gs["kprime"]


def test_rmat22_wc_sketches_full_size(pkg):
    gold = _golden("rmat22_wc")
    if "sketches" not in gold:
        pytest.skip("no stored sketches")
    w = synth.WORKLOADS["rmat22_wc"]
    g = w.graph(device="cuda")
    assert g.digest() == gold["graph_sha256"]
    ks = w.keys()
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        assert _digest(x, ln) == gold["sketches"]["sha256"]
        est = sk.query_batch([q["seeds"] for q in gold["queries"]])
        for q, e in zip(gold["queries"], est):
            assert _close(float(e), q["estimate"])


def test_rmat24_p01_skim_full_size(pkg):
    """R-MAT scale 24, uniform p = 0.01, l = k = 64: every sketch (where the
    oracle's digest is stored), sampled rows, the query set and 200 SKIM seeds
    against stored oracle values."""
    gold = _golden("rmat24_p01")
    if "skim" not in gold:
        pytest.skip("no stored seeds")
    w = synth.WORKLOADS["rmat24_p01"]
    g = w.graph(device="cuda")
    assert g.digest() == gold["graph_sha256"]
    ks = w.keys()
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
        if "sketches" in gold:
            sk.build_sketches()
            x, ln = sk.sketches()
            for v, row in gold["sketches"]["sample_rows"].items():
                assert [str(int(r)) for r in x[int(v), : ln[int(v)]]] == row
            assert _digest(x, ln) == gold["sketches"]["sha256"]
            del x, ln
            est = sk.query_batch([q["seeds"] for q in gold["queries"]])
            for q, e in zip(gold["queries"], est):
                assert _close(float(e), q["estimate"])
        _check_skim(sk, gold["skim"], w.seeds)


def test_query_sum_is_correctly_rounded(pkg):
    """The estimate equals the exact sum of the per-rank terms 1/tau, rounded
    once to double, then divided by l."""
    g = synth.random_small_graph(3000, 20000, 17)
    ks = synth.Keys.from_seed(17)
    l, k = 16, 8
    with pkg.Skim(g.n, g.src, g.dst, l, k, 0, 0.2, ks.coin, ks.rank, ks.prob) as sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        rng = np.random.default_rng(3)
        for size in (1, 2, 17, 200, 1000):
            S = rng.choice(g.n, size=size, replace=False)
            best = {}
            for u in S:
                m = int(ln[u])
                tau = int(x[u, k - 1]) if m == k else (1 << 64) - 1
                body = x[u, : k - 1] if m == k else x[u, :m]
                for z in body:
                    z = int(z)
                    best[z] = max(best.get(z, 0), tau)
            exact = sum((Fraction(1.0 / math.ldexp(float(t), -64)) for t in best.values()), Fraction(0))
            ref = float(exact) / l
            assert sk.query(S) == ref


def test_error_codes(pkg):
    g = synth.random_small_graph(50, 200, 2)
    with pkg.Skim(g.n, g.src, g.dst, 4, 4, 0, 0.2, 1, 2, 3) as sk:
        with pytest.raises(pkg.SkimError) as e:
            sk.query([1, 2])
        assert e.value.code == -3  # not built
        sk.build_sketches()
        with pytest.raises(pkg.SkimError) as e:
            sk.query([1, 50])
        assert e.value.code == -1
        with pytest.raises(pkg.SkimError) as e:
            sk.greedy(51)
        assert e.value.code == -1
    src = np.array([1, 0], np.uint32)
    dst = np.array([2, 1], np.uint32)  # not sorted
    with pytest.raises(pkg.SkimError) as e:
        pkg.Skim(3, src, dst, 4, 4)
    assert e.value.code == -6
    with pytest.raises(pkg.SkimError) as e:
        pkg.Skim(3, np.array([1], np.uint32), np.array([1], np.uint32), 4, 4)  # self-loop
    assert e.value.code == -6


def test_long_path_graph(pkg):
    """A 200000-node path, every edge live: reverse searches are long chains
    of single successors (the local-continuation limit and the progress
    watchdog must both hold)."""
    g = synth.chain(200000)
    pb, sk = _both(pkg, g, 4, 4, 0, 1.0, 5)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_sketches(pb)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov, tau, kp = sk.greedy_stops(5)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, 5)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)

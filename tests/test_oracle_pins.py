"""Pins of the CPU oracle against things other than itself: published hash
vectors, brute force on tiny graphs (independent Python, tests/_brute.py),
exact greedy, closed forms, a hand-worked estimator example, invariants and
statistics.  CPU only."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import _brute as B
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(g, l, k, model=0, p=0.3, seed=7):
    ks = synth.Keys.from_seed(seed)
    return oracle.Problem(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob)


def _inst(pb):
    return B.Instances(pb.n, pb.src, pb.dst, pb.l, pb.model, pb.p, pb.coin_key, pb.prob_key)


TINY = [
    ("chain", lambda: synth.chain(7)),
    ("star", lambda: synth.star_out(6)),
    ("cycle", lambda: synth.cycle(6)),
    ("clique", lambda: synth.clique(5)),
    ("empty", lambda: synth.empty_graph(4)),
    ("er_a", lambda: synth.random_small_graph(10, 25, 11)),
    ("er_b", lambda: synth.random_small_graph(12, 40, 12)),
    ("er_c", lambda: synth.random_small_graph(9, 30, 13)),
]
PARAMS = [(1, 2, 0, 0.5), (2, 3, 0, 0.3), (3, 5, 1, 0.0), (4, 4, 2, 0.0), (2, 40, 0, 0.6)]


# --------------------------------------------------------------------------
# Hashes, ranks and coins
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, val = line.split()
        # rank(key=0, l=1, v=t, i=0) = fmix(0 + t*G): output t of the stream with state 0
        assert oracle.rank(0, 1, int(t), 0) == int(val, 16)


def test_rank_formula_and_distinctness():
    key, l = 0x1234, 5
    vals = {oracle.rank(key, l, v, i) for v in range(40) for i in range(l)}
    assert len(vals) == 40 * l
    for v, i in [(0, 0), (3, 4), (39, 2)]:
        assert oracle.rank(key, l, v, i) == B.rank(key, l, v, i)


@pytest.mark.parametrize("model,p", [(0, 0.1), (0, 0.01), (1, 0.0), (2, 0.0), (0, 1.0)])
def test_coin_matches_independent_definition(model, p):
    g = synth.random_small_graph(30, 200, 5)
    pb = _problem(g, 8, 4, model, p)
    inst = _inst(pb)
    for e in range(0, g.m, 7):
        u, v = int(g.src[e]), int(g.dst[e])
        for i in range(pb.l):
            assert oracle.live(pb, u, v, i) == (v in inst.out[i][u])


def test_coin_frequency_and_special_thresholds():
    g = synth.random_small_graph(200, 3000, 9)
    pb = _problem(g, 16, 4, 0, 0.1)
    inst = _inst(pb)
    live = sum(len(inst.out[i][u]) for i in range(16) for u in range(g.n))
    trials = g.m * 16
    sd = math.sqrt(trials * 0.1 * 0.9)
    assert abs(live - 0.1 * trials) < 5 * sd
    # p = 1: every edge live in every instance
    pb1 = _problem(g, 4, 4, 0, 1.0)
    assert all(oracle.live(pb1, int(g.src[e]), int(g.dst[e]), i) for e in range(0, g.m, 50) for i in range(4))
    # weighted cascade: an edge into a node of in-degree 1 is always live
    ch = synth.chain(6)
    pbw = _problem(ch, 8, 4, 1)
    assert all(oracle.live(pbw, u, u + 1, i) for u in range(5) for i in range(8))


# --------------------------------------------------------------------------
# Sketches: Eq. combinedrs by brute force; Algorithm 2 must give the same
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", TINY)
@pytest.mark.parametrize("l,k,model,p", PARAMS)
def test_sketches_match_brute_force(name, mk, l, k, model, p):
    g = mk()
    pb = _problem(g, l, k, model, p)
    inst = _inst(pb)
    x, ln, cnt = oracle.build_sketches(pb)
    for u in range(g.n):
        ref = B.sketch(inst, u, k, pb.rank_key)
        assert list(x[u, : ln[u]]) == ref, (name, u)
        xs, reach = oracle.sketch_of_node(pb, u)
        assert list(xs) == ref
        assert reach == len(inst.combined_reach(u))


def test_single_instance_is_cohen_reachability_sketch():
    # l = 1 (Section 3): the combined sketch is the reachability sketch of the one instance
    g = synth.random_small_graph(12, 30, 21)
    pb = _problem(g, 1, 3, 0, 0.5)
    inst = _inst(pb)
    x, ln, _ = oracle.build_sketches(pb)
    for u in range(g.n):
        rs = sorted(B.rank(pb.rank_key, 1, v, 0) for v in inst.reach(u, 0))
        assert list(x[u, : ln[u]]) == rs[:3]


def test_sketch_invariants_midsize():
    g = synth.random_small_graph(300, 1500, 31)
    pb = _problem(g, 6, 8, 1)
    x, ln, _ = oracle.build_sketches(pb)
    assert np.all(ln <= pb.k) and np.all(ln >= 1)
    for u in range(0, g.n, 17):
        row = x[u, : ln[u]]
        assert np.all(np.diff(row.astype(object)) > 0)
        xs, reach = oracle.sketch_of_node(pb, u)
        assert np.array_equal(xs, row)
        assert ln[u] == min(pb.k, reach)
    # live edge w->v in instance i: every instance-i rank of X_v below tau_w is in X_w
    inst = _inst(pb)
    rank_inst = {oracle.rank(pb.rank_key, pb.l, v, i): i for v in range(g.n) for i in range(pb.l)}
    for i in range(pb.l):
        for w in range(0, g.n, 7):
            tw = x[w, pb.k - 1] if ln[w] == pb.k else None
            for v in inst.out[i][w]:
                for r in x[v, : ln[v]]:
                    if rank_inst[int(r)] == i and (tw is None or r <= tw):
                        assert r in set(x[w, : ln[w]])


# --------------------------------------------------------------------------
# Exact coverage (Eq. InfbinaryIC)
# --------------------------------------------------------------------------

def test_exact_coverage_brute_force():
    g = synth.random_small_graph(15, 50, 41)
    pb = _problem(g, 3, 4, 0, 0.4)
    inst = _inst(pb)
    seeds = [3, 7, 3, 0]
    pre = oracle.exact_coverage(pb, seeds)
    for j in range(len(seeds)):
        assert pre[j] == inst.coverage(seeds[: j + 1])


# --------------------------------------------------------------------------
# SKIM, Algorithm 1
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", TINY)
@pytest.mark.parametrize("l,model,p", [(1, 0, 0.5), (3, 0, 0.3), (2, 1, 0.0), (3, 2, 0.0)])
def test_skim_large_k_is_exact_greedy(name, mk, l, model, p):
    # k > n*l: no partial sketch can fill, every rank is processed and the
    # choice is argmax size = exact marginal gain (Section 4)
    g = mk()
    pb = _problem(g, l, g.n * l + 1, model, p)
    inst = _inst(pb)
    s = g.n
    seeds, cov, _, _ = oracle.skim(pb, s)
    ref_seeds, ref_gain = B.exact_greedy(inst, s)
    assert list(seeds) == ref_seeds
    assert list(cov) == ref_gain
    assert sorted(seeds) == list(range(g.n))  # a permutation of the nodes


def _sorted_pairs(pb):
    pairs = [(oracle.rank(pb.rank_key, pb.l, v, i), v, i) for v in range(pb.n) for i in range(pb.l)]
    pairs.sort()
    return pairs


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_skim_first_to_k_and_lemma(seed):
    g = synth.random_small_graph(14, 45, 100 + seed)
    pb = _problem(g, 3, 3 + seed % 3, seed % 2, 0.35, seed=seed)
    inst = _inst(pb)
    reach = [[inst.reach(u, i) for i in range(pb.l)] for u in range(g.n)]
    pairs = _sorted_pairs(pb)
    k, nl = pb.k, g.n * pb.l
    covered = [set() for _ in range(pb.l)]
    prev_consumed = 0
    S = 8
    for j in range(1, S + 1):
        seeds, cov, size, cnt = oracle.skim(pb, j)
        consumed = cnt["ranks_consumed"]
        x = int(seeds[-1])

        def c_at(u, upto):  # processed uncovered pairs (z,i) with u ~> z in the current residual
            return sum(1 for (_, z, i) in pairs[:upto] if z not in covered[i] and z in reach[u][i])

        cmax_end = max(c_at(u, consumed) for u in range(g.n))
        if cmax_end >= k:  # found by first-to-k on the last consumed rank
            filled = [u for u in range(g.n) if c_at(u, consumed) >= k]
            assert x == min(filled)
            assert max(c_at(u, consumed - 1) for u in range(g.n)) < k
            assert consumed > prev_consumed
        else:
            assert consumed == nl
        # residual: forward reach of x, then the lemma on every partial sketch
        newly = 0
        for i in range(pb.l):
            add = reach[x][i] - covered[i]
            newly += len(add)
            covered[i] |= add
        assert cov[-1] == newly
        for u in range(g.n):
            assert size[u] == c_at(u, consumed), (j, u)
        assert size[x] == 0
        prev_consumed = consumed
    pre = oracle.exact_coverage(pb, seeds)
    assert np.array_equal(np.cumsum(cov), pre)


def test_skim_prefix_is_consistent_and_coverage_monotone():
    g = synth.random_small_graph(200, 900, 77)
    pb = _problem(g, 8, 6, 1)
    s20, c20, _, _ = oracle.skim(pb, 20)
    s7, c7, _, _ = oracle.skim(pb, 7)
    assert np.array_equal(s20[:7], s7) and np.array_equal(c20[:7], c7)
    assert len(set(s20.tolist())) == 20
    pre = oracle.exact_coverage(pb, s20)
    assert np.array_equal(np.cumsum(c20), pre)
    assert np.all(np.diff(pre.astype(np.int64)) >= 0)


# --------------------------------------------------------------------------
# Influence estimation (Section 5.1)
# --------------------------------------------------------------------------

def test_union_estimator_worked_example():
    k, l = 3, 2
    x = np.zeros((3, k), np.uint64)
    ln = np.zeros(3, np.uint32)
    rows = {"a": [10, 20, 40], "b": [20, 30], "c": [10, 30, 50]}
    ids = {"a": 0, "b": 1, "c": 2}
    for name, r in rows.items():
        x[ids[name], : len(r)] = r
        ln[ids[name]] = len(r)
    for line in open(os.path.join(GOLDEN, "unionest_worked_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        names, num, den = line.split()
        seeds = [ids[s] for s in names.split(",")]
        exact = Fraction(int(num), int(den)) / l
        assert B.union_estimate_exact([rows[s] for s in names.split(",")], k) / l == exact
        got = oracle.union_estimate(x, ln, l, seeds)
        assert abs(got - float(exact)) <= 1e-15 * float(exact)


def test_single_seed_estimate_closed_form():
    g = synth.random_small_graph(300, 1500, 51)
    pb = _problem(g, 4, 8, 0, 0.4)
    x, ln, _ = oracle.build_sketches(pb)
    for u in range(0, g.n, 13):
        est = oracle.union_estimate(x, ln, pb.l, [u])
        if ln[u] == pb.k:
            tau = math.ldexp(float(int(x[u, pb.k - 1])), -64)
            ref = (pb.k - 1) / tau / pb.l
        else:
            ref = ln[u] / pb.l
        assert est == pytest.approx(ref, rel=1e-15)
        assert oracle.bottomk_union_estimate(x, ln, pb.l, [u]) == pytest.approx(ref, rel=1e-15)


def test_estimate_is_exact_when_sketches_not_full():
    g = synth.random_small_graph(12, 20, 61)
    pb = _problem(g, 3, 64, 0, 0.3)  # k > n*l: every sketch holds its whole R_u
    inst = _inst(pb)
    x, ln, _ = oracle.build_sketches(pb)
    assert np.all(ln < pb.k)
    for seeds in ([0], [1, 2, 3], [5, 5, 6], list(range(12)), []):
        est = oracle.union_estimate(x, ln, pb.l, seeds)
        assert est == pytest.approx(inst.coverage(seeds) / pb.l, rel=1e-15, abs=0)


def test_identical_sets_match_bottomk_of_union():
    g = synth.random_small_graph(300, 2000, 71)
    pb = _problem(g, 4, 6, 0, 0.5)
    x, ln, _ = oracle.build_sketches(pb)
    u = int(np.argmax(ln))
    for seeds in ([u, u], [u, u, u, u]):
        a = oracle.union_estimate(x, ln, pb.l, seeds)
        b = oracle.bottomk_union_estimate(x, ln, pb.l, seeds)
        assert a == pytest.approx(b, rel=1e-15)
    # distinct nodes with identical reachability sets (a cycle): same result
    cy = synth.cycle(40)
    pbc = _problem(cy, 2, 6, 0, 1.0)
    xc, lc, _ = oracle.build_sketches(pbc)
    a = oracle.union_estimate(xc, lc, 2, [0, 5, 17])
    b = oracle.bottomk_union_estimate(xc, lc, 2, [0, 5, 17])
    assert a == pytest.approx(b, rel=1e-15)


def test_union_estimator_matches_exact_rationals_on_random_sketches():
    rng = np.random.default_rng(5)
    k, l, n = 5, 3, 8
    x = np.zeros((n, k), np.uint64)
    ln = np.zeros(n, np.uint32)
    pool = rng.choice(1 << 40, size=30, replace=False).astype(np.uint64) * np.uint64(1 << 20)
    rows = []
    for v in range(n):
        m = int(rng.integers(1, k + 1))
        r = sorted(int(t) for t in rng.choice(pool, size=m, replace=False))
        rows.append(r)
        x[v, :m] = r
        ln[v] = m
    for seeds in ([0, 1], [2, 3, 4], list(range(n)), [7, 7, 1]):
        exact = B.union_estimate_exact([rows[s] for s in seeds], k) / l
        assert oracle.union_estimate(x, ln, l, seeds) == pytest.approx(float(exact), rel=1e-14)


@pytest.mark.slow
def test_estimator_unbiased_and_cv_bound():
    # Theorem of Section 5: unbiased; single-node CV <= 1/sqrt(k-2) (Section 3)
    g = synth.random_small_graph(400, 1600, 81)
    l, k = 4, 10
    ks = synth.Keys.from_seed(3)
    inst = B.Instances(g.n, g.src, g.dst, l, 0, 0.45, ks.coin, 0)
    u = 0
    qs = [0, 1, 2, 3, 4, 5, 6, 7]
    exact_u = len(inst.combined_reach(u)) / l
    exact_q = inst.coverage(qs) / l
    eu, eq = [], []
    for t in range(300):
        pb = oracle.Problem(g.n, g.src, g.dst, l, k, 0, 0.45, ks.coin, 1000 + t, 0)
        x, ln, _ = oracle.build_sketches(pb)
        eu.append(oracle.union_estimate(x, ln, l, [u]))
        eq.append(oracle.union_estimate(x, ln, l, qs))
    for est, ex in ((np.array(eu), exact_u), (np.array(eq), exact_q)):
        assert abs(est.mean() - ex) < 4 * est.std() / math.sqrt(len(est)) + 1e-9
    if exact_u * l > k:
        cv = np.std(eu) / exact_u
        assert cv <= 1.25 / math.sqrt(k - 2)


@pytest.mark.parametrize("name,mk", TINY[:6])
def test_work_counters_without_pruning_match_brute_force(name, mk):
    # With k > n*l no local sketch fills, so the reverse search of every pair
    # (u,i) expands each v that reaches u in instance i: expansions =
    # sum over (v,i) of |R(G_i, v)|, live reverse edges = the same weighted by
    # v's live in-degree in instance i.
    g = mk()
    l = 3
    pb = _problem(g, l, g.n * l + 1, 0, 0.4)
    inst = _inst(pb)
    indeg_live = [[0] * g.n for _ in range(l)]
    for i in range(l):
        for u in range(g.n):
            for v in inst.out[i][u]:
                indeg_live[i][v] += 1
    reach = [[len(inst.reach(v, i)) for i in range(l)] for v in range(g.n)]
    _, _, cnt = oracle.build_sketches(pb)
    assert cnt["rev_expansions"] == sum(reach[v][i] for v in range(g.n) for i in range(l))
    assert cnt["rev_live_edges"] == sum(reach[v][i] * indeg_live[i][v] for v in range(g.n) for i in range(l))
    indeg = np.bincount(g.dst, minlength=g.n) if g.m else np.zeros(g.n, int)
    assert cnt["rev_edge_scans"] == sum(reach[v][i] * int(indeg[v]) for v in range(g.n) for i in range(l))

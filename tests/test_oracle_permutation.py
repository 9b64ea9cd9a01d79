"""Structured permutation ranks (Section 3.1), IC-model sketches (Section 3.2)
and their estimators: the oracle against brute force (tests/_brute.py),
invariants, exact expectations and statistics.  CPU only."""
from __future__ import annotations

import math
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

import _brute as B
import oracle
import synth


def _problem(g, l, k, model=0, p=0.3, seed=7):
    ks = synth.Keys.from_seed(seed)
    return oracle.Problem(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob)


def _inst(pb, l=None):
    return B.Instances(pb.n, pb.src, pb.dst, l or pb.l, pb.model, pb.p, pb.coin_key, pb.prob_key)


TINY = [
    ("chain", lambda: synth.chain(6)),
    ("star", lambda: synth.star_out(5)),
    ("cycle", lambda: synth.cycle(5)),
    ("clique", lambda: synth.clique(4)),
    ("empty", lambda: synth.empty_graph(3)),
    ("er_a", lambda: synth.random_small_graph(9, 22, 31)),
    ("er_b", lambda: synth.random_small_graph(11, 35, 32)),
]


# --------------------------------------------------------------------------
# The structured permutation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,l", [(1, 1), (5, 1), (7, 3), (40, 8), (300, 64)])
def test_positions_are_a_chunked_permutation(n, l):
    key = 0xABCDEF + n * l
    pos = oracle.perm_positions(n, l, key).reshape(n, l)
    assert sorted(pos.ravel().tolist()) == list(range(n * l))  # a bijection
    chunk = pos // n
    for v in range(n):  # each node once per chunk, so its instances form a permutation
        assert sorted(chunk[v].tolist()) == list(range(l))
    if n * l <= 64 * 40:
        ref = B.perm_positions(n, l, key)
        assert all(int(pos[v, i]) == ref[(v, i)] for v in range(n) for i in range(l))


def test_ic_nodes_chunks_are_permutations():
    n, k, key = 37, 5, 99
    nodes = oracle.ic_nodes(n, k, key)
    assert nodes.tolist() == B.ic_nodes(n, k, key)
    for c in range(k):
        assert sorted(nodes[c * n:(c + 1) * n].tolist()) == list(range(n))
    # the same chunk order as the instance model's structured permutation
    pos = oracle.perm_positions(n, k, key).reshape(n, k)
    for t in range(n * k):
        v = int(nodes[t])
        assert t in pos[v].tolist()


def test_positions_look_uniform():
    n, l = 20000, 8
    pos = oracle.perm_positions(n, l, 4242).reshape(n, l).astype(np.int64)
    chunk = pos // n
    # the instance a node uses in chunk 0 is uniform over the l instances
    first = np.argmin(chunk, axis=1)
    cnt = np.bincount(first, minlength=l)
    chi2 = float(((cnt - n / l) ** 2 / (n / l)).sum())
    assert chi2 < 35.0  # chi-square with 7 d.o.f.: P[> 35] ~ 1e-5
    # positions within consecutive chunks are independent of each other
    within = pos % n
    order = np.argsort(chunk, axis=1)
    w0 = within[np.arange(n), order[:, 0]]
    w1 = within[np.arange(n), order[:, 1]]
    assert abs(np.corrcoef(w0, w1)[0, 1]) < 0.04


# --------------------------------------------------------------------------
# Sketches
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,mk", TINY)
@pytest.mark.parametrize("l,k,model,p", [(1, 2, 0, 0.5), (3, 2, 0, 0.4), (3, 5, 1, 0.0), (4, 3, 2, 0.0),
                                         (2, 30, 0, 0.6)])
def test_permutation_sketches_match_brute_force(name, mk, l, k, model, p):
    g = mk()
    pb = _problem(g, l, k, model, p)
    inst = _inst(pb)
    pos = B.perm_positions(g.n, l, pb.rank_key)
    x, ln, _ = oracle.build_sketches(pb, rank_mode=1)
    for u in range(g.n):
        ref = sorted(pos[pair] for pair in inst.combined_reach(u))[:k]
        assert x[u, : ln[u]].tolist() == ref, (u, ref)
        # only the first min(k, l) chunks can appear (u reaches itself)
        assert all(q < min(k, l) * g.n for q in ref)


@pytest.mark.parametrize("name,mk", TINY)
@pytest.mark.parametrize("k,model,p", [(2, 0, 0.5), (3, 1, 0.0), (4, 0, 0.3), (3, 2, 0.0)])
def test_ic_sketches_match_brute_force(name, mk, k, model, p):
    g = mk()
    pb = _problem(g, 1, k, model, p, seed=3)
    npos = k * g.n
    inst = _inst(pb, l=npos)  # instance t is G_t of position t
    nodes = B.ic_nodes(g.n, k, pb.rank_key)
    x, ln, _ = oracle.build_ic_sketches(pb)
    for u in range(g.n):
        ref = [t for t in range(npos) if nodes[t] in inst.reach(u, t)][:k]
        assert ln[u] == k  # u reaches itself once per chunk
        assert x[u].tolist() == ref


# --------------------------------------------------------------------------
# SKIM over the structured permutation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_permutation_skim_matches_brute_force(seed):
    g = synth.random_small_graph(14, 45, 700 + seed)
    l, k = 3, 2 + seed % 3
    pb = _problem(g, l, k, seed % 2, 0.35, seed=seed)
    inst = _inst(pb)
    reach = [[inst.reach(u, i) for i in range(l)] for u in range(g.n)]
    rank = B.perm_positions(g.n, l, pb.rank_key)
    seeds, cov, tau, kp, _ = oracle.skim_stops(pb, g.n, rank_mode=1)
    covered = [set() for _ in range(l)]
    for j in range(g.n):
        x = int(seeds[j])
        uncovered = [(v, i) for (v, i) in rank if v not in covered[i]]
        if kp[j] < 0:
            for u in range(g.n):
                assert sum(1 for (v, i) in uncovered if v in reach[u][i]) < k
        else:
            t = int(tau[j])
            stop = [(v, i) for (v, i) in uncovered if rank[(v, i)] == t]
            assert len(stop) == 1 and stop[0][0] in reach[x][stop[0][1]]
            cnt = [sum(1 for (v, i) in uncovered if rank[(v, i)] < t and v in reach[u][i]) for u in range(g.n)]
            hit = [cnt[u] + (stop[0][0] in reach[u][stop[0][1]]) for u in range(g.n)]
            assert max(cnt) <= k - 1
            assert x == min(u for u in range(g.n) if hit[u] == k)
            assert int(kp[j]) == max([cnt[u] for u in range(g.n) if u != x], default=0)
        gain = 0
        for i in range(l):
            add = reach[x][i] - covered[i]
            gain += len(add)
            covered[i] |= add
        assert int(cov[j]) == gain


def test_permutation_skim_with_large_k_is_exact_greedy():
    g = synth.random_small_graph(10, 30, 55)
    pb = _problem(g, 3, 10 * 3 + 1, 0, 0.4)
    seeds, cov, _, _, _ = oracle.skim_stops(pb, g.n, rank_mode=1)
    ref_seeds, ref_gain = B.exact_greedy(_inst(pb), g.n)
    assert seeds.tolist() == ref_seeds and cov.tolist() == ref_gain


# --------------------------------------------------------------------------
# Estimators
# --------------------------------------------------------------------------

def _single(n, l, k, q):
    """A sketch of node 0 whose k-th smallest position is q."""
    x = np.zeros((n, k), np.uint64)
    x[0, :] = np.arange(q - k + 1, q + 1)
    ln = np.zeros(n, np.uint32)
    ln[0] = k
    return x, ln


def test_permutation_estimators_worked_example():
    # n = 5, l = 4 (D = 20 pairs), k = 3, positions {1, 4, 6}: T - 1 = 6.
    # Node estimator 1 + (k-1)(D-1)/(T-1) = 1 + 2*19/6 = 22/3 pairs, / l;
    # the union form for one set charges its k-1 lower ranks (D-1)/6 each.
    x = np.zeros((5, 3), np.uint64)
    x[0] = [1, 4, 6]
    ln = np.array([3, 0, 0, 0, 0], np.uint32)
    assert oracle.node_estimates(x, ln, 4, rank_mode=1)[0] == pytest.approx(22 / 3 / 4, rel=1e-15)
    assert oracle.union_estimate(x, ln, 4, [0], rank_mode=1) == pytest.approx(2 * 19 / 6 / 4, rel=1e-15)
    # IC model: n (k-1) / (T-1) = 5 * 2 / 6
    assert oracle.node_estimates(x, ln, 4, rank_mode=2)[0] == pytest.approx(10 / 6, rel=1e-15)
    assert oracle.union_estimate(x, ln, 4, [0], rank_mode=2) == pytest.approx(10 / 6, rel=1e-15)


@pytest.mark.parametrize("n,l,k,N", [(5, 4, 3, 7), (6, 2, 4, 10), (8, 3, 2, 5), (10, 1, 2, 10), (7, 3, 5, 6),
                                     (40, 5, 8, 30)])
def test_permutation_estimator_bias_is_between_zero_and_one(n, l, k, N):
    # A set of N of the D = n*l positions, uniformly at random: its k-th
    # smallest position q has P[q] = C(q, k-1) C(D-1-q, N-k) / C(D, N).  In
    # exact arithmetic the printed estimator 1 + (k-1)(D-1)/q averages to
    # between N and N + 1 (N exactly when N = D); the union form without
    # the set-aside element averages to between N - 1 and N.
    D = n * l
    node = Fraction(0)
    union = Fraction(0)
    for q in range(k - 1, D - N + k):
        x, ln = _single(n, l, k, q)
        prob = Fraction(math.comb(q, k - 1) * math.comb(D - 1 - q, N - k), math.comb(D, N))
        node += prob * Fraction(oracle.node_estimates(x, ln, l, rank_mode=1)[0] * l)
        union += prob * Fraction(oracle.union_estimate(x, ln, l, [0], rank_mode=1) * l)
    eps = Fraction(1, 10 ** 9)
    assert N - eps <= node <= N + 1 + eps
    assert N - 1 - eps <= union <= N + eps
    if N == D:
        assert abs(node - N) < eps


def test_estimates_are_exact_when_sketches_are_not_full():
    g = synth.random_small_graph(12, 20, 8)
    pb = _problem(g, 4, 50, 0, 0.3)
    x, ln, _ = oracle.build_sketches(pb, rank_mode=1)
    assert np.all(ln < 50)
    inst = _inst(pb)
    for S in ([0], [1, 2, 3], list(range(12))):
        exact = len(set().union(*[inst.combined_reach(u) for u in S]))
        assert oracle.union_estimate(x, ln, 4, S, rank_mode=1) == pytest.approx(exact / 4, rel=1e-14)
    est = oracle.node_estimates(x, ln, 4, rank_mode=1)
    for u in range(12):
        assert est[u] == pytest.approx(len(inst.combined_reach(u)) / 4, rel=1e-14)


def test_union_estimator_modes_agree_on_their_definitions():
    rng = np.random.default_rng(1)
    n, l, k = 30, 4, 5
    D = n * l
    for _ in range(20):
        ln = rng.integers(1, k + 1, n).astype(np.uint32)
        x = np.zeros((n, k), np.uint64)
        for u in range(n):
            x[u, : ln[u]] = np.sort(rng.choice(D, ln[u], replace=False))
        S = rng.choice(n, 6, replace=False)
        # Eq. unionest with exact rationals: threshold q reads as q / (D - 1)
        best = {}
        for u in S:
            full = ln[u] == k
            thr = Fraction(int(x[u, k - 1]), D - 1) if full else Fraction(1)
            for z in x[u, : (k - 1 if full else ln[u])]:
                z = int(z)
                best[z] = max(best.get(z, Fraction(0)), thr)
        ref = float(sum((1 / t for t in best.values()), Fraction(0)) / l)
        assert oracle.union_estimate(x, ln, l, S, rank_mode=1) == pytest.approx(ref, rel=1e-12)
        # IC mode: l -> infinity.  Threshold q adds n / q; a sketch that is not
        # full has threshold 1, the largest, and 1 / l -> 0 for its ranks.
        best = {}
        for u in S:
            full = ln[u] == k
            thr = int(x[u, k - 1]) if full else None
            for z in x[u, : (k - 1 if full else ln[u])]:
                z = int(z)
                if z in best and best[z] is None:
                    continue
                best[z] = None if thr is None else max(best.get(z, 0), thr)
        ref2 = float(sum((Fraction(n, q) for q in best.values() if q is not None), Fraction(0)))
        assert oracle.union_estimate(x, ln, l, S, rank_mode=2) == pytest.approx(ref2, rel=1e-12)


def _exact_ic_influence(g, p):
    """E |R(u)| under the IC model with edge probability p, by enumerating
    every live-edge subset."""
    m = g.m
    inf = np.zeros(g.n)
    for live in product([0, 1], repeat=m):
        w = p ** sum(live) * (1 - p) ** (m - sum(live))
        adj = [[] for _ in range(g.n)]
        for e in range(m):
            if live[e]:
                adj[int(g.src[e])].append(int(g.dst[e]))
        for u in range(g.n):
            seen, st = {u}, [u]
            while st:
                a = st.pop()
                for b in adj[a]:
                    if b not in seen:
                        seen.add(b)
                        st.append(b)
            inf[u] += w * len(seen)
    return inf


def test_ic_estimator_closed_form_for_sinks():
    # A sink reaches only itself, once per chunk, so its k-th smallest
    # position is (k-1) n + j with j its place in chunk k-1.
    g = synth.star_out(5)  # 0 -> 1..4: nodes 1..4 are sinks
    for seed, k in ((1, 2), (2, 3), (3, 5)):
        pb = _problem(g, 1, k, 0, 0.7, seed=seed)
        x, ln, _ = oracle.build_ic_sketches(pb)
        est = oracle.node_estimates(x, ln, 1, rank_mode=2)
        last = B.ic_nodes(g.n, k, pb.rank_key)[(k - 1) * g.n:]
        for u in range(1, 5):
            j = last.index(u)
            assert est[u] == pytest.approx(g.n * (k - 1) / ((k - 1) * g.n + j), rel=1e-15)


def test_ic_estimator_is_close_to_exact_ic_influence():
    # The chunk structure puts each node once per chunk, so the estimator
    # n(k-1)/(T-1) can sit below the influence by up to about 1/(2(k-1)) of it
    # (the sink case above); with k = 24 that allowance is 2%.
    g = synth.random_small_graph(6, 9, 77)
    p, k, trials = 0.5, 24, 300
    exact = _exact_ic_influence(g, p)
    acc = np.zeros(g.n)
    sq = np.zeros(g.n)
    for t in range(trials):
        pb = _problem(g, 1, k, 0, p, seed=1000 + t)
        x, ln, _ = oracle.build_ic_sketches(pb)
        e = oracle.node_estimates(x, ln, 1, rank_mode=2)
        acc += e
        sq += e * e
    mean = acc / trials
    se = np.sqrt(np.maximum(sq / trials - mean ** 2, 1e-12) / trials)
    assert np.all(np.abs(mean - exact) <= 4 * se + exact / (2 * (k - 1))), (mean, exact, se)

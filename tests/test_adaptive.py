"""Adaptive error estimation (Section 4.3.2).

Pins of the oracle against things other than itself:
  - the threshold rank and k' recorded by oracle SKIM against a brute-force
    recount of every partial sketch from explicit reachability
    (tests/_brute.py);
  - the Chernoff tail of Eq. chernoff against the exponential-moment bound
    minimised numerically, and against exact binomial tails, which it must
    never undercut;
  - the discretisation and convolution against sampling;
  - the bound against exact greedy discrepancies on small graphs;
and the library's host implementation against the oracle.  CPU only.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import _brute as B
import oracle
import synth
from oracle import discrepancy as D


def _problem(g, l, k, model=0, p=0.3, seed=7):
    ks = synth.Keys.from_seed(seed)
    return oracle.Problem(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_stop_rank_and_kprime_match_brute_force(seed):
    g = synth.random_small_graph(16, 50, 300 + seed)
    l, k = 3, 2 + seed % 3
    pb = _problem(g, l, k, seed % 2, 0.35, seed=seed)
    inst = B.Instances(pb.n, pb.src, pb.dst, l, pb.model, pb.p, pb.coin_key, pb.prob_key)
    reach = [[inst.reach(u, i) for i in range(l)] for u in range(g.n)]
    rank = {(v, i): B.rank(pb.rank_key, l, v, i) for v in range(g.n) for i in range(l)}
    s = g.n
    seeds, cov, tau, kp, _ = oracle.skim_stops(pb, s)
    covered = [set() for _ in range(l)]
    for j in range(s):
        x = int(seeds[j])
        uncovered = [(v, i) for (v, i) in rank if v not in covered[i]]
        if kp[j] < 0:
            # the ranks ran out: no node reaches k uncovered pairs
            assert int(tau[j]) == 0
            for u in range(g.n):
                assert sum(1 for (v, i) in uncovered if v in reach[u][i]) < k
        else:
            t = int(tau[j])
            stop = [(v, i) for (v, i) in uncovered if rank[(v, i)] == t]
            assert len(stop) == 1 and stop[0][0] in reach[x][stop[0][1]]

            def count(u):  # uncovered pairs ranked below tau that u reaches
                return sum(1 for (v, i) in uncovered if rank[(v, i)] < t and v in reach[u][i])

            cnt = [count(u) for u in range(g.n)]
            assert max(cnt) <= k - 1
            hit = [cnt[u] + (stop[0][0] in reach[u][stop[0][1]]) for u in range(g.n)]
            assert x == min(u for u in range(g.n) if hit[u] == k)
            assert int(kp[j]) == max([cnt[u] for u in range(g.n) if u != x], default=0)
        gain = 0
        for i in range(l):
            add = reach[x][i] - covered[i]
            gain += len(add)
            covered[i] |= add
        assert int(cov[j]) == gain


@pytest.mark.parametrize("kp", [0, 1, 3, 10, 63])
def test_chernoff_tail_is_the_optimised_moment_bound(kp):
    # For a sum Z of independent Bernoulli trials with mean mu,
    # P[Z <= k'] <= min_t exp(t k') E[exp(-t Z)] <= min_t exp(t k' + mu (e^-t - 1)).
    from scipy.optimize import minimize_scalar
    for mu in (kp + 0.5, kp * 1.3 + 1, 2.0 * kp + 4, 5.0 * kp + 20):
        f = minimize_scalar(lambda t: t * kp + mu * (math.exp(-t) - 1.0), bounds=(0.0, 60.0),
                            method="bounded", options={"xatol": 1e-12})
        assert D.chernoff_tail(kp, mu) == pytest.approx(math.exp(f.fun), rel=1e-7)
    assert D.chernoff_tail(kp, float(kp)) == 1.0
    assert D.chernoff_tail(kp, kp * 0.5) == 1.0


def test_chernoff_tail_never_undercuts_exact_binomial_tails():
    from scipy.stats import binom, poisson
    rng = np.random.default_rng(4)
    for _ in range(300):
        n = int(rng.integers(5, 5000))
        p = float(rng.uniform(1e-3, 0.5))
        mu = n * p
        kp = int(rng.integers(0, max(1, int(mu))))
        b = D.chernoff_tail(kp, mu)
        assert b >= binom.cdf(kp, n, p) * (1 - 1e-12)
        assert b >= poisson.cdf(kp, mu) * (1 - 1e-12)
    assert D.chernoff_tail(0, 3.0) == pytest.approx(poisson.pmf(0, 3.0), rel=1e-14)


def test_single_iteration_ccdf_is_its_tail_on_the_grid():
    delta, tau, kp, h, bins = 5000, 1 << 55, 40, 37.0, 300
    ccdf = D.discrepancy_ccdf([delta], [tau], [kp], h, bins)
    t = math.ldexp(float(tau), -64)
    for i in range(bins):
        assert ccdf[i] == pytest.approx(D.chernoff_tail(kp, t * (delta + i * h)), rel=1e-9, abs=1e-300)
    assert ccdf[bins] == pytest.approx(D.chernoff_tail(kp, t * (delta + (bins - 1) * h)), rel=1e-12)
    exact = D.discrepancy_ccdf([delta, 77, 1234], [tau, 0, 0], [kp, -1, -1], h, bins)
    assert np.allclose(exact, ccdf, rtol=1e-12, atol=0)  # exact selections add nothing
    assert np.all(D.discrepancy_ccdf([9, 9], [0, 0], [-1, -1], 1.0, 10) == 0.0)


def test_convolution_matches_sampling():
    # four iterations of a SKIM-like run: tau * delta near k - 1 = 31
    its = [(4000, 31.0 / 4000, 27), (2500, 31.0 / 2400, 30), (900, 31.0 / 950, 25), (300, 31.0 / 300, 29)]
    delta = [a for a, _, _ in its]
    tau = [int(math.ldexp(t, 64)) for _, t, _ in its]
    kp = [c for _, _, c in its]
    rng = np.random.default_rng(12)
    N = 200_000
    # a wide grid, and a narrow one whose last cell the sum often overruns
    for h, bins, probe in ((25.0, 400, (0, 3, 10, 30, 80, 150)), (25.0, 40, (0, 10, 25, 39, 40))):
        ccdf = D.discrepancy_ccdf(delta, tau, kp, h, bins)
        total = np.zeros(N)
        for d, t, c in zip(delta, tau, kp):
            tt = math.ldexp(float(t), -64)
            grid = np.array([D.chernoff_tail(c, tt * (d + i * h)) for i in range(bins)])
            u = rng.random(N)
            # the grid variable exceeds i*h exactly when u < B(i h)
            cells = (u[:, None] < grid[None, :]).sum(axis=1)
            val = cells * h
            val[cells == bins] = np.inf
            total += val
        total[total >= bins * h] = np.inf  # a sum past the last cell is overflow
        for i in probe:
            emp = float((total > i * h).mean()) if i < bins else float(np.isinf(total).mean())
            sd = math.sqrt(max(ccdf[i] * (1 - ccdf[i]), 1.0 / N) / N)
            assert abs(emp - ccdf[i]) <= 5 * sd + 1e-12, (bins, i, emp, ccdf[i])
        assert ccdf[bins] > 0.01 or bins == 400


def test_bound_holds_against_exact_greedy_discrepancies():
    # The gap between the largest exact marginal gain and SKIM's choice, summed
    # over the iterations, should rarely exceed the 90% bound.
    trials, over, finite = 24, 0, 0
    for t in range(trials):
        g = synth.random_small_graph(90, 420, 500 + t)
        pb = _problem(g, 6, 6, 0, 0.2, seed=500 + t)
        s = 5
        seeds, cov, tau, kp, _ = oracle.skim_stops(pb, s)
        gap = 0
        for j in range(s):
            base = int(oracle.exact_coverage(pb, seeds[:j])[-1]) if j else 0
            best = max(int(oracle.exact_coverage(pb, np.append(seeds[:j], v).astype(np.uint32))[-1]) - base
                       for v in range(g.n))
            assert best >= int(cov[j])
            gap += best - int(cov[j])
        b90 = D.discrepancy_bound(cov, tau, kp, 1.0, 4 * int(cov.sum()) + 64, [0.9])[0]
        finite += math.isfinite(b90)
        over += gap > b90
    assert finite >= trials // 2
    assert over <= 0.1 * trials + 3 * math.sqrt(0.09 * trials)


def test_library_bound_matches_oracle():
    import paper_1408_6282_gb300 as pkg
    g = synth.random_small_graph(2000, 12000, 61)
    pb = _problem(g, 16, 16, 1, 0.0, seed=61)
    seeds, cov, tau, kp, _ = oracle.skim_stops(pb, 30)
    for step, bins in ((float(cov.sum()) / 512, 2048), (1.0, 700)):
        conf = [0.5, 0.9, 0.99]
        got, ccdf = pkg.discrepancy_bound(cov, tau, kp, step, bins, conf)
        ref = D.discrepancy_ccdf(cov, tau, kp, step, bins)
        assert np.allclose(ccdf, ref, rtol=1e-9, atol=1e-15)
        want = D.discrepancy_bound(cov, tau, kp, step, bins, conf)
        for a, b in zip(got, want):
            assert a == b or (math.isfinite(a) and abs(a - b) <= step)
    # no iterations: the sum is 0 with certainty
    got, ccdf = pkg.discrepancy_bound([], [], [], 1.0, 8, [0.9])
    assert got[0] == 0.0 and np.all(ccdf == 0.0)


def test_library_bound_rejects_bad_arguments():
    import paper_1408_6282_gb300 as pkg
    one = ([10], [1 << 60], [3])
    for kw in (dict(step=0.0), dict(step=math.inf), dict(bins=0), dict(conf=[1.0]), dict(conf=[0.0])):
        args = dict(step=1.0, bins=16, conf=[0.9])
        args.update(kw)
        with pytest.raises(pkg.SkimError) as e:
            pkg.discrepancy_bound(*one, **args)
        assert e.value.code == -1
    with pytest.raises(pkg.SkimError):
        pkg.discrepancy_bound([10], [1], [-2], 1.0, 16, [0.9])

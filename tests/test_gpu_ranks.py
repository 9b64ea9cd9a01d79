"""GPU path vs the oracle for structured permutation ranks (Section 3.1) and
IC-model sketches (Section 3.2): sketches, SKIM records and node estimates bit
for bit, union estimates within 1e-12 relative."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
REL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import paper_1408_6282_gb300 as p
    from paper_1408_6282_gb300 import build as b
    b.build()
    p.load()
    return p


def _close(a, b):
    return abs(a - b) <= REL * max(abs(a), abs(b)) or (a == 0 and b == 0)


def _pair(pkg, g, l, k, model, p, seed, mode, bl=0):
    ks = synth.Keys.from_seed(seed)
    pb = oracle.Problem(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob)
    sk = pkg.Skim(g.n, g.src, g.dst, l, k, model, p, ks.coin, ks.rank, ks.prob, batch_lanes=bl, rank_mode=mode)
    return pb, sk


GRAPHS = [
    ("chain", lambda: synth.chain(40)),
    ("star", lambda: synth.star_out(50)),
    ("clique", lambda: synth.clique(9)),
    ("single", lambda: synth.empty_graph(1)),
    ("er_sparse", lambda: synth.random_small_graph(300, 900, 3)),
    ("er_dense", lambda: synth.random_small_graph(120, 3000, 4)),
    ("rmat10", lambda: synth.rmat(10, 8, 99)),
]
PERM = [(1, 2, 0, 0.5, 0), (3, 4, 0, 0.3, 64), (16, 16, 0, 0.1, 0), (64, 8, 1, 0.0, 0), (64, 64, 1, 0.0, 128),
        (7, 5, 2, 0.0, 0), (4, 40, 0, 0.6, 0)]


def _queries(n, seeds):
    rng = np.random.default_rng(5)
    return [[], [0], list(seeds[:3]), rng.integers(0, n, 10).tolist(), list(range(n))]


@pytest.mark.parametrize("name,mk", GRAPHS)
@pytest.mark.parametrize("l,k,model,p,bl", PERM)
def test_permutation_ranks(pkg, name, mk, l, k, model, p, bl):
    g = mk()
    pb, sk = _pair(pkg, g, l, k, model, p, 13, pkg.RANKS_PERMUTATION, bl)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_sketches(pb, rank_mode=1)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        assert np.array_equal(sk.node_estimates(), oracle.node_estimates(ox, oln, l, rank_mode=1))
        s = min(g.n, 25)
        seeds, cov, tau, kp = sk.greedy_stops(s)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, s, rank_mode=1)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)
        sets = _queries(g.n, seeds)
        single = [sk.query(q) for q in sets]
        batch = sk.query_batch(sets)
        for q, a, b in zip(sets, single, batch):
            assert a == b
            assert _close(a, oracle.union_estimate(ox, oln, l, q, rank_mode=1))


@pytest.mark.parametrize("name,mk", GRAPHS)
@pytest.mark.parametrize("k,model,p,bl", [(2, 0, 0.5, 0), (4, 0, 0.3, 64), (16, 1, 0.0, 0), (8, 2, 0.0, 256),
                                          (32, 0, 0.1, 0)])
def test_ic_model_sketches(pkg, name, mk, k, model, p, bl):
    g = mk()
    pb, sk = _pair(pkg, g, 1, k, model, p, 17, pkg.RANKS_IC_MODEL, bl)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_ic_sketches(pb)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        assert np.array_equal(sk.node_estimates(), oracle.node_estimates(ox, oln, 1, rank_mode=2))
        sets = _queries(g.n, [v for v in (0, 1, 2) if v < g.n])
        for q, a in zip(sets, sk.query_batch(sets)):
            assert _close(float(a), oracle.union_estimate(ox, oln, 1, q, rank_mode=2))
        with pytest.raises(pkg.SkimError) as e:
            sk.greedy(1)  # IC-model SKIM is not built
        assert e.value.code == -1


def test_permutation_full_run_and_uniform_modes_differ(pkg):
    g = synth.random_small_graph(200, 1200, 8)
    pb, sk = _pair(pkg, g, 8, 6, 1, 0.0, 21, pkg.RANKS_PERMUTATION, 0)
    with sk:
        seeds, cov, tau, kp = sk.greedy_stops(g.n)  # to exhaustion
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, g.n, rank_mode=1)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)
        assert sorted(seeds.tolist()) == list(range(g.n))
    # the uniform-rank run of the same keys takes another order
    useeds, _, _, _, _ = oracle.skim_stops(pb, 10)
    assert not np.array_equal(useeds, os_[:10])


@pytest.mark.parametrize("scale,k", [(12, 16), (13, 8)])
def test_ic_model_rmat(pkg, scale, k):
    ks = synth.Keys.from_seed(60 + scale)
    g = synth.rmat(scale, 16, ks.graph)
    pb, sk = _pair(pkg, g, 1, k, 1, 0.0, 60 + scale, pkg.RANKS_IC_MODEL)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_ic_sketches(pb)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)


@pytest.mark.parametrize("scale", [12, 13])
def test_permutation_rmat(pkg, scale):
    ks = synth.Keys.from_seed(80 + scale)
    g = synth.rmat(scale, 16, ks.graph)
    pb, sk = _pair(pkg, g, 64, 32, 1, 0.0, 80 + scale, pkg.RANKS_PERMUTATION)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        ox, oln, _ = oracle.build_sketches(pb, rank_mode=1)
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov, tau, kp = sk.greedy_stops(30)
        os_, oc, otau, okp, _ = oracle.skim_stops(pb, 30, rank_mode=1)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        assert np.array_equal(tau, otau) and np.array_equal(kp, okp)

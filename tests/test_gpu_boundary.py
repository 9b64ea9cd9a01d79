"""The C ABI's smaller calls on the GPU: the per-node sketch read, the device
wait limit (made to run out on purpose in a build and in SKIM: the search
gives up, returns SKIM_ETIMEOUT, and a fresh context then builds correct
sketches), and the server's host-side wait timeout."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1408_6282_gb300 as p
    from paper_1408_6282_gb300 import build as b
    b.build()
    p.load()
    return p


def test_get_sketch_rows_match_oracle(pkg):
    w = synth.WORKLOADS["er4096"]
    g = w.graph()
    ks = w.keys()
    pb = oracle.Problem(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob)
    ox, oln, _ = oracle.build_sketches(pb)
    with pkg.Skim(g.n, g.src, g.dst, w.l, w.k, w.prob_model, w.p, ks.coin, ks.rank, ks.prob) as sk:
        with pytest.raises(pkg.SkimError) as e:
            sk.sketch(0)
        assert e.value.code == -3  # not built
        sk.build_sketches()
        for v in (0, 1, 17, g.n // 2, g.n - 1):
            assert np.array_equal(sk.sketch(v), ox[v, : oln[v]]), v
        with pytest.raises(pkg.SkimError) as e:
            sk.sketch(g.n)
        assert e.value.code == -1
    # a node with a short sketch: a sink of a chain reaches only itself
    g = synth.chain(10)
    pb = oracle.Problem(g.n, g.src, g.dst, 4, 8, 0, 1.0, 1, 2, 3)
    ox, oln, _ = oracle.build_sketches(pb)
    with pkg.Skim(g.n, g.src, g.dst, 4, 8, 0, 1.0, 1, 2, 3) as sk:
        sk.build_sketches()
        for v in range(g.n):
            got = sk.sketch(v)
            assert got.shape[0] == oln[v] and np.array_equal(got, ox[v, : oln[v]])


def test_wait_limit_runs_out_then_a_fresh_context_is_correct(pkg):
    """A 1 ns wait limit: on a long live chain one warp walks the search while
    the others wait for it, see no progress and give up.  Every warp returns,
    the call reports SKIM_ETIMEOUT, the context refuses further work, and a
    new context on the same device builds the oracle's sketches."""
    g = synth.chain(60000)
    with pkg.Skim(g.n, g.src, g.dst, 1, 2, 0, 1.0, 5, 6, 7, batch_lanes=64) as sk:
        sk.set_wait_limit_ns(1)
        with pytest.raises(pkg.SkimError) as e:
            sk.build_sketches()
        assert e.value.code == -4
        with pytest.raises(pkg.SkimError) as e:
            sk.build_sketches()
        assert e.value.code == -5  # unusable after a timeout
    g = synth.random_small_graph(2000, 12000, 9)
    pb = oracle.Problem(g.n, g.src, g.dst, 8, 8, 0, 0.2, 5, 6, 7)
    ox, oln, _ = oracle.build_sketches(pb)
    with pkg.Skim(g.n, g.src, g.dst, 8, 8, 0, 0.2, 5, 6, 7) as sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        assert np.array_equal(ln, oln) and np.array_equal(x, ox)
        seeds, cov = sk.greedy(5)
        os_, oc, _, _ = oracle.skim(pb, 5)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)


def test_wait_limit_runs_out_during_skim(pkg):
    """The wait limit bounds SKIM's searches too.  Two seeds taken with the
    default limit match the oracle; with a 1 ns limit the next seed's search
    (the residual search of the last seed, finished at the next read-back, or
    the reverse search of a new batch) gives up, the call reports SKIM_ETIMEOUT
    and the context refuses further work."""
    g = synth.random_small_graph(2000, 12000, 9)
    pb = oracle.Problem(g.n, g.src, g.dst, 8, 8, 0, 0.2, 5, 6, 7)
    os_, oc, _, _ = oracle.skim(pb, 2)
    with pkg.Skim(g.n, g.src, g.dst, 8, 8, 0, 0.2, 5, 6, 7) as sk:
        seeds, cov = sk.greedy(2)
        assert np.array_equal(seeds, os_) and np.array_equal(cov, oc)
        sk.set_wait_limit_ns(1)
        with pytest.raises(pkg.SkimError) as e:
            sk.greedy(3)
        assert e.value.code == -4
        with pytest.raises(pkg.SkimError) as e:
            sk.greedy(1)
        assert e.value.code == -5


def test_server_wait_times_out_and_server_keeps_serving(pkg):
    g = synth.random_small_graph(3000, 20000, 12)
    with pkg.Skim(g.n, g.src, g.dst, 16, 16, 0, 0.1, 1, 2, 3) as sk:
        sk.build_sketches()
        with sk.server(max_inflight=64, scratch_slots=1 << 16, streams=2) as srv:
            with pytest.raises(pkg.SkimError) as e:
                srv.wait(123456789, timeout_ms=20)  # a ticket nothing will complete
            assert e.value.code == -4
            q = np.arange(0, g.n, 11, dtype=np.uint32)
            t = srv.submit(q)
            assert srv.wait(t, timeout_ms=60000) == sk.query(q)

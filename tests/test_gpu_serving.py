"""The continuous-batching query server: every result is bitwise the same as
the single-query call, whatever group, stream or arrival pattern it met."""
import threading

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    import paper_1408_6282_gb300 as pkg
    from paper_1408_6282_gb300 import build as b
    b.build()
    ks = synth.Keys.from_seed(77)
    g = synth.rmat(14, 16, ks.graph)
    s = pkg.Skim(g.n, g.src, g.dst, 64, 32, 1, 0.0, ks.coin, ks.rank, ks.prob)
    s.build_sketches()
    yield s
    s.close()


def _queries(n, count, key):
    sizes = synth.query_sizes(count, key, max_size=400)
    return [synth.uniform_seed_set(n, int(z), key, q) for q, z in enumerate(sizes)]


def test_results_equal_single_query_under_queueing(sk):
    qs = _queries(sk.n, 300, 5) + [np.zeros(0, np.uint32), np.array([3, 3, 3], np.uint32)]
    ref = [sk.query(q) for q in qs]
    # tiny pool: few slots and little scratch, so requests wait for each other
    with sk.server(max_inflight=8, scratch_slots=1 << 17, streams=2) as srv:
        tickets = [srv.submit(q) for q in qs]
        got = [srv.wait(t) for t in tickets]
        groups, queries = srv.stats()
    assert got == ref
    assert queries == len(qs) and groups < len(qs)


def test_replay_burst_and_poisson(sk):
    qs = _queries(sk.n, 400, 9)
    ref = np.array([sk.query(q) for q in qs])
    with sk.server(max_inflight=256, scratch_slots=1 << 22, streams=4) as srv:
        lat, est = srv.replay(np.zeros(len(qs)), qs)  # everything at once
        assert np.array_equal(est, ref)
        assert np.all(lat > 0)
        arr = synth.poisson_arrivals(len(qs), 20000.0, 9)
        lat2, est2 = srv.replay(arr, qs)
        assert np.array_equal(est2, ref)
        assert np.all(lat2 > 0)


def test_submit_from_several_threads_and_poll(sk):
    qs = _queries(sk.n, 240, 13)
    ref = [sk.query(q) for q in qs]
    out = [None] * len(qs)
    with sk.server(max_inflight=64, scratch_slots=1 << 20, streams=3) as srv:
        def worker(lo):
            ts = [(i, srv.submit(qs[i])) for i in range(lo, len(qs), 4)]
            for i, t in ts:
                while True:
                    done, e = srv.poll(t)
                    if done:
                        out[i] = e
                        break
        th = [threading.Thread(target=worker, args=(j,)) for j in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    assert out == ref


def test_too_large_for_scratch_is_rejected(sk):
    import paper_1408_6282_gb300 as pkg
    with sk.server(max_inflight=4, scratch_slots=1 << 12, streams=1) as srv:
        with pytest.raises(pkg.SkimError) as e:
            srv.submit(np.arange(200, dtype=np.uint32))
        assert e.value.code == -7
        with pytest.raises(pkg.SkimError) as e:
            srv.submit(np.array([sk.n], np.uint32))
        assert e.value.code == -1
        t = srv.submit(np.array([1, 2], np.uint32))
        assert srv.wait(t) == sk.query([1, 2])

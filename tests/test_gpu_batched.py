"""Many graphs in one context: every graph's slice of the sketches equals the
oracle's sketches of that graph alone (its own keys and probability model)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graphs(count, seed):
    ks = synth.Keys.from_seed(seed)
    h = synth.stream(ks.graph, 4 * count)
    out = []
    for g in range(count):
        scale = 6 + int(h[4 * g] % np.uint64(5))
        ef = 4 + int(h[4 * g + 1] % np.uint64(12))
        gr = synth.rmat(scale, ef, int(h[4 * g + 2]))
        model = int(h[4 * g + 3] % np.uint64(3))
        out.append((gr, model, 0.05 + 0.1 * (g % 3)))
    return out


@pytest.mark.parametrize("bl", [0, 256])
def test_batch_matches_each_graph_alone(bl):
    import paper_1408_6282_gb300 as pkg
    from paper_1408_6282_gb300 import build as b
    b.build()
    gs = _graphs(12, 31)
    l, k = 16, 8
    keys = [synth.Keys.from_seed(100 + g) for g in range(len(gs))]
    sk = pkg.Skim.batch([(gr.n, gr.src, gr.dst) for gr, _, _ in gs], l, k, [m for _, m, _ in gs],
                        [p for _, _, p in gs], [kk.coin for kk in keys], [kk.rank for kk in keys],
                        [kk.prob for kk in keys], batch_lanes=bl)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        for g, ((gr, model, p), kk) in enumerate(zip(gs, keys)):
            pb = oracle.Problem(gr.n, gr.src, gr.dst, l, k, model, p, kk.coin, kk.rank, kk.prob)
            ox, oln, _ = oracle.build_sketches(pb)
            o = sk.offsets[g]
            assert np.array_equal(ln[o:o + gr.n], oln), g
            assert np.array_equal(x[o:o + gr.n], ox), g
            # a query inside graph g uses union ids
            q = np.arange(0, gr.n, 5, dtype=np.uint32)
            ref = oracle.union_estimate(ox, oln, l, q)
            assert abs(sk.query(q + o) - ref) <= 1e-12 * max(1.0, abs(ref))
        with pytest.raises(pkg.SkimError):
            sk.greedy(1)
        best, secs = sk.autotune([64, 1024, 1 << 16])
        assert best in (64, 1024, 1 << 16) and np.all(secs > 0)
        sk.build_sketches()
        x2, ln2 = sk.sketches()
        assert np.array_equal(x2, x) and np.array_equal(ln2, ln)
        # the autotuner over whole settings (lanes, queue switch, record order)
        grid = [(256, 0.0, 4), (1024, 8.0, 1), (4096, 1e9, 1 << 20)]
        bi, secs = sk.autotune_settings(grid)
        assert 0 <= bi < len(grid) and np.all(secs > 0)
        assert tuple(sk.tuning().values()) == grid[bi]
        sk.build_sketches()
        x3, ln3 = sk.sketches()
        assert np.array_equal(x3, x) and np.array_equal(ln3, ln)


def _digest(x, ln):
    import hashlib
    x = np.array(x, dtype=np.uint64, copy=True)
    k = x.shape[1]
    x[np.arange(k)[None, :] >= ln[:, None].astype(np.int64)] = 0
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ln, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(x, dtype="<u8").tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("bl", [0, 1 << 20])
def test_batched256_trivalency_matches_oracle(bl):
    """The many-graph workload at its own size: 256 R-MAT graphs (scale 10..16,
    edge factor 8..32, about 4.7M nodes and 79M edges in all), trivalency
    probabilities, l = 64, k = 32, in one context.  Batches of 2M (default)
    and 1M lanes hold tens of millions of visit records, so the records are
    placed node by node.  Every graph's slice of the sketches must hash to the
    digest the oracle stored for that graph built alone."""
    import json
    import os

    import paper_1408_6282_gb300 as pkg
    from paper_1408_6282_gb300 import build as b
    b.build()
    path = os.path.join(os.path.dirname(__file__), "golden", "batched256_trivalency.json")
    gold = json.load(open(path))
    specs = synth.batched_graph_specs(256)
    gl = [synth.rmat(sc, ef, key, device="cuda") for sc, ef, key in specs]
    for gr, gg, (sc, ef, key) in zip(gl, gold["per_graph"], specs):
        assert (gg["scale"], gg["edge_factor"], int(gg["key"])) == (sc, ef, key)
        assert gr.digest() == gg["graph_sha256"]
    keys = [synth.Keys.from_seed(key) for _, _, key in specs]
    sk = pkg.Skim.batch([(gr.n, gr.src, gr.dst) for gr in gl], gold["l"], gold["k"], [gold["prob_model"]] * 256,
                        [0.0] * 256, [kk.coin for kk in keys], [kk.rank for kk in keys], [kk.prob for kk in keys],
                        batch_lanes=bl)
    with sk:
        sk.build_sketches()
        x, ln = sk.sketches()
        bad = [g for g, gg in enumerate(gold["per_graph"])
               if _digest(x[sk.offsets[g]:sk.offsets[g + 1]], ln[sk.offsets[g]:sk.offsets[g + 1]]) != gg["sketch_sha256"]]
        assert not bad, bad

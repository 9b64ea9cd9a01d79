"""The allocation-free query entry point (skim_union_estimate_static).

It exists for callers that cannot allocate device memory: code that runs
inside another framework's memory pool, or under a fixed memory budget where a
cudaMalloc is not allowed.  Its scratch table is static device memory instead.
It must give the oracle's estimate (Eq. unionest) on the same sketches, call
after call, under each rank reading, whether this file runs alone in a fresh
process or after every other test.  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _static(pkg, x_dev, len_dev, n, k, l, s, out, stream, rank_mode):
    import torch
    seeds_d = torch.from_numpy(s.view(np.int32)).cuda() if s.size else None
    got = []
    for _ in range(2):  # two calls in a row share (and re-clear) the static table
        out.fill_(-1.0)
        pkg.skim_union_estimate_static(x_dev, len_dev, n, k, l, seeds_d.data_ptr() if seeds_d is not None else 0,
                                       int(s.size), out.data_ptr(), stream.cuda_stream, rank_mode=rank_mode)
        stream.synchronize()
        got.append(float(out.item()))
    return got


@pytest.mark.parametrize("rank_mode", [0, 1, 2])
def test_static_query_matches_oracle_and_ordinary_query_twice(rank_mode):
    import torch

    import paper_1408_6282_gb300 as pkg
    from paper_1408_6282_gb300 import build as b
    b.build()
    g = synth.random_small_graph(3000, 24000, 29)
    ks = synth.Keys.from_seed(29)
    l, k = (1, 32) if rank_mode == 2 else (16, 32)
    stream = torch.cuda.current_stream()
    pb = oracle.Problem(g.n, g.src, g.dst, l, k, 0, 0.15, ks.coin, ks.rank, ks.prob)
    if rank_mode == 2:
        ox, oln, _ = oracle.build_ic_sketches(pb)
    else:
        ox, oln, _ = oracle.build_sketches(pb, rank_mode=rank_mode)
    with pkg.Skim(g.n, g.src, g.dst, l, k, 0, 0.15, ks.coin, ks.rank, ks.prob, stream=stream.cuda_stream,
                  rank_mode=rank_mode) as sk:
        sk.build_sketches()
        x_dev, len_dev = pkg.skim_sketch_pointers(sk.ctx)
        rng = np.random.default_rng(11)
        sets = [np.zeros(0, np.uint32), np.array([5], np.uint32), np.array([7, 7, 8], np.uint32),
                rng.choice(g.n, 300, replace=False).astype(np.uint32),
                rng.choice(g.n, 2000, replace=False).astype(np.uint32)]
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        for s in sets:
            ref = oracle.union_estimate(ox, oln, l, s, rank_mode=rank_mode)
            ordinary = sk.query(s)
            for v in _static(pkg, x_dev, len_dev, g.n, k, l, s, out, stream, rank_mode):
                assert abs(v - ref) <= 1e-12 * max(abs(ref), 1.0), (s.size, v, ref)
                assert v == ordinary, (s.size, v, ordinary)  # both sums are exact and rounded once
        # beyond the static table: rejected with SKIM_ERANGE, nothing launched
        big = torch.zeros(5000, dtype=torch.int32, device="cuda")
        with pytest.raises(pkg.SkimError) as e:
            pkg.skim_union_estimate_static(x_dev, len_dev, g.n, k, l, big.data_ptr(), 5000, out.data_ptr(),
                                           stream.cuda_stream, rank_mode=rank_mode)
        assert e.value.code == -7
        # an id >= n gives a quiet NaN, asynchronously
        bad = torch.tensor([1, g.n + 3], dtype=torch.int32, device="cuda")
        pkg.skim_union_estimate_static(x_dev, len_dev, g.n, k, l, bad.data_ptr(), 2, out.data_ptr(),
                                       stream.cuda_stream, rank_mode=rank_mode)
        stream.synchronize()
        assert np.isnan(out.item())
        # a rank reading the sketches cannot have: rejected before any launch
        with pytest.raises(pkg.SkimError) as e:
            pkg.skim_union_estimate_static(x_dev, len_dev, g.n, k, l, 0, 0, out.data_ptr(), stream.cuda_stream,
                                           rank_mode=3)
        assert e.value.code == -1

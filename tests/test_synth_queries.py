"""Input generators for queries (no method arithmetic): the uniform seed sets
and the neighbourhood generator of Section 6.2.  CPU only."""
from collections import deque

import numpy as np

import synth


def _dist(n, src, dst, root):
    adj = [[] for _ in range(n)]
    for a, b in zip(src.tolist(), dst.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    d = {root: 0}
    q = deque([root])
    while q:
        a = q.popleft()
        for b in adj[a]:
            if b not in d:
                d[b] = d[a] + 1
                q.append(b)
    return d


def test_neighborhood_sets_are_balls_of_minimal_radius():
    g = synth.rmat(10, 8, 5)
    for qid, size in enumerate((1, 5, 50, 300)):
        s, radius = synth.neighborhood_seed_set(g.n, g.src, g.dst, size, 77, qid)
        assert len(s) == len(set(s.tolist())) == size
        # some node reaches every seed within `radius` undirected hops, and
        # the ball of radius - 1 around it is smaller than `size`
        ok = False
        for root in set(g.src.tolist()) | set(g.dst.tolist()):
            d = _dist(g.n, g.src, g.dst, root)
            if all(int(v) in d and d[int(v)] <= radius for v in s):
                if radius == 0 or sum(1 for x in d.values() if x <= radius - 1) < size:
                    ok = True
                    break
        assert ok, (qid, size, radius)


def test_neighborhood_small_component_and_determinism():
    g = synth.chain(4)  # 0 -> 1 -> 2 -> 3: one component of 4 nodes
    s, radius = synth.neighborhood_seed_set(g.n, g.src, g.dst, 10, 3, 0)
    assert sorted(s.tolist()) == [0, 1, 2, 3]
    a, ra = synth.neighborhood_seed_set(g.n, g.src, g.dst, 2, 9, 4)
    b, rb = synth.neighborhood_seed_set(g.n, g.src, g.dst, 2, 9, 4)
    assert np.array_equal(a, b) and ra == rb


def test_root_is_degree_proportional():
    # a star: the centre holds half of all edge ends
    g = synth.star_out(41)
    hits = 0
    for q in range(2000):
        s, r = synth.neighborhood_seed_set(g.n, g.src, g.dst, 1, 5, q)
        hits += r == 0 and int(s[0]) == 0
    assert abs(hits / 2000 - 0.5) < 0.05

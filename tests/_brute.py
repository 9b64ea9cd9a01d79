"""Brute-force references for tiny graphs, written independently of oracle/.

Pure Python, big-integer arithmetic, explicit per-instance BFS.  Used only to
pin the oracle (and, through it, the GPU path) on inputs small enough to
enumerate every node-instance pair.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction

M64 = (1 << 64) - 1
G = 0x9E3779B97F4A7C15


def fmix(z: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    z &= M64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def rank(rank_key: int, l: int, v: int, i: int) -> int:
    return fmix(rank_key + G * (v * l + i))


def threshold(model: int, p: float, indeg_v: int, u: int, v: int, prob_key: int) -> int:
    """Largest coin value that makes edge (u,v) live."""
    def unif(q):
        if q >= 1.0:
            return M64
        # floor(q * 2^64) for a double q: exact via its integer ratio
        a, b = Fraction(q).as_integer_ratio()
        return (a << 64) // b - 1
    if model == 0:
        return unif(p)
    if model == 1:
        return M64 // indeg_v
    cls = fmix(prob_key ^ ((u << 32) | v)) % 3
    return unif((0.1, 0.01, 0.001)[cls])


class Instances:
    """All l live-edge instances of a small graph, materialised."""

    def __init__(self, n, src, dst, l, model, p, coin_key, prob_key=0):
        self.n, self.l = n, l
        indeg = [0] * n
        for v in dst:
            indeg[int(v)] += 1
        self.out = [[[] for _ in range(n)] for _ in range(l)]
        for u, v in zip(src, dst):
            u, v = int(u), int(v)
            he = fmix(coin_key ^ ((u << 32) | v))
            t = threshold(model, p, indeg[v], u, v, prob_key)
            for i in range(l):
                if fmix(he + G * (i + 1)) <= t:
                    self.out[i][u].append(v)

    def reach(self, u: int, i: int, blocked=None) -> set[int]:
        """Nodes reachable from u in instance i (u included), never entering
        a node in `blocked`."""
        if blocked and u in blocked:
            return set()
        seen = {u}
        q = deque([u])
        while q:
            x = q.popleft()
            for y in self.out[i][x]:
                if y not in seen and not (blocked and y in blocked):
                    seen.add(y)
                    q.append(y)
        return seen

    def combined_reach(self, u: int) -> set[tuple[int, int]]:
        return {(v, i) for i in range(self.l) for v in self.reach(u, i)}

    def coverage(self, seeds) -> int:
        tot = 0
        for i in range(self.l):
            cov = set()
            for s in seeds:
                cov |= self.reach(int(s), i)
            tot += len(cov)
        return tot


def sketch(inst: Instances, u: int, k: int, rank_key: int) -> list[int]:
    """X_u: the k smallest ranks over the combined reachability set R_u."""
    rs = sorted(rank(rank_key, inst.l, v, i) for (v, i) in inst.combined_reach(u))
    return rs[:k]


def exact_greedy(inst: Instances, s: int):
    """Greedy with exact marginal gains; ties to the smallest node id; nodes
    already chosen are never chosen again."""
    chosen, gains = [], []
    covered = [set() for _ in range(inst.l)]
    reach = [[inst.reach(u, i) for i in range(inst.l)] for u in range(inst.n)]
    for _ in range(s):
        best, bestg = None, -1
        for u in range(inst.n):
            if u in chosen:
                continue
            g = sum(len(reach[u][i] - covered[i]) for i in range(inst.l))
            if g > bestg:
                best, bestg = u, g
        chosen.append(best)
        gains.append(bestg)
        for i in range(inst.l):
            covered[i] |= reach[best][i]
    return chosen, gains


def union_estimate_exact(sketches: list[list[int]], k: int) -> Fraction:
    """Eq. unionest with exact rationals: taus as h/2^64 (1 for short sketches)."""
    def tau(x):
        return Fraction(x[k - 1], 1 << 64) if len(x) == k else Fraction(1)
    best: dict[int, Fraction] = {}
    for x in sketches:
        t = tau(x)
        body = x[: k - 1] if len(x) == k else x
        for z in body:
            if z not in best or t > best[z]:
                best[z] = t
    return sum((1 / t for t in best.values()), Fraction(0))


# ---- structured permutation ranks (Section 3.1) and IC-model positions ------

PERM_SALT = 0x7065726d75746531


def _chunk_order(n: int, c: int, kw: int) -> list[int]:
    return sorted(range(n), key=lambda v: fmix(kw + G * (c * n + v)))


def perm_positions(n: int, l: int, rank_key: int) -> dict[tuple[int, int], int]:
    """Position of every pair (v, i): chunk c lists each node once, in the order
    of its key for that chunk, paired with the node's c-th instance in the
    order of the pair ranks r(v, i)."""
    kw = fmix(rank_key ^ PERM_SALT)
    sigma = {v: sorted(range(l), key=lambda i: rank(rank_key, l, v, i)) for v in range(n)}
    pos = {}
    for c in range(l):
        for j, v in enumerate(_chunk_order(n, c, kw)):
            pos[(v, sigma[v][c])] = c * n + j
    return pos


def ic_nodes(n: int, chunks: int, rank_key: int) -> list[int]:
    kw = fmix(rank_key ^ PERM_SALT)
    out = []
    for c in range(chunks):
        out += _chunk_order(n, c, kw)
    return out

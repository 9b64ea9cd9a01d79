"""Seeded synthetic inputs: graphs, keys and query streams.

This module is the one piece shared by the oracle tests, the GPU tests and
the benchmark.  It produces *inputs* only (edge lists, per-run keys, seed
sets, arrival times) and holds none of the method's arithmetic: ranks, live
edge coins, sketches and estimators live in ``oracle/`` (CPU) and in the CUDA
library, each written separately.

The paper measured on SNAP/WebGraph networks (Section 6); those datasets are
not available here, so seeded Erdos-Renyi and R-MAT graphs of the same scale
range stand in for them.

Random draws come from the SplitMix64 generator (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the t-th
output of the stream with state s is ``fmix(s + t * GOLDEN)``, t >= 1.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

_G = np.uint64(GOLDEN)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _fmix_np(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _fmix_int(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream(state: int, count: int, start: int = 1) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream with `state`."""
    t = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(state & MASK64) + t * _G
    return _fmix_np(x)


@dataclass(frozen=True)
class Keys:
    """Per-run keys: graph generator, coins, ranks, trivalency classes, queries."""
    graph: int
    coin: int
    rank: int
    prob: int
    query: int

    @staticmethod
    def from_seed(seed: int) -> "Keys":
        out = [_fmix_int(seed + t * GOLDEN) for t in range(1, 6)]
        return Keys(*out)


@dataclass
class Graph:
    """Canonical directed graph: edges sorted by (src, dst), no duplicates,
    no self-loops.  Node ids are < n."""
    n: int
    src: np.ndarray  # uint32[m]
    dst: np.ndarray  # uint32[m]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.uint64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.src, dtype=np.uint32).tobytes())
        h.update(np.ascontiguousarray(self.dst, dtype=np.uint32).tobytes())
        return h.hexdigest()


def _canonical(n: int, u: np.ndarray, v: np.ndarray, name: str, meta: dict) -> Graph:
    u = u.astype(np.uint64)
    v = v.astype(np.uint64)
    keep = u != v
    key = np.unique((u[keep] << np.uint64(32)) | v[keep])
    src = (key >> np.uint64(32)).astype(np.uint32)
    dst = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return Graph(n=n, src=src, dst=dst, name=name, meta=meta)


def erdos_renyi(n: int, m: int, key: int) -> Graph:
    """Directed G(n, m): draw ordered pairs from the key stream, drop
    self-loops and repeats (first occurrence wins) until m distinct edges."""
    if m > n * (n - 1):
        raise ValueError("m exceeds the number of possible directed edges")
    chosen = np.empty(0, dtype=np.uint64)
    drawn = 0
    batch = max(1024, int(m * 1.3))
    while chosen.shape[0] < m:
        h = stream(key, batch, start=drawn + 1)
        drawn += batch
        u = ((h >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
        v = ((h & np.uint64(0xFFFFFFFF)) * np.uint64(n)) >> np.uint64(32)
        cand = (u << np.uint64(32)) | v
        cand = cand[u != v]
        allc = np.concatenate([chosen, cand])
        _, first = np.unique(allc, return_index=True)
        first.sort()
        chosen = allc[first]
        batch = max(1024, int((m - chosen.shape[0]) * 1.5) + 1024)
    chosen = chosen[:m]
    u = chosen >> np.uint64(32)
    v = chosen & np.uint64(0xFFFFFFFF)
    return _canonical(n, u, v, f"er_n{n}_m{m}", {"kind": "er", "n": n, "m_target": m})


# R-MAT quadrant thresholds on a 16-bit uniform (a, b, c, d) = (0.57, 0.19, 0.19, 0.05)
RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def _rmat_thresholds(abcd) -> tuple[int, int, int]:
    a, b, c, _ = abcd
    ta = int(math.floor(a * 65536 + 0.5))
    tb = ta + int(math.floor(b * 65536 + 0.5))
    tc = tb + int(math.floor(c * 65536 + 0.5))
    return ta, tb, tc


def _fmix_t(z):
    """SplitMix64 output function on an int64 torch tensor holding uint64 bits."""
    import torch
    z = z ^ ((z >> 30) & ((1 << 34) - 1))
    z = z * _signed(0xBF58476D1CE4E5B9)
    z = z ^ ((z >> 27) & ((1 << 37) - 1))
    z = z * _signed(0x94D049BB133111EB)
    z = z ^ ((z >> 31) & ((1 << 33) - 1))
    return z


def _signed(x: int) -> int:
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def rmat(scale: int, edge_factor: int, key: int, abcd=RMAT_ABCD, device: str = "cpu",
         chunk: int = 1 << 24) -> Graph:
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004) without noise or vertex
    permutation.  Draw j picks one quadrant per level, most significant bit
    first; level L of draw j reads 16 bits of stream output j*8 + L//4 + 1.
    Self-loops and duplicates are removed afterwards, so m < n * edge_factor.
    Integer-exact on any torch device, so CPU and GPU give the same graph."""
    import torch
    if not 1 <= scale <= 31:
        raise ValueError("scale must be in 1..31")
    n = 1 << scale
    draws = n * edge_factor
    ta, tb, tc = _rmat_thresholds(abcd)
    kk_all = []
    g = _signed(GOLDEN)
    for j0 in range(0, draws, chunk):
        cnt = min(chunk, draws - j0)
        j = torch.arange(j0, j0 + cnt, dtype=torch.int64, device=device)
        u = torch.zeros(cnt, dtype=torch.int64, device=device)
        v = torch.zeros(cnt, dtype=torch.int64, device=device)
        h = None
        for lvl in range(scale):
            if lvl % 4 == 0:
                x = (j * 8 + (lvl // 4 + 1)) * g + _signed(key)
                h = _fmix_t(x)
            w = (h >> (16 * (lvl % 4))) & 0xFFFF
            ubit = (w >= tb).to(torch.int64)
            vbit = (((w >= ta) & (w < tb)) | (w >= tc)).to(torch.int64)
            u = (u << 1) | ubit
            v = (v << 1) | vbit
        kk = (u << 32) | v
        kk_all.append(kk[u != v])
    kk = torch.unique(torch.cat(kk_all))  # sorted ascending; keys < 2^63
    src = (kk >> 32).to(torch.int32).cpu().numpy().astype(np.uint32)
    dst = (kk & 0xFFFFFFFF).to(torch.int64).cpu().numpy().astype(np.uint32)
    return Graph(n=n, src=src, dst=dst, name=f"rmat_s{scale}_ef{edge_factor}",
                 meta={"kind": "rmat", "scale": scale, "edge_factor": edge_factor, "abcd": list(abcd)})


def random_small_graph(n: int, m: int, key: int) -> Graph:
    """Tiny test graphs: G(n, m) with m clamped to the possible edges."""
    m = min(m, n * (n - 1))
    return erdos_renyi(n, m, key)


def chain(n: int) -> Graph:
    u = np.arange(n - 1, dtype=np.uint32)
    return _canonical(n, u, u + 1, f"chain{n}", {"kind": "chain"})


def star_out(n: int) -> Graph:
    v = np.arange(1, n, dtype=np.uint32)
    return _canonical(n, np.zeros(n - 1, np.uint32), v, f"star{n}", {"kind": "star"})


def cycle(n: int) -> Graph:
    u = np.arange(n, dtype=np.uint32)
    return _canonical(n, u, (u + 1) % n, f"cycle{n}", {"kind": "cycle"})


def clique(n: int) -> Graph:
    u, v = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    return _canonical(n, u.ravel(), v.ravel(), f"clique{n}", {"kind": "clique"})


def empty_graph(n: int) -> Graph:
    z = np.zeros(0, np.uint32)
    return Graph(n=n, src=z, dst=z.copy(), name=f"empty{n}", meta={"kind": "empty"})


# ----------------------------------------------------------------------------
# Query streams for the influence oracle (uniform seed sets, Section 6.2)
# ----------------------------------------------------------------------------

def query_sizes(count: int, key: int, max_size: int = 1000) -> np.ndarray:
    """|S| = floor(10^(3U)) clamped to 1..max_size, U uniform from the stream."""
    h = stream(key, count)
    u = (h >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    s = np.floor(np.power(10.0, 3.0 * u)).astype(np.int64)
    return np.clip(s, 1, max_size)


def uniform_seed_set(n: int, size: int, key: int, qid: int) -> np.ndarray:
    """`size` distinct nodes, uniform without replacement (rejection on repeats)."""
    size = min(size, n)
    out: list[int] = []
    seen: set[int] = set()
    t = 1
    base = _fmix_int(key + (qid + 1) * GOLDEN)
    while len(out) < size:
        h = stream(base, max(16, 2 * (size - len(out))), start=t)
        t += h.shape[0]
        for x in ((h >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32):
            xi = int(x)
            if xi not in seen:
                seen.add(xi)
                out.append(xi)
                if len(out) == size:
                    break
    return np.asarray(out, dtype=np.uint32)


class Neighborhoods:
    """The neighbourhood query generator of Section 6.2 over one graph: a root
    drawn with probability proportional to its degree (a uniformly random end
    of a uniformly random edge: in- plus out-degree), then the smallest radius
    d whose ball (all nodes within d hops, edges taken in either direction)
    holds at least `size` nodes, and `size` distinct nodes drawn uniformly from
    that ball.  A component smaller than `size` gives all of its nodes."""

    def __init__(self, n: int, src: np.ndarray, dst: np.ndarray):
        src = np.asarray(src, dtype=np.int64)
        dst = np.asarray(dst, dtype=np.int64)
        self.n, self.m = n, src.shape[0]
        self.src, self.dst = src, dst
        both_u = np.concatenate([src, dst])
        order = np.argsort(both_u, kind="stable")
        self.adj = np.concatenate([dst, src])[order]
        ptr = np.zeros(n + 1, np.int64)
        np.add.at(ptr, both_u + 1, 1)
        self.ptr = np.cumsum(ptr)

    def draw(self, size: int, key: int, qid: int) -> tuple[np.ndarray, int]:
        """Seed set (uint32) and the radius of its ball."""
        base = _fmix_int((key ^ 0x4E45494748424F52) + (qid + 1) * GOLDEN)
        h = int(stream(base, 1)[0])
        if self.m == 0:
            root = ((h >> 32) * self.n) >> 32
        else:
            e = ((h >> 32) * (2 * self.m)) >> 32
            root = int(self.src[e] if e < self.m else self.dst[e - self.m])
        seen = {root}
        ball = [root]
        frontier = [root]
        radius = 0
        while len(ball) < size and frontier:
            nxt = []
            for a in frontier:
                for b in self.adj[self.ptr[a]:self.ptr[a + 1]].tolist():
                    if b not in seen:
                        seen.add(b)
                        nxt.append(b)
            if not nxt:
                break
            radius += 1
            ball += nxt
            frontier = nxt
        take = min(size, len(ball))
        # partial Fisher-Yates over the ball with the query's stream
        r = stream(base, take, start=2)
        for i in range(take):
            j = i + ((int(r[i]) >> 32) * (len(ball) - i) >> 32)
            ball[i], ball[j] = ball[j], ball[i]
        return np.asarray(ball[:take], dtype=np.uint32), radius


def neighborhood_seed_set(n: int, src: np.ndarray, dst: np.ndarray, size: int, key: int, qid: int):
    """One draw of the neighbourhood generator (see Neighborhoods)."""
    return Neighborhoods(n, src, dst).draw(size, key, qid)


def poisson_arrivals(count: int, rate_per_s: float, key: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps by inversion."""
    h = stream(key ^ 0x5A5A5A5A5A5A5A5A, count)
    u = ((h >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    return np.cumsum(-np.log(u) / rate_per_s)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    kind: str            # "er" or "rmat"
    n_or_scale: int
    m_or_ef: int
    prob_model: int      # 0 uniform, 1 weighted cascade, 2 trivalency
    p: float
    l: int
    k: int
    seeds: int

    def keys(self) -> Keys:
        return Keys.from_seed(self.seed)

    def graph(self, device: str = "cpu") -> Graph:
        ks = self.keys()
        if self.kind == "er":
            return erdos_renyi(self.n_or_scale, self.m_or_ef, ks.graph)
        return rmat(self.n_or_scale, self.m_or_ef, ks.graph, device=device)


WORKLOADS = {
    "er4096": Workload("er4096", 1, "er", 4096, 32768, 0, 0.1, 16, 16, 10),
    "rmat18_wc": Workload("rmat18_wc", 3, "rmat", 18, 16, 1, 0.0, 64, 64, 50),
    "rmat20_wc": Workload("rmat20_wc", 2, "rmat", 20, 16, 1, 0.0, 64, 64, 50),
    "rmat22_wc": Workload("rmat22_wc", 4, "rmat", 22, 16, 1, 0.0, 64, 64, 0),
    # the hub-heavy searches of R-MAT 24 p = 0.01 at a sixteenth of its size
    "rmat20_p01": Workload("rmat20_p01", 6, "rmat", 20, 16, 0, 0.01, 64, 64, 50),
    "rmat24_p01": Workload("rmat24_p01", 5, "rmat", 24, 16, 0, 0.01, 64, 64, 200),
}


def batched_graph_specs(count: int = 256, seed: int = 3) -> list[tuple[int, int, int]]:
    """(scale, edge_factor, graph key) for the many-graph workload: scale
    uniform in 10..16 and edge factor uniform in 8..32."""
    ks = Keys.from_seed(seed)
    h = stream(ks.graph, 3 * count)
    out = []
    for g in range(count):
        scale = 10 + int(h[3 * g] % np.uint64(7))
        ef = 8 + int(h[3 * g + 1] % np.uint64(25))
        out.append((scale, ef, int(h[3 * g + 2])))
    return out

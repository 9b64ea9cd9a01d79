"""CPU oracle for SKIM and the sketch-based influence oracle (arXiv 1408.6282).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or runs anything here.

Thin ctypes wrapper around ``skim_oracle.c`` (plain, single-threaded C).  The
C file is compiled by :func:`build` with gcc; nothing here is shared with the
CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skim_oracle.c")
_LIB = os.path.join(_HERE, "libskim_oracle.so")
_lib = None

NCOUNT = 10
COUNTER_NAMES = ("rev_expansions", "rev_edge_scans", "insertions", "fwd_expansions",
                 "fwd_edge_scans", "ranks_processed", "ranks_consumed", "index_erased",
                 "rev_live_edges", "fwd_live_edges")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vectorisation flags: plain C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        u32p = C.POINTER(C.c_uint32)
        u64p = C.POINTER(C.c_uint64)
        g = [C.c_uint32, C.c_uint64, u32p, u32p]
        _lib.or_rank.restype = C.c_uint64
        _lib.or_rank.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        _lib.or_live.argtypes = g + [C.c_int, C.c_double, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        common = g + [C.c_uint32, C.c_uint32, C.c_int, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64]
        _lib.or_sketch_of_node.argtypes = common + [C.c_uint32, u64p, u32p, u64p]
        _lib.or_build_sketches.argtypes = common + [u64p, u32p, u64p]
        _lib.or_skim.argtypes = common + [C.c_uint32, u32p, u64p, u32p, u64p, u64p, C.POINTER(C.c_int32)]
        _lib.or_skim_mode.argtypes = common + [C.c_uint32, u32p, u64p, u32p, u64p, u64p, C.POINTER(C.c_int32),
                                               C.c_int]
        _lib.or_build_sketches_mode.argtypes = common + [u64p, u32p, u64p, C.c_int]
        _lib.or_build_ic_sketches.argtypes = g + [C.c_uint32, C.c_int, C.c_double, C.c_uint64, C.c_uint64,
                                                  C.c_uint64, u64p, u32p, u64p]
        _lib.or_perm_positions.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, u64p]
        _lib.or_ic_nodes.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, u32p]
        _lib.or_union_estimate_mode.argtypes = [u64p, u32p, C.c_uint32, C.c_uint32, C.c_uint32, u32p, C.c_uint32,
                                                C.c_int, C.POINTER(C.c_double)]
        _lib.or_node_estimates.argtypes = [u64p, u32p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int,
                                           C.POINTER(C.c_double)]
        _lib.or_exact_coverage.argtypes = g + [C.c_uint32, C.c_int, C.c_double, C.c_uint64, C.c_uint64,
                                               u32p, C.c_uint32, u64p]
        est = [u64p, u32p, C.c_uint32, C.c_uint32, C.c_uint32, u32p, C.c_uint32, C.POINTER(C.c_double)]
        _lib.or_union_estimate.argtypes = est
        _lib.or_bottomk_union_estimate.argtypes = est
    return _lib


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint32))


def _p64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


@dataclass
class Problem:
    """Graph (canonical edge list) plus the IC parameters and keys."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    l: int
    k: int
    model: int = 0          # 0 uniform, 1 weighted cascade, 2 trivalency
    p: float = 0.1
    coin_key: int = 0
    rank_key: int = 0
    prob_key: int = 0

    def __post_init__(self):
        self.src = np.ascontiguousarray(self.src, dtype=np.uint32)
        self.dst = np.ascontiguousarray(self.dst, dtype=np.uint32)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def _g(self):
        return [self.n, self.m, _p32(self.src), _p32(self.dst)]

    def _common(self):
        return self._g() + [self.l, self.k, self.model, self.p, self.coin_key, self.rank_key, self.prob_key]


def rank(rank_key: int, l: int, v: int, i: int) -> int:
    """Rank r(v,i) of a node-instance pair as a 64-bit integer."""
    return int(_load().or_rank(rank_key, l, v, i))


def live(pb: Problem, u: int, v: int, i: int) -> bool:
    """Live-edge coin of edge (u,v) in instance i."""
    r = _load().or_live(*pb._g(), pb.model, pb.p, pb.coin_key, pb.prob_key, u, v, i)
    if r < 0:
        _check(r, "live")
    return bool(r)


def sketch_of_node(pb: Problem, u: int):
    """X_u by the definition (Eq. combinedrs); returns (ranks, |R_u|)."""
    x = np.zeros(pb.k, np.uint64)
    ln = np.zeros(1, np.uint32)
    reach = np.zeros(1, np.uint64)
    _check(_load().or_sketch_of_node(*pb._common(), u, _p64(x), _p32(ln), _p64(reach)), "sketch_of_node")
    return x[: int(ln[0])].copy(), int(reach[0])


def build_sketches(pb: Problem, rank_mode: int = 0):
    """Algorithm 2: all combined sketches. Returns (X[n,k], len[n], counters).
    rank_mode 0: uniform 64-bit ranks; 1: structured permutation positions."""
    x = np.zeros((pb.n, pb.k), np.uint64)
    ln = np.zeros(pb.n, np.uint32)
    cnt = np.zeros(NCOUNT, np.uint64)
    _check(_load().or_build_sketches_mode(*pb._common(), _p64(x), _p32(ln), _p64(cnt), rank_mode),
           "build_sketches")
    return x, ln, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))


def build_ic_sketches(pb: Problem):
    """IC-model sketches (Section 3.2; pb.l is not used): X[n,k] of positions."""
    x = np.zeros((pb.n, pb.k), np.uint64)
    ln = np.zeros(pb.n, np.uint32)
    cnt = np.zeros(NCOUNT, np.uint64)
    _check(_load().or_build_ic_sketches(*pb._g(), pb.k, pb.model, pb.p, pb.coin_key, pb.rank_key, pb.prob_key,
                                        _p64(x), _p32(ln), _p64(cnt)), "build_ic_sketches")
    return x, ln, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))


def perm_positions(n: int, l: int, rank_key: int) -> np.ndarray:
    """Structured permutation (Section 3.1): position of pair (v,i) at [v*l+i]."""
    pos = np.zeros(n * l, np.uint64)
    _check(_load().or_perm_positions(n, l, rank_key, _p64(pos)), "perm_positions")
    return pos


def ic_nodes(n: int, chunks: int, rank_key: int) -> np.ndarray:
    """Node at each IC-model position t < chunks * n."""
    out = np.zeros(n * chunks, np.uint32)
    _check(_load().or_ic_nodes(n, chunks, rank_key, _p32(out)), "ic_nodes")
    return out


def skim(pb: Problem, n_seeds: int):
    """Algorithm 1: seeds and integer marginal coverages (l * I_j)."""
    seeds = np.zeros(n_seeds, np.uint32)
    cov = np.zeros(n_seeds, np.uint64)
    size = np.zeros(pb.n, np.uint32)
    cnt = np.zeros(NCOUNT, np.uint64)
    _check(_load().or_skim(*pb._common(), n_seeds, _p32(seeds), _p64(cov), _p32(size), _p64(cnt), None, None), "skim")
    return seeds, cov, size, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))


def skim_stops(pb: Problem, n_seeds: int, rank_mode: int = 0):
    """Algorithm 1 with what each iteration's selection saw (Section 4.3.2):
    seeds, coverages, the threshold rank tau of the search that stopped (as the
    64-bit rank; 0 when the ranks ran out), and k', the largest sketch size
    among the other nodes without that rank (-1 when the ranks ran out and the
    selection used exact residual counts).  rank_mode 1 orders the pairs by
    the structured permutation (Section 3.1); tau is then a position."""
    seeds = np.zeros(n_seeds, np.uint32)
    cov = np.zeros(n_seeds, np.uint64)
    tau = np.zeros(n_seeds, np.uint64)
    kp = np.zeros(n_seeds, np.int32)
    cnt = np.zeros(NCOUNT, np.uint64)
    _check(_load().or_skim_mode(*pb._common(), n_seeds, _p32(seeds), _p64(cov), None, _p64(cnt), _p64(tau),
                                kp.ctypes.data_as(C.POINTER(C.c_int32)), rank_mode), "skim")
    return seeds, cov, tau, kp, dict(zip(COUNTER_NAMES, (int(c) for c in cnt)))


def exact_coverage(pb: Problem, seeds) -> np.ndarray:
    """Prefix coverages: |union of R_u over the first j+1 seeds| for every j."""
    s = np.ascontiguousarray(seeds, dtype=np.uint32)
    out = np.zeros(max(1, s.shape[0]), np.uint64)
    _check(_load().or_exact_coverage(*pb._g(), pb.l, pb.model, pb.p, pb.coin_key, pb.prob_key,
                                     _p32(s), s.shape[0], _p64(out)), "exact_coverage")
    return out[: s.shape[0]]


def union_estimate(x: np.ndarray, ln: np.ndarray, l: int, seeds, rank_mode: int = 0) -> float:
    """Eq. unionest divided by l (the influence estimate); rank_mode 1/2 read
    positions as Sections 3.1/3.2 say."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    ln = np.ascontiguousarray(ln, dtype=np.uint32)
    s = np.ascontiguousarray(seeds, dtype=np.uint32)
    out = C.c_double()
    _check(_load().or_union_estimate_mode(_p64(x), _p32(ln), x.shape[0], x.shape[1], l, _p32(s),
                                          s.shape[0], rank_mode, C.byref(out)), "union_estimate")
    return out.value


def node_estimates(x: np.ndarray, ln: np.ndarray, l: int, rank_mode: int = 0) -> np.ndarray:
    """Single-node influence estimates from each node's own sketch."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    ln = np.ascontiguousarray(ln, dtype=np.uint32)
    out = np.zeros(x.shape[0], np.float64)
    _check(_load().or_node_estimates(_p64(x), _p32(ln), x.shape[0], x.shape[1], l, rank_mode,
                                     out.ctypes.data_as(C.POINTER(C.c_double))), "node_estimates")
    return out


def bottomk_union_estimate(x: np.ndarray, ln: np.ndarray, l: int, seeds) -> float:
    """(k-1)/tau of the union's bottom-k sketch, divided by l."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    ln = np.ascontiguousarray(ln, dtype=np.uint32)
    s = np.ascontiguousarray(seeds, dtype=np.uint32)
    out = C.c_double()
    _check(_load().or_bottomk_union_estimate(_p64(x), _p32(ln), x.shape[0], x.shape[1], l, _p32(s),
                                             s.shape[0], C.byref(out)), "bottomk_union_estimate")
    return out.value

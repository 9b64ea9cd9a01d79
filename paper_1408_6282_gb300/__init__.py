"""Python binding of libskim (SKIM and the sketch-based influence oracle on a
GB300 GPU).  Argument marshalling only: every step of the computation runs in
the CUDA library.  There is no CPU fallback -- if ``libskim.so`` is missing
or fails to load, every call raises.

The module-level functions carry the names of the C ABI (``include/skim.h``);
:class:`Skim` wraps them for numpy / torch callers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libskim.so")

SKIM_OK = 0
_ERR = {-1: "SKIM_EINVAL", -2: "SKIM_ENOMEM", -3: "SKIM_ENOTBUILT", -4: "SKIM_ETIMEOUT", -5: "SKIM_ECUDA",
        -6: "SKIM_EGRAPH", -7: "SKIM_ERANGE"}
PROB_UNIFORM, PROB_WC, PROB_TRIVALENCY = 0, 1, 2
RANKS_UNIFORM, RANKS_PERMUTATION, RANKS_IC_MODEL = 0, 1, 2
KERNEL_NAMES = ("rev_search", "fwd_search", "accept", "record_sort", "skim_step", "rank_order", "query", "setup",
                "instances", "rev_sources")
STAT_NAMES = ("rev_visits", "rev_coins", "insertions", "fwd_visits", "fwd_coins", "batches", "ranks", "retries",
              "rev_edges", "fwd_edges", "requeues")


class SkimError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_ERR.get(code, code)} ({code})")
        self.code = code


class skim_graph(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("on_device", C.c_int)]


class skim_tuning(C.Structure):
    _fields_ = [("batch_lanes", C.c_uint32), ("ring_records_per_lane", C.c_double),
                ("node_sort_density", C.c_uint32)]


class skim_params(C.Structure):
    _fields_ = [("l", C.c_uint32), ("k", C.c_uint32), ("prob_model", C.c_int), ("p", C.c_double),
                ("coin_key", C.c_uint64), ("rank_key", C.c_uint64), ("prob_key", C.c_uint64),
                ("batch_lanes", C.c_uint32), ("rank_mode", C.c_uint32)]


_lib = None


def load():
    """Load libskim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libskim.so not found at {LIB_PATH}; build it with "
                           "`python -m paper_1408_6282_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
    lib.skim_create.argtypes = [C.POINTER(skim_graph), C.POINTER(skim_params), vp, C.POINTER(vp)]
    lib.skim_build_sketches.argtypes = [vp]
    lib.skim_get_sketches.argtypes = [vp, vp, vp, C.c_int]
    lib.skim_sketch_pointers.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
    lib.skim_get_sketch.argtypes = [vp, u32, vp, vp]
    lib.skim_get_tuning.argtypes = [vp, C.POINTER(skim_tuning)]
    lib.skim_set_tuning.argtypes = [vp, C.POINTER(skim_tuning)]
    lib.skim_autotune.argtypes = [vp, C.POINTER(skim_tuning), u32, vp, vp]
    lib.skim_set_wait_limit_ns.argtypes = [vp, u64]
    lib.skim_set_live_rows.argtypes = [vp, C.c_int]
    lib.skim_greedy.argtypes = [vp, u32, vp, vp]
    lib.skim_greedy_reset.argtypes = [vp]
    lib.skim_greedy_ex.argtypes = [vp, u32, vp, vp, vp, vp]
    lib.skim_node_estimates.argtypes = [vp, vp, C.c_int]
    lib.skim_discrepancy_bound.argtypes = [u32, vp, vp, vp, C.c_double, u32, u32, vp, vp, vp]
    lib.skim_oracle_query.argtypes = [vp, vp, u32, vp]
    lib.skim_oracle_query_batch.argtypes = [vp, vp, u32, vp, vp, C.c_int]
    lib.skim_get_stats.argtypes = [vp, vp, u32]
    lib.skim_destroy.argtypes = [vp]
    lib.skim_release_memory.argtypes = []
    lib.skim_rank_order.argtypes = [vp]
    lib.skim_instances.argtypes = [vp]
    lib.skim_instance_stats.argtypes = [vp, vp, vp]
    lib.skim_set_timing.argtypes = [vp, C.c_int]
    lib.skim_kernel_times.argtypes = [vp, vp, vp, u32, C.c_int]
    lib.skim_kernel_launches.argtypes = [vp]
    lib.skim_union_estimate_static.argtypes = [vp, vp, u32, u32, u32, u32, vp, u32, vp, vp]
    lib.skim_context_shape.argtypes = [vp, vp, vp, vp]
    lib.skim_create_batch.argtypes = [vp, vp, u32, vp, C.POINTER(vp)]
    lib.skim_autotune_batch_lanes.argtypes = [vp, vp, u32, vp, vp]
    lib.skim_server_start.argtypes = [vp, u32, u64, u32, C.POINTER(vp)]
    lib.skim_server_submit.argtypes = [vp, vp, u32, vp]
    lib.skim_server_poll.argtypes = [vp, u64, vp, vp]
    lib.skim_server_wait.argtypes = [vp, u64, vp, u32]
    lib.skim_server_replay.argtypes = [vp, vp, vp, vp, u32, vp, vp]
    lib.skim_server_stats.argtypes = [vp, vp, vp]
    lib.skim_server_stop.argtypes = [vp]
    lib.skim_strerror.argtypes = [C.c_int]
    lib.skim_strerror.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != SKIM_OK:
        raise SkimError(rc, what)


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


# ---- C ABI names -------------------------------------------------------------

def skim_create(graph: skim_graph, params: skim_params, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().skim_create(C.byref(graph), C.byref(params), C.c_void_p(stream or None), C.byref(h)),
           "skim_create")
    return h.value


def skim_create_batch(graphs, params, stream: int = 0) -> int:
    """graphs: sequence of skim_graph (host edge lists), params: sequence of skim_params."""
    G = (skim_graph * len(graphs))(*graphs)
    P = (skim_params * len(params))(*params)
    h = C.c_void_p()
    _check(load().skim_create_batch(C.cast(G, C.c_void_p), C.cast(P, C.c_void_p), len(graphs),
                                    C.c_void_p(stream or None), C.byref(h)), "skim_create_batch")
    return h.value


def skim_autotune_batch_lanes(ctx: int, candidates) -> tuple[int, np.ndarray]:
    cand = np.ascontiguousarray(candidates, dtype=np.uint32)
    best = np.zeros(1, np.uint32)
    secs = np.zeros(cand.shape[0], np.float64)
    _check(load().skim_autotune_batch_lanes(ctx, _ptr(cand), cand.shape[0], _ptr(best), _ptr(secs)),
           "skim_autotune_batch_lanes")
    return int(best[0]), secs


def skim_rank_order(ctx: int):
    _check(load().skim_rank_order(ctx), "skim_rank_order")


def skim_set_timing(ctx: int, on: int):
    _check(load().skim_set_timing(ctx, on), "skim_set_timing")


def skim_kernel_times(ctx: int, ms_out: np.ndarray, launches_out: np.ndarray, count: int, reset: int):
    _check(load().skim_kernel_times(ctx, _ptr(ms_out), _ptr(launches_out), count, reset), "skim_kernel_times")


def skim_build_sketches(ctx: int):
    _check(load().skim_build_sketches(ctx), "skim_build_sketches")


def skim_get_sketches(ctx: int, x_out, len_out, out_on_device: int = 0):
    _check(load().skim_get_sketches(ctx, _ptr(x_out), _ptr(len_out), out_on_device), "skim_get_sketches")


def skim_get_sketch(ctx: int, v: int, out_k: np.ndarray) -> int:
    """X_v into out_k (host uint64, >= k entries); returns |X_v|."""
    ln = np.zeros(1, np.uint32)
    _check(load().skim_get_sketch(ctx, v, _ptr(out_k), _ptr(ln)), "skim_get_sketch")
    return int(ln[0])


def skim_set_wait_limit_ns(ctx: int, ns: int):
    _check(load().skim_set_wait_limit_ns(ctx, ns), "skim_set_wait_limit_ns")


def skim_set_live_rows(ctx: int, on: bool):
    _check(load().skim_set_live_rows(ctx, 1 if on else 0), "skim_set_live_rows")


def skim_sketch_pointers(ctx: int) -> tuple[int, int]:
    x, ln = C.c_void_p(), C.c_void_p()
    _check(load().skim_sketch_pointers(ctx, C.byref(x), C.byref(ln)), "skim_sketch_pointers")
    return x.value, ln.value


def skim_greedy(ctx: int, n_seeds: int, seeds_out: np.ndarray, cov_out: np.ndarray):
    _check(load().skim_greedy(ctx, n_seeds, _ptr(seeds_out), _ptr(cov_out)), "skim_greedy")


def skim_greedy_ex(ctx: int, n_seeds: int, seeds_out, cov_out, tau_out=None, kprime_out=None):
    _check(load().skim_greedy_ex(ctx, n_seeds, _ptr(seeds_out), _ptr(cov_out),
                                 _ptr(tau_out) if tau_out is not None else None,
                                 _ptr(kprime_out) if kprime_out is not None else None), "skim_greedy_ex")


def skim_discrepancy_bound(s: int, delta, tau, kprime, step: float, bins: int, n_conf: int, conf, bound_out,
                           ccdf_out=None):
    _check(load().skim_discrepancy_bound(s, _ptr(delta) if s else None, _ptr(tau) if s else None,
                                         _ptr(kprime) if s else None, step, bins, n_conf,
                                         _ptr(conf) if n_conf else None, _ptr(bound_out) if n_conf else None,
                                         _ptr(ccdf_out) if ccdf_out is not None else None),
           "skim_discrepancy_bound")


def discrepancy_bound(delta, tau, kprime, step: float, bins: int = 4096, conf=(0.9, 0.95, 0.99)):
    """Section 4.3.2 bound on the sum of discrepancies of a SKIM run (pairs):
    returns (bounds per confidence, ccdf over the grid plus the overflow)."""
    d = np.ascontiguousarray(delta, dtype=np.uint64)
    t = np.ascontiguousarray(tau, dtype=np.uint64)
    kp = np.ascontiguousarray(kprime, dtype=np.int32)
    cf = np.ascontiguousarray(conf, dtype=np.float64)
    out = np.zeros(max(1, cf.shape[0]), np.float64)
    ccdf = np.zeros(bins + 1, np.float64)
    skim_discrepancy_bound(int(d.shape[0]), d, t, kp, float(step), int(bins), int(cf.shape[0]), cf, out, ccdf)
    return out[: cf.shape[0]], ccdf


def skim_node_estimates(ctx: int, out, out_on_device: int = 0):
    _check(load().skim_node_estimates(ctx, _ptr(out), out_on_device), "skim_node_estimates")


def skim_instances(ctx: int):
    _check(load().skim_instances(ctx), "skim_instances")


def skim_greedy_reset(ctx: int):
    _check(load().skim_greedy_reset(ctx), "skim_greedy_reset")


def skim_oracle_query(ctx: int, seeds: np.ndarray, n_seeds: int, est_out: np.ndarray):
    _check(load().skim_oracle_query(ctx, _ptr(seeds) if n_seeds else None, n_seeds, _ptr(est_out)),
           "skim_oracle_query")


def skim_oracle_query_batch(ctx: int, offsets: np.ndarray, q: int, seeds, est_out, on_device: int = 0):
    _check(load().skim_oracle_query_batch(ctx, _ptr(offsets), q, _ptr(seeds), _ptr(est_out), on_device),
           "skim_oracle_query_batch")


def skim_get_stats(ctx: int, out: np.ndarray, count: int):
    _check(load().skim_get_stats(ctx, _ptr(out), count), "skim_get_stats")


def skim_kernel_launches() -> int:
    out = np.zeros(1, np.uint64)
    _check(load().skim_kernel_launches(_ptr(out)), "skim_kernel_launches")
    return int(out[0])


def skim_union_estimate_static(x_dev: int, len_dev: int, n: int, k: int, l: int, seeds_dev: int, n_seeds: int,
                               est_dev: int, stream: int = 0, rank_mode: int = 0):
    """Allocation-free query (static scratch); all pointers are device addresses.
    rank_mode is the SKIM_RANKS_* reading of the context the sketches came from."""
    _check(load().skim_union_estimate_static(x_dev, len_dev, n, k, l, rank_mode, seeds_dev or None, n_seeds,
                                             est_dev, stream or None), "skim_union_estimate_static")


def skim_server_start(ctx: int, max_inflight: int, scratch_slots: int, streams: int) -> int:
    h = C.c_void_p()
    _check(load().skim_server_start(ctx, max_inflight, scratch_slots, streams, C.byref(h)), "skim_server_start")
    return h.value


def skim_server_submit(srv: int, seeds: np.ndarray, n_seeds: int) -> int:
    t = np.zeros(1, np.uint64)
    _check(load().skim_server_submit(srv, _ptr(seeds) if n_seeds else None, n_seeds, _ptr(t)), "skim_server_submit")
    return int(t[0])


def skim_server_poll(srv: int, ticket: int):
    done = np.zeros(1, np.int32)
    est = np.zeros(1, np.float64)
    _check(load().skim_server_poll(srv, ticket, _ptr(done), _ptr(est)), "skim_server_poll")
    return bool(done[0]), float(est[0])


def skim_server_wait(srv: int, ticket: int, timeout_ms: int = 60000) -> float:
    est = np.zeros(1, np.float64)
    _check(load().skim_server_wait(srv, ticket, _ptr(est), timeout_ms), "skim_server_wait")
    return float(est[0])


def skim_server_replay(srv: int, arrival_s: np.ndarray, offsets: np.ndarray, seeds: np.ndarray, q: int,
                       latency_s: np.ndarray, est_out: np.ndarray):
    _check(load().skim_server_replay(srv, _ptr(arrival_s), _ptr(offsets), _ptr(seeds), q, _ptr(latency_s),
                                     _ptr(est_out)), "skim_server_replay")


def skim_server_stats(srv: int) -> tuple[int, int]:
    g = np.zeros(1, np.uint64)
    q = np.zeros(1, np.uint64)
    _check(load().skim_server_stats(srv, _ptr(g), _ptr(q)), "skim_server_stats")
    return int(g[0]), int(q[0])


def skim_server_stop(srv: int):
    _check(load().skim_server_stop(srv), "skim_server_stop")


def skim_destroy(ctx: int):
    _check(load().skim_destroy(ctx), "skim_destroy")


def skim_release_memory():
    """Hand the device memory pooled from destroyed contexts back to the device."""
    _check(load().skim_release_memory(), "skim_release_memory")


def skim_strerror(code: int) -> str:
    return load().skim_strerror(code).decode()


# ---- convenience wrapper -------------------------------------------------------

class Skim:
    """One graph, its IC parameters and the device state built from them.

    src/dst: canonical edge list (sorted by (src, dst), no duplicates, no
    self-loops) as uint32 numpy arrays (host) or int32/uint32 CUDA tensors.
    """

    def __init__(self, n: int, src, dst, l: int, k: int, prob_model: int = PROB_UNIFORM, p: float = 0.1,
                 coin_key: int = 0, rank_key: int = 0, prob_key: int = 0, batch_lanes: int = 0, stream: int = 0,
                 rank_mode: int = 0):
        on_device = not isinstance(src, np.ndarray)
        if not on_device:
            src = np.ascontiguousarray(src, dtype=np.uint32)
            dst = np.ascontiguousarray(dst, dtype=np.uint32)
        self._keep = (src, dst)
        m = int(src.shape[0])
        g = skim_graph(n, m, _ptr(src) if m else None, _ptr(dst) if m else None, 1 if on_device else 0)
        prm = skim_params(l, k, prob_model, p, coin_key & (2**64 - 1), rank_key & (2**64 - 1),
                          prob_key & (2**64 - 1), batch_lanes, rank_mode)
        self.n, self.m, self.l, self.k, self.rank_mode = n, m, l, k, rank_mode
        self.ctx = skim_create(g, prm, stream)
        self._keep = None

    @classmethod
    def batch(cls, graphs, l: int, k: int, models, ps, coin_keys, rank_keys, prob_keys, batch_lanes: int = 0,
              stream: int = 0) -> "Skim":
        """Many graphs in one context: graphs = [(n, src, dst), ...] (host uint32 arrays)."""
        keep, gs, prms = [], [], []
        for (n, src, dst), mdl, p, ck, rk, pk in zip(graphs, models, ps, coin_keys, rank_keys, prob_keys):
            src = np.ascontiguousarray(src, dtype=np.uint32)
            dst = np.ascontiguousarray(dst, dtype=np.uint32)
            keep += [src, dst]
            m = int(src.shape[0])
            gs.append(skim_graph(n, m, _ptr(src) if m else None, _ptr(dst) if m else None, 0))
            prms.append(skim_params(l, k, mdl, p, ck & (2**64 - 1), rk & (2**64 - 1), pk & (2**64 - 1), batch_lanes))
        self = cls.__new__(cls)
        self.n = sum(g[0] for g in graphs)
        self.m = sum(int(g[1].shape[0]) for g in graphs)
        self.l, self.k = l, k
        self.ctx = skim_create_batch(gs, prms, stream)
        self.offsets = np.concatenate([[0], np.cumsum([g[0] for g in graphs])]).astype(np.int64)
        return self

    def autotune(self, candidates) -> tuple[int, np.ndarray]:
        return skim_autotune_batch_lanes(self.ctx, candidates)

    def tuning(self) -> dict:
        t = skim_tuning()
        _check(load().skim_get_tuning(self.ctx, C.byref(t)), "skim_get_tuning")
        return {"batch_lanes": t.batch_lanes, "ring_records_per_lane": t.ring_records_per_lane,
                "node_sort_density": t.node_sort_density}

    def set_tuning(self, batch_lanes: int, ring_records_per_lane: float, node_sort_density: int):
        t = skim_tuning(batch_lanes, ring_records_per_lane, node_sort_density)
        _check(load().skim_set_tuning(self.ctx, C.byref(t)), "skim_set_tuning")

    def autotune_settings(self, settings) -> tuple[int, np.ndarray]:
        """settings: [(batch_lanes, ring_records_per_lane, node_sort_density), ...];
        returns (index of the fastest, seconds of each)."""
        arr = (skim_tuning * len(settings))(*[skim_tuning(*x) for x in settings])
        best = np.zeros(1, np.uint32)
        secs = np.zeros(len(settings), np.float64)
        _check(load().skim_autotune(self.ctx, arr, len(settings), _ptr(best), _ptr(secs)), "skim_autotune")
        return int(best[0]), secs

    def close(self):
        if getattr(self, "ctx", None):
            skim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def build_sketches(self):
        skim_build_sketches(self.ctx)

    def sketches(self) -> tuple[np.ndarray, np.ndarray]:
        x = np.zeros((self.n, self.k), np.uint64)
        ln = np.zeros(self.n, np.uint32)
        skim_get_sketches(self.ctx, x, ln, 0)
        return x, ln

    def sketch(self, v: int) -> np.ndarray:
        """X_v of one node (ascending ranks)."""
        out = np.zeros(self.k, np.uint64)
        return out[: skim_get_sketch(self.ctx, v, out)]

    def set_live_rows(self, on: bool):
        """Walk materialised live rows (True) or hash coins during the search (False)."""
        skim_set_live_rows(self.ctx, on)

    def set_wait_limit_ns(self, ns: int):
        skim_set_wait_limit_ns(self.ctx, ns)

    def greedy(self, n_seeds: int) -> tuple[np.ndarray, np.ndarray]:
        seeds = np.zeros(max(1, n_seeds), np.uint32)
        cov = np.zeros(max(1, n_seeds), np.uint64)
        skim_greedy(self.ctx, n_seeds, seeds, cov)
        return seeds[:n_seeds], cov[:n_seeds]

    def greedy_stops(self, n_seeds: int):
        """greedy() plus each selection's threshold rank and k' (Section 4.3.2)."""
        m = max(1, n_seeds)
        seeds, cov = np.zeros(m, np.uint32), np.zeros(m, np.uint64)
        tau, kp = np.zeros(m, np.uint64), np.zeros(m, np.int32)
        skim_greedy_ex(self.ctx, n_seeds, seeds, cov, tau, kp)
        return seeds[:n_seeds], cov[:n_seeds], tau[:n_seeds], kp[:n_seeds]

    def greedy_reset(self):
        skim_greedy_reset(self.ctx)

    def instances(self):
        """Regenerate the live-edge instances (done at creation)."""
        skim_instances(self.ctx)

    def instance_stats(self) -> tuple[int, bool]:
        """(live edge-instance pairs, whether searches use them)."""
        lp = np.zeros(1, np.uint64)
        mt = np.zeros(1, np.int32)
        _check(load().skim_instance_stats(self.ctx, _ptr(lp), _ptr(mt)), "skim_instance_stats")
        return int(lp[0]), bool(mt[0])

    def node_estimates(self) -> np.ndarray:
        """Single-node influence estimates from every node's own sketch."""
        out = np.zeros(self.n, np.float64)
        skim_node_estimates(self.ctx, out, 0)
        return out

    def query(self, seeds) -> float:
        s = np.ascontiguousarray(seeds, dtype=np.uint32)
        out = np.zeros(1, np.float64)
        skim_oracle_query(self.ctx, s, int(s.shape[0]), out)
        return float(out[0])

    def query_batch(self, seed_sets) -> np.ndarray:
        sets = [np.ascontiguousarray(s, dtype=np.uint32) for s in seed_sets]
        off = np.zeros(len(sets) + 1, np.uint64)
        off[1:] = np.cumsum([s.shape[0] for s in sets])
        flat = np.concatenate(sets) if sets and off[-1] else np.zeros(1, np.uint32)
        out = np.zeros(max(1, len(sets)), np.float64)
        skim_oracle_query_batch(self.ctx, off, len(sets), flat, out, 0)
        return out[: len(sets)]

    def rank_order(self):
        skim_rank_order(self.ctx)

    def set_timing(self, on: bool = True):
        skim_set_timing(self.ctx, 1 if on else 0)

    def kernel_times(self, reset: bool = False) -> dict:
        ms = np.zeros(len(KERNEL_NAMES), np.float64)
        cnt = np.zeros(len(KERNEL_NAMES), np.uint64)
        skim_kernel_times(self.ctx, ms, cnt, len(KERNEL_NAMES), 1 if reset else 0)
        return {n: (float(a), int(b)) for n, a, b in zip(KERNEL_NAMES, ms, cnt)}

    def server(self, max_inflight: int = 4096, scratch_slots: int = 1 << 24, streams: int = 4) -> "Server":
        return Server(self, max_inflight, scratch_slots, streams)

    def stats(self) -> dict:
        out = np.zeros(len(STAT_NAMES), np.uint64)
        skim_get_stats(self.ctx, out, len(STAT_NAMES))
        return dict(zip(STAT_NAMES, (int(v) for v in out)))


class Server:
    """Continuous-batching query server over a Skim context's sketches."""

    def __init__(self, sk: Skim, max_inflight: int = 4096, scratch_slots: int = 1 << 24, streams: int = 4):
        self.sk = sk
        self.srv = skim_server_start(sk.ctx, max_inflight, scratch_slots, streams)

    def submit(self, seeds) -> int:
        s = np.ascontiguousarray(seeds, dtype=np.uint32)
        return skim_server_submit(self.srv, s, int(s.shape[0]))

    def poll(self, ticket: int):
        return skim_server_poll(self.srv, ticket)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> float:
        return skim_server_wait(self.srv, ticket, timeout_ms)

    def replay(self, arrival_s, seed_sets):
        sets = [np.ascontiguousarray(x, dtype=np.uint32) for x in seed_sets]
        off = np.zeros(len(sets) + 1, np.uint64)
        off[1:] = np.cumsum([x.shape[0] for x in sets])
        flat = np.concatenate(sets) if sets and off[-1] else np.zeros(1, np.uint32)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(max(1, len(sets)), np.float64)
        est = np.zeros(max(1, len(sets)), np.float64)
        skim_server_replay(self.srv, arr, off, flat, len(sets), lat, est)
        return lat[: len(sets)], est[: len(sets)]

    def stats(self) -> tuple[int, int]:
        return skim_server_stats(self.srv)

    def stop(self):
        if self.srv:
            skim_server_stop(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()

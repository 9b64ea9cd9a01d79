// common.cuh -- device-side building blocks shared by the libskim kernels.
//
// Ranks and live-edge coins follow Sections 2-3 of Cohen, Delling, Pajor,
// Werneck (arXiv 1408.6282): one independent uniform rank per node-instance
// pair, one independent coin per (edge, instance) of the binary IC model.
// Both are drawn from the SplitMix64 output function (Steele, Lea, Flood
// 2014), read as 64-bit integers, so instances are never materialised.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#define SKIM_DEV __device__ __forceinline__
#define SKIM_HD __host__ __device__ __forceinline__

namespace skim {

// Kernels launched by this library since it was loaded (every launch site
// calls note_launch()).
inline std::atomic<unsigned long long> g_kernel_launches{0};
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kEmptyKey = ~0ull;
// Materialised live rows: 32-bit offsets into the row array; the top bit of
// row r's start (r = v * l + i) says that the instance-local sketch of (v, i)
// holds k ranks (Algorithm 2's pruning), so one load gives the row and the
// pruning decision.  Offsets therefore stay below 2^31.
constexpr uint32_t kRowMask = 0x7FFFFFFFu;
constexpr uint32_t kRowFull = 0x80000000u;
// key of the within-chunk node order of permutation ranks: fmix(rank_key ^ salt)
constexpr uint64_t kPermSalt = 0x7065726d75746531ull;
constexpr unsigned kFull = 0xffffffffu;

// Work items are cut so that one item costs about kTargetCoins coin
// evaluations (edges x lanes): a hub never serialises a warp for long.  At
// most 2^kChunkBits chunks per node; index-erase items hold kChunk entries.
constexpr uint32_t kChunk = 4096;
constexpr uint32_t kChunkBits = 12;          // chunk id field width in Item::w
constexpr uint32_t kTargetCoins = 8192;
constexpr uint32_t kMinChunkEdges = 32;
constexpr uint32_t kEraseTag = 0x80000000u;
constexpr uint32_t kNopTag = 0xFFFFFFFEu;      // placeholder item (a spilled reservation)
constexpr uint32_t kMaxWords = 1u << 19;       // lane words per batch (w field: word << 12 | chunk < 2^31)

// SplitMix64 output function.
SKIM_HD uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rank r(v,i) of pair index x = v*l + i.
SKIM_HD uint64_t pair_rank(uint64_t rank_key, uint64_t x) { return fmix(rank_key + kGolden * x); }

// State of the coin stream of directed edge (u,v); coin of instance i is
// output i+1 of that stream.
SKIM_HD uint64_t edge_state(uint64_t coin_key, uint32_t u, uint32_t v) {
    return fmix(coin_key ^ ((static_cast<uint64_t>(u) << 32) | v));
}
SKIM_HD bool coin_live(uint64_t he, uint32_t inst, uint64_t tm1) {
    return fmix(he + kGolden * static_cast<uint64_t>(inst + 1)) <= tm1;
}

// Edges per work item for a node of degree deg expanded for the lanes of mask.
SKIM_HD uint32_t chunk_edges(uint32_t deg, uint64_t mask) {
    const uint32_t pc = static_cast<uint32_t>(__builtin_popcountll(mask));
    uint32_t want = kTargetCoins / (pc ? pc : 1);
    if (want < kMinChunkEdges) want = kMinChunkEdges;
    if (want > kChunk) want = kChunk;
    const uint32_t floor_c = (deg + (1u << kChunkBits) - 1) >> kChunkBits;  // keeps chunk ids < 2^kChunkBits
    return want > floor_c ? want : floor_c;
}

// Materialised row items name the lane's instance too: w = inst << 25 |
// word << 6 | lane bit (word < kMaxWords = 2^19).
constexpr uint32_t kInstShift = 25;

// Work item of the asynchronous traversals (16 bytes).  Reverse searches:
// v = node, w = (lane word << 12) | chunk, mask = lanes of that word visiting
// v.  Residual searches: w = chunk, mask = instances.  Index-erase items:
// w = kEraseTag | chunk, v = segment length, mask = segment start + 1.
// In the queue, v and w are stored plus one; every field of a written slot
// is then non-zero, so a reader that sees three non-zero fields has the whole
// item, and the queue needs no fences (slots start zeroed).
struct __align__(16) Item {
    uint32_t v;
    uint32_t w;
    uint64_t mask;
};

// Error bits in DevCtl::err.  Records/hash overflow: the batch is re-run
// with fewer lanes.  A full queue is not an error: the work is spilled to
// per-entry pending masks and re-queued after the queue drains.
constexpr unsigned kErrRecords = 2u, kErrHash = 4u, kErrTimeout = 8u;
constexpr unsigned kErrRetryable = kErrRecords | kErrHash;

// A counter alone on its 128-byte line: the queue cursors are hit by every
// warp, and sharing a line would serialise them at one L2 slice.
struct alignas(128) HotCounter {
    unsigned long long v;
    unsigned long long pad[15];
};

// Device control block: queue cursors, counters, flags, reductions.
// src_next, busy and beat serve the reverse searches with per-warp queues:
// the next unclaimed source lane of the batch, the warps that hold work, and
// a progress count that working warps advance now and then.
struct DevCtl {
    HotCounter q_head, q_tail, q_done, rec_count;
    HotCounter src_next, busy, beat;
    unsigned long long best;        // SKIM stop candidate: (lane << 32) | node
    unsigned long long ix_cov;      // pairs newly covered by the residual search
    unsigned long long argmax;      // (size << 32) | ~node
    unsigned long long total;       // generic total (lane commits)
    unsigned long long stats[8];
    unsigned int err;
    unsigned int spill;   // some work was parked in pending masks
    unsigned int pad[2];
};

enum Stat { kStRevVisits = 0, kStRevCoins, kStInsert, kStFwdVisits, kStFwdCoins, kStRevEdges, kStFwdEdges };

SKIM_DEV uint64_t ld_acquire(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
SKIM_DEV void st_release(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
SKIM_DEV unsigned long long ld_volatile(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
SKIM_DEV uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// n-th (0-based) set bit of a 64-bit mask; the mask must have > n bits set.
SKIM_DEV int nth_set_bit(uint64_t m, int n) {
    uint32_t lo = static_cast<uint32_t>(m);
    int cl = __popc(lo);
    if (n < cl) return __fns(lo, 0, n + 1);
    return 32 + __fns(static_cast<uint32_t>(m >> 32), 0, n - cl + 1);
}

SKIM_DEV unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Warp-aggregated add of a per-lane value to a global counter.
SKIM_DEV void warp_add(unsigned long long *ctr, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, v);
}

// Exclusive warp prefix sum; returns the exclusive value, total via *tot.
SKIM_DEV unsigned long long warp_excl_scan(unsigned long long v, unsigned long long *tot) {
    const int lane = threadIdx.x & 31;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    *tot = __shfl_sync(kFull, x, 31);
    return x - v;
}

}  // namespace skim

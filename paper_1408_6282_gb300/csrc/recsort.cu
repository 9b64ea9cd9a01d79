// recsort.cu -- order one batch's visit records by (node, lane word), node by
// node.
//
// The reverse search leaves its records (node << tbits | word, table slot) in
// arrival order; the acceptance of Algorithm 2 wants each node's records
// together and in word order (= rank order: lane j of word t has rank
// position 64 t + j within the batch).  When the records are dense over the
// nodes they are placed per node instead of by a radix sort over all key bits:
//
//   count   records per node (atomics on a per-node counter);
//   scan    node offsets off[v] = records of nodes < v;
//   scatter each record into its node's segment (the counter counts down, so
//           it is zero again for the next batch);
//   order   each segment by word.  Words are distinct within a node (one
//           table slot per (node, word)), so a segment of s records is put in
//           order by its node's thread in registers (s <= 8), by a warp
//           across its lanes (s <= 32), or by a block through a bitmap of
//           the 2^tbits words (any s).
//
// The result is the same array a full sort gives (keys are distinct), and the
// node offsets are left for the caller.  A caller may pass buckets of 2^s
// consecutive nodes as the "nodes" (n / 2^s of them) and tbits + s as the
// word bits: a bucket's records are then ordered by (node, word), which is the
// key order too.
#include "internal.cuh"
#include "prims.cuh"

namespace skim {

namespace {

inline unsigned grid_for(size_t n, int threads, unsigned cap = 152 * 32) {
    size_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g ? g : 1);
}

constexpr uint32_t kThreadSeg = 8;  // records a node's thread orders itself
constexpr uint32_t kWarpSeg = 32;   // records a warp orders across its lanes
constexpr int kBigThreads = 256;
#ifndef SKIM_BIG_BLOCKS
#define SKIM_BIG_BLOCKS (152 * 8)
#endif

__global__ void k_node_count(const uint64_t *__restrict__ rec_key, uint64_t R, uint32_t tbits,
                             unsigned long long *cnt) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[rec_key[r] >> tbits], 1ull);
}

// tmp[off[v] + p] = word << 32 | slot, p counted down from the node's count
__global__ void k_node_scatter(const uint64_t *__restrict__ rec_key, const uint32_t *__restrict__ rec_val, uint64_t R,
                               uint32_t tbits, const uint64_t *__restrict__ off, unsigned long long *cnt,
                               uint64_t *__restrict__ tmp) {
    const uint64_t tmask = (1ull << tbits) - 1;
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t key = rec_key[r];
        const uint64_t v = key >> tbits;
        const uint64_t p = atomicAdd(&cnt[v], ~0ull) - 1;  // count down
        tmp[off[v] + p] = ((key & tmask) << 32) | rec_val[r];
    }
}

// Output of the ordering: key and table slot of each record.
struct OrderOut {
    uint64_t *rec_key;
    uint32_t *rec_val;
};

SKIM_DEV void put(const OrderOut &o, uint64_t at, uint64_t vhi, uint64_t p) {
    o.rec_key[at] = vhi | (p >> 32);
    o.rec_val[at] = static_cast<uint32_t>(p);
}

SKIM_DEV void cswap(uint64_t &a, uint64_t &b) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

// One thread per node: segments of up to kThreadSeg records are ordered in
// registers (odd-even transposition network, padded with all-ones keys);
// longer ones are listed for the warp (front of `list`) or block (back) pass.
__global__ void k_node_order(const uint64_t *__restrict__ tmp, const uint64_t *__restrict__ off, uint32_t n,
                             uint32_t tbits, OrderOut o, uint32_t *list, unsigned *nlist) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = blockIdx.x * static_cast<uint64_t>(blockDim.x); base < n;
         base += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t v = base + threadIdx.x;
        uint64_t b0 = 0, s = 0;
        if (v < n) {
            b0 = off[v];
            s = off[v + 1] - b0;
        }
        if (s > 0 && s <= kThreadSeg) {
            uint64_t a[kThreadSeg];
#pragma unroll
            for (uint32_t i = 0; i < kThreadSeg; i++) a[i] = i < s ? tmp[b0 + i] : ~0ull;
#pragma unroll
            for (uint32_t round = 0; round < kThreadSeg; round++) {
#pragma unroll
                for (uint32_t i = round & 1; i + 1 < kThreadSeg; i += 2) cswap(a[i], a[i + 1]);
            }
            const uint64_t vhi = v << tbits;
#pragma unroll
            for (uint32_t i = 0; i < kThreadSeg; i++)
                if (i < s) put(o, b0 + i, vhi, a[i]);
        }
        // warp-aggregated appends to the two lists
        const bool mid = s > kThreadSeg && s <= kWarpSeg, big = s > kWarpSeg;
        const unsigned mb = __ballot_sync(kFull, mid), bb = __ballot_sync(kFull, big);
        unsigned m0 = 0, g0 = 0;
        if (lane == 0) {
            if (mb) m0 = atomicAdd(&nlist[0], __popc(mb));
            if (bb) g0 = atomicAdd(&nlist[1], __popc(bb));
        }
        m0 = __shfl_sync(kFull, m0, 0);
        g0 = __shfl_sync(kFull, g0, 0);
        if (mid) list[m0 + __popc(mb & lanemask_lt())] = static_cast<uint32_t>(v);
        if (big) list[n - 1 - (g0 + __popc(bb & lanemask_lt()))] = static_cast<uint32_t>(v);
    }
}

// One warp per listed node of kThreadSeg < s <= kWarpSeg records: bitonic
// network across the 32 lanes, padded with all-ones keys.
__global__ void k_node_order_warp(const uint64_t *__restrict__ tmp, const uint64_t *__restrict__ off,
                                  const uint32_t *__restrict__ list, const unsigned *__restrict__ nlist,
                                  uint32_t tbits, OrderOut o) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t cnt = nlist[0];
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < cnt; w += warps) {
        const uint64_t v = list[w];
        const uint64_t b0 = off[v], s = off[v + 1] - b0;
        uint64_t x = lane < s ? tmp[b0 + lane] : ~0ull;
#pragma unroll
        for (uint32_t kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                const uint64_t y = __shfl_xor_sync(kFull, x, j);
                const bool up = (lane & kk) == 0, lower = (lane & j) == 0;
                x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
            }
        }
        if (lane < s) put(o, b0 + lane, v << tbits, x);
    }
}

// One block per listed node of more than kWarpSeg records: mark the node's
// words in a bitmap of 2^tbits bits, prefix-count it, and write each record
// at the number of marked words below its own.
__global__ void __launch_bounds__(kBigThreads)
    k_node_order_block(const uint64_t *__restrict__ tmp, const uint64_t *__restrict__ off,
                       const uint32_t *__restrict__ list, const unsigned *__restrict__ nlist, uint32_t n,
                       uint32_t tbits, OrderOut o) {
    extern __shared__ uint32_t sm[];
    __shared__ uint32_t wsum[kBigThreads / 32];
    const uint32_t words = tbits > 5 ? 1u << (tbits - 5) : 1u;
    uint32_t *bm = sm, *pre = sm + words;
    const uint32_t per = (words + kBigThreads - 1) / kBigThreads;
    const uint32_t cnt = nlist[1];
    for (uint32_t q = blockIdx.x; q < cnt; q += gridDim.x) {
        const uint64_t v = list[n - 1 - q];
        const uint64_t b0 = off[v], s = off[v + 1] - b0;
        for (uint32_t w = threadIdx.x; w < words; w += kBigThreads) bm[w] = 0;
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < s; i += kBigThreads) {
            const uint32_t t = static_cast<uint32_t>(tmp[b0 + i] >> 32);
            atomicOr(&bm[t >> 5], 1u << (t & 31));
        }
        __syncthreads();
        // exclusive prefix of the per-word counts: thread th owns words
        // [th * per, th * per + per)
        const uint32_t w0 = threadIdx.x * per;
        uint32_t tot = 0;
        for (uint32_t w = w0; w < w0 + per && w < words; w++) tot += __popc(bm[w]);
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if ((threadIdx.x & 31) >= static_cast<unsigned>(o)) inc += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
        __syncthreads();
        uint32_t run = inc - tot;
        for (uint32_t w = 0; w < (threadIdx.x >> 5); w++) run += wsum[w];
        for (uint32_t w = w0; w < w0 + per && w < words; w++) {
            pre[w] = run;
            run += __popc(bm[w]);
        }
        __syncthreads();
        const uint64_t vhi = v << tbits;
        for (uint64_t i = threadIdx.x; i < s; i += kBigThreads) {
            const uint64_t p = tmp[b0 + i];
            const uint32_t t = static_cast<uint32_t>(p >> 32);
            const uint32_t pos = pre[t >> 5] + __popc(bm[t >> 5] & ((1u << (t & 31)) - 1));
            put(o, b0 + pos, vhi, p);
        }
        __syncthreads();
    }
}

inline size_t block_smem(uint32_t tbits) {
    const size_t words = tbits > 5 ? size_t{1} << (tbits - 5) : 1;
    return 2 * words * sizeof(uint32_t);
}

}  // namespace

cudaError_t launch_node_sort(uint64_t *rec_key, uint32_t *rec_val, uint64_t R, uint32_t tbits, uint32_t n,
                             uint64_t *cnt, uint64_t *off, uint64_t *tmp, uint32_t *list, unsigned *nlist,
                             void *scan_ws, cudaStream_t s) {
    const OrderOut o{rec_key, rec_val};
    // empty batch: off must still read all zeros for the acceptance
    cudaError_t e = cudaMemsetAsync(nlist, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (R) {
        note_launch();
        k_node_count<<<grid_for(R, 256), 256, 0, s>>>(rec_key, R, tbits, reinterpret_cast<unsigned long long *>(cnt));
    }
    // off[v] = records of nodes < v; off[n] = R (cnt[n] stays 0)
    e = exclusive_scan_u64(cnt, off, static_cast<size_t>(n) + 1, nullptr, scan_ws, s);
    if (e != cudaSuccess || R == 0) return e;
    note_launch();
    k_node_scatter<<<grid_for(R, 256), 256, 0, s>>>(rec_key, rec_val, R, tbits, off,
                                                    reinterpret_cast<unsigned long long *>(cnt), tmp);
    note_launch();
    k_node_order<<<grid_for(n, 256), 256, 0, s>>>(tmp, off, n, tbits, o, list, nlist);
    note_launch();
    k_node_order_warp<<<152 * 4, 256, 0, s>>>(tmp, off, list, nlist, tbits, o);
    const size_t smem = block_smem(tbits);  // up to 128 KB (19 word bits)
    e = cudaFuncSetAttribute(k_node_order_block, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    note_launch();
    k_node_order_block<<<SKIM_BIG_BLOCKS, kBigThreads, smem, s>>>(tmp, off, list, nlist, n, tbits, o);
    return cudaGetLastError();
}

}  // namespace skim

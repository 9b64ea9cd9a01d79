// graph.cu -- graph setup (CSR in both directions, weighted-cascade
// thresholds) and the rank order of all node-instance pairs (Section 3; the
// "shuffle" of Algorithms 1 and 2 read as increasing rank order).
#include "internal.cuh"
#include "prims.cuh"

namespace skim {

namespace {

inline unsigned grid_for(size_t n, int threads, unsigned cap = 152 * 32) {
    size_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g ? g : 1);
}

// Canonical edge list: ids < n, no self-loop, strictly increasing (src,dst).
__global__ void k_check_edges(const uint32_t *src, const uint32_t *dst, uint64_t m, uint32_t n, unsigned *bad) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint32_t u = src[e], v = dst[e];
        bool ok = u < n && v < n && u != v;
        if (ok && e > 0) {
            uint64_t a = (static_cast<uint64_t>(src[e - 1]) << 32) | dst[e - 1];
            uint64_t b = (static_cast<uint64_t>(u) << 32) | v;
            ok = a < b;
        }
        if (!ok) atomicOr(bad, 1u);
    }
}

__global__ void k_degree_count(const uint32_t *idx, uint64_t m, uint64_t *deg) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long *>(&deg[idx[e]]), 1ull);
}

__global__ void k_u64_to_u32(const uint64_t *in, uint32_t *out, size_t n) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        out[i] = static_cast<uint32_t>(in[i]);
}

__global__ void k_make_rev_keys(const uint32_t *src, const uint32_t *dst, uint64_t m, uint64_t *key, uint32_t *val) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        key[e] = (static_cast<uint64_t>(dst[e]) << 32) | src[e];
        val[e] = static_cast<uint32_t>(e);  // forward CSR position (the input is sorted by (src, dst))
    }
}

// reverse CSR from the (dst, src)-sorted keys: column (src), row (dst) and the
// edge's forward CSR position
__global__ void k_split_rev(const uint64_t *key, const uint32_t *val, uint64_t m, uint32_t *rcol, uint32_t *rrow,
                            uint32_t *rev2fwd) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        rcol[e] = static_cast<uint32_t>(key[e]);
        rrow[e] = static_cast<uint32_t>(key[e] >> 32);
        rev2fwd[e] = val[e];
    }
}

__global__ void k_wc_thresholds(const uint32_t *rptr, uint32_t n, uint64_t *thr) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = rptr[v + 1] - rptr[v];
        thr[v] = d ? (~0ull) / d : 0ull;
    }
}

__global__ void k_edge_states(const uint32_t *ptr, const uint32_t *col, uint32_t n, uint64_t coin_key, int reverse,
                              uint64_t *he) {
    // one warp per row
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        for (uint32_t e = ptr[v] + lane; e < ptr[v + 1]; e += 32) {
            const uint32_t c = col[e];
            he[e] = reverse ? edge_state(coin_key, c, v) : edge_state(coin_key, v, c);
        }
    }
}

// ---- materialised instances ------------------------------------------------
// Live threshold of CSR edge e in row r with other end x (the head of the edge
// is r in the reverse CSR and x in the forward one).
SKIM_DEV uint64_t row_edge_tm1(const CoinModel &cm, const uint64_t *tm1e, uint64_t e, uint32_t r, uint32_t x,
                               int reverse) {
    const uint32_t head = reverse ? r : x, tail = reverse ? x : r;
    if (cm.model == 3) return tm1e[e];
    if (cm.model == 0) return cm.tm1_uniform;
    if (cm.model == 1) return cm.thr_wc[head];
    return cm.tm1_class[fmix(cm.prob_key ^ ((static_cast<uint64_t>(tail) << 32) | head)) % 3u];
}

// One thread per edge (reverse CSR order): bit i of the mask is the coin of
// the edge in instance i, fmix(he + (i+1) G) <= tm1 (two independent chains
// per step).  The mask is stored at the edge's reverse and forward positions.
__global__ void k_live_masks(const uint32_t *rrow, const uint32_t *rcol, const uint64_t *rhe, const uint64_t *rtm1,
                             const uint32_t *rev2fwd, CoinModel cm, uint64_t m, uint32_t l, uint64_t *rmask,
                             uint64_t *fmask) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t t1 = row_edge_tm1(cm, rtm1, e, rrow[e], rcol[e], 1);
        const uint64_t h = rhe[e];
        uint64_t mk = 0;
        uint32_t i = 0;
        for (; i + 1 < l; i += 2) {
            const uint64_t c0 = fmix(h + kGolden * (i + 1)), c1 = fmix(h + kGolden * (i + 2));
            mk |= (static_cast<uint64_t>(c0 <= t1) << i) | (static_cast<uint64_t>(c1 <= t1) << (i + 1));
        }
        if (i < l) mk |= static_cast<uint64_t>(fmix(h + kGolden * (i + 1)) <= t1) << i;
        rmask[e] = mk;
        fmask[rev2fwd[e]] = mk;
    }
}

// One warp per node v, tiles of 32 in-edges (one per lane): for instance b
// the tile holds popc(ballot(bit b)) live in-edges; lane b % 32 keeps the
// counts of instances b < 32 and b >= 32.
__global__ void k_live_count(const uint32_t *rptr, const uint64_t *rmask, uint32_t n, uint32_t l, uint64_t *off) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        uint64_t c0 = 0, c1 = 0;
        const uint32_t e1 = rptr[v + 1];
        for (uint32_t e0 = rptr[v]; e0 < e1; e0 += 32) {
            const uint64_t mk = e0 + lane < e1 ? rmask[e0 + lane] : 0;
            uint64_t any = mk;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(kFull, any, o);
            for (uint64_t bits = any; bits; bits &= bits - 1) {
                const uint32_t b = __ffsll(bits) - 1;
                const uint32_t c = __popc(__ballot_sync(kFull, (mk >> b) & 1ull));
                if (lane == (b & 31)) {
                    if (b < 32) c0 += c;
                    else c1 += c;
                }
            }
        }
        const uint64_t base = static_cast<uint64_t>(v) * l;
        if (lane < l) off[base + lane] = c0;
        if (lane + 32 < l) off[base + lane + 32] = c1;
    }
}

// Same tiles: the live in-neighbours of (v, b) are written in row order from
// off[v*l + b] on; lane b % 32 keeps the write cursors of instances b, b + 32.
__global__ void k_live_fill(const uint32_t *rptr, const uint32_t *rcol, const uint64_t *rmask, uint32_t n,
                            uint32_t l, const uint64_t *off, uint32_t *live) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        const uint64_t base = static_cast<uint64_t>(v) * l;
        uint64_t p0 = lane < l ? off[base + lane] : 0, p1 = lane + 32 < l ? off[base + lane + 32] : 0;
        const uint32_t e1 = rptr[v + 1];
        for (uint32_t e0 = rptr[v]; e0 < e1; e0 += 32) {
            const bool in = e0 + lane < e1;
            const uint64_t mk = in ? rmask[e0 + lane] : 0;
            const uint32_t w = in ? rcol[e0 + lane] : 0;
            uint64_t any = mk;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(kFull, any, o);
            for (uint64_t bits = any; bits; bits &= bits - 1) {
                const uint32_t b = __ffsll(bits) - 1;
                const unsigned bb = __ballot_sync(kFull, (mk >> b) & 1ull);
                const uint64_t cur = __shfl_sync(kFull, b < 32 ? p0 : p1, b & 31);
                if ((mk >> b) & 1ull) live[cur + __popc(bb & lanemask_lt())] = w;
                if (lane == (b & 31)) {
                    if (b < 32) p0 += __popc(bb);
                    else p1 += __popc(bb);
                }
            }
        }
    }
}

__global__ void k_max_degree(const uint32_t *ptr, uint32_t n, unsigned long long *out) {
    unsigned long long best = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        best = max(best, static_cast<unsigned long long>(ptr[v + 1] - ptr[v]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// ---- rank order ---------------------------------------------------------
constexpr int kBucketCap = 4096;     // pairs sorted in shared memory per bucket
constexpr int kBucketThreads = 512;
constexpr uint64_t kBucketMean = 1024;  // target mean bucket size

SKIM_DEV uint64_t rank_of(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t x) {
    return rbase ? fmix(rbase[x / l] + kGolden * (x % l)) : pair_rank(rank_key, x);
}

// Sort keys of the rank order.  An element x is sorted by key(x) inside
// bucket(x); buckets are laid out in the order of the result.
//  UniformKeys: x = v*l + i, the uniform rank r(v,i) (Section 3); the output
//    rank is the key itself.
//  ChunkKeys: structured permutation (Section 3.1) and IC-model positions
//    (Section 3.2): x = c*n + v, chunk c first, then w(v,c) = fmix(K_w + G x);
//    the output rank is the position, the output pair (v, sigma_v(c)) or, in
//    the IC model (sigma null), the node v.
struct UniformKeys {
    uint64_t rank_key;
    const uint64_t *rbase;
    uint32_t l;
    int bb;
    SKIM_DEV uint64_t key(uint64_t x) const { return rank_of(rank_key, rbase, l, x); }
    SKIM_DEV uint64_t bucket(uint64_t, uint64_t key) const { return bb ? (key >> (64 - bb)) : 0; }
    SKIM_DEV uint64_t out_rank(uint64_t, uint64_t key) const { return key; }
    SKIM_DEV uint32_t out_pair(uint64_t x) const { return static_cast<uint32_t>(x); }
};

struct ChunkKeys {
    uint64_t kw;
    uint32_t n, l;
    int bb;                // bucket bits per chunk
    const uint8_t *sigma;  // sigma[v*l + c]: node v's instance in chunk c (null: IC model)
    SKIM_DEV uint64_t key(uint64_t x) const { return fmix(kw + kGolden * x); }
    SKIM_DEV uint64_t bucket(uint64_t x, uint64_t key) const {
        return ((x / n) << bb) | (bb ? (key >> (64 - bb)) : 0);
    }
    SKIM_DEV uint64_t out_rank(uint64_t pos, uint64_t) const { return pos; }
    SKIM_DEV uint32_t out_pair(uint64_t x) const {
        const uint32_t v = static_cast<uint32_t>(x % n);
        if (!sigma) return v;
        const uint64_t c = x / n;
        return v * l + sigma[static_cast<uint64_t>(v) * l + c];
    }
};

template <class K>
__global__ void k_rank_count(K kf, uint64_t total, unsigned long long *cnt) {
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[kf.bucket(x, kf.key(x))], 1ull);
}

template <class K>
__global__ void k_rank_scatter(K kf, uint64_t total, const uint64_t *off, unsigned *fill, uint32_t *tmp) {
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < total;
         x += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t b = kf.bucket(x, kf.key(x));
        unsigned p = atomicAdd(&fill[b], 1u);
        tmp[off[b] + p] = static_cast<uint32_t>(x);
    }
}

// Sort one bucket by key.  Keys are distinct (each key map is a bijection of
// x), so a bucket larger than the shared-memory capacity can be placed by
// counting smaller keys; that path is correct for any size and only its speed
// depends on the (uniform) bucket sizes.
template <class K>
__global__ void __launch_bounds__(kBucketThreads) k_bucket_sort(K kf, const uint64_t *off, const uint32_t *tmp,
                                                                uint64_t *sorted_rank, uint32_t *sorted_pair) {
    __shared__ uint64_t key[kBucketCap];
    __shared__ uint32_t val[kBucketCap];
    const uint64_t b0 = off[blockIdx.x], b1 = off[blockIdx.x + 1];
    const uint32_t s = static_cast<uint32_t>(b1 - b0);
    if (s == 0) return;
    if (s <= kBucketCap) {
        uint32_t P = 1;
        while (P < s) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
            if (i < s) {
                uint32_t x = tmp[b0 + i];
                val[i] = x;
                key[i] = kf.key(x);
            } else {
                key[i] = ~0ull;
                val[i] = 0;
            }
        }
        __syncthreads();
        for (uint32_t kk = 2; kk <= P; kk <<= 1) {
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                    uint32_t p = i ^ j;
                    if (p > i) {
                        bool up = (i & kk) == 0;
                        uint64_t a = key[i], c = key[p];
                        if ((a > c) == up) {
                            key[i] = c; key[p] = a;
                            uint32_t t = val[i]; val[i] = val[p]; val[p] = t;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
            sorted_rank[b0 + i] = kf.out_rank(b0 + i, key[i]);
            sorted_pair[b0 + i] = kf.out_pair(val[i]);
        }
        return;
    }
    // oversize bucket: keys to the output rank slots, then place elements by count
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) sorted_rank[b0 + i] = kf.key(tmp[b0 + i]);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
        uint64_t r = sorted_rank[b0 + i];
        uint32_t pos = 0;
        for (uint32_t j = 0; j < s; j++) pos += sorted_rank[b0 + j] < r;
        sorted_pair[b0 + pos] = tmp[b0 + i];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
        const uint32_t x = sorted_pair[b0 + i];
        sorted_rank[b0 + i] = kf.out_rank(b0 + i, kf.key(x));
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) sorted_pair[b0 + i] = kf.out_pair(sorted_pair[b0 + i]);
}

// Section 3.1: sigma[v*l + c] = the instance of node v with the (c+1)-th
// smallest rank r(v,i); one warp per node, l <= 64 keys in two registers.
__global__ void k_perm_sigma(uint64_t rank_key, uint32_t n, uint32_t l, uint8_t *sigma) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t v = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t base = v * l;
        const uint64_t k0 = lane < l ? pair_rank(rank_key, base + lane) : ~0ull;
        const uint64_t k1 = lane + 32 < l ? pair_rank(rank_key, base + lane + 32) : ~0ull;
        uint32_t c0 = 0, c1 = 0;
        for (uint32_t j = 0; j < l; j++) {
            const uint64_t kj = __shfl_sync(kFull, j < 32 ? k0 : k1, j & 31);
            c0 += kj < k0;
            c1 += kj < k1;
        }
        if (lane < l) sigma[base + c0] = static_cast<uint8_t>(lane);
        if (lane + 32 < l) sigma[base + c1] = static_cast<uint8_t>(lane + 32);
    }
}

// ---- graphs of a batch -----------------------------------------------------
__global__ void k_node_graph(const uint32_t *node_off, uint32_t count, uint32_t *node_graph) {
    for (uint32_t g = blockIdx.x; g < count; g += gridDim.x)
        for (uint32_t v = node_off[g] + threadIdx.x; v < node_off[g + 1]; v += blockDim.x) node_graph[v] = g;
}

__global__ void k_edge_states_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, BatchDesc b, int reverse,
                                    uint64_t *he) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t g = b.node_graph[v], o = b.node_off[g];
        for (uint32_t e = ptr[v] + lane; e < ptr[v + 1]; e += 32) {
            const uint32_t c = col[e] - o, r = v - o;  // ids inside the graph
            he[e] = reverse ? edge_state(b.coin_key[g], c, r) : edge_state(b.coin_key[g], r, c);
        }
    }
}

__global__ void k_edge_tm1_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, BatchDesc b,
                                 const uint64_t *thr_wc, int reverse, uint64_t *tm1) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t g = b.node_graph[v], o = b.node_off[g];
        const int model = b.model[g];
        for (uint32_t e = ptr[v] + lane; e < ptr[v + 1]; e += 32) {
            const uint32_t c = col[e];
            const uint32_t head = reverse ? v : c;
            const uint32_t tu = (reverse ? c : v) - o, tv = head - o;  // edge (tu -> tv) inside the graph
            uint64_t t;
            if (model == 0)
                t = b.tm1_uniform[g];
            else if (model == 1)
                t = thr_wc[head];
            else
                t = b.tm1_class[fmix(b.prob_key[g] ^ ((static_cast<uint64_t>(tu) << 32) | tv)) % 3u];
            tm1[e] = t;
        }
    }
}

__global__ void k_rank_bases(BatchDesc b, uint32_t n, uint32_t l, uint64_t *rbase) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t g = b.node_graph[v];
        rbase[v] = b.rank_key[g] + kGolden * (static_cast<uint64_t>(v - b.node_off[g]) * l);
    }
}

int bucket_bits(uint64_t nl) {
    int bb = 0;
    while (bb < 40 && (nl >> bb) > kBucketMean) bb++;
    return bb;
}

}  // namespace

cudaError_t launch_check_edges(const uint32_t *src, const uint32_t *dst, uint64_t m, uint32_t n, unsigned *bad,
                               cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_check_edges<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, n, bad);
    return cudaGetLastError();
}
cudaError_t launch_degree_count(const uint32_t *idx, uint64_t m, uint64_t *deg, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_degree_count<<<grid_for(m, 256), 256, 0, s>>>(idx, m, deg);
    return cudaGetLastError();
}
cudaError_t launch_u64_to_u32(const uint64_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    note_launch();
    k_u64_to_u32<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_make_rev_keys(const uint32_t *src, const uint32_t *dst, uint64_t m, uint64_t *key, uint32_t *val,
                                 cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_make_rev_keys<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, key, val);
    return cudaGetLastError();
}
cudaError_t launch_split_rev(const uint64_t *key, const uint32_t *val, uint64_t m, uint32_t *rcol, uint32_t *rrow,
                             uint32_t *rev2fwd, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_split_rev<<<grid_for(m, 256), 256, 0, s>>>(key, val, m, rcol, rrow, rev2fwd);
    return cudaGetLastError();
}
cudaError_t launch_wc_thresholds(const uint32_t *rptr, uint32_t n, uint64_t *thr, cudaStream_t s) {
    note_launch();
    k_wc_thresholds<<<grid_for(n, 256), 256, 0, s>>>(rptr, n, thr);
    return cudaGetLastError();
}
cudaError_t launch_edge_states(const uint32_t *ptr, const uint32_t *col, uint32_t n, uint64_t coin_key, int reverse,
                               uint64_t *he, cudaStream_t s) {
    note_launch();
    k_edge_states<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(ptr, col, n, coin_key, reverse, he);
    return cudaGetLastError();
}

cudaError_t launch_live_masks(const uint32_t *rrow, const uint32_t *rcol, const uint64_t *rhe, const uint64_t *rtm1,
                              const uint32_t *rev2fwd, const CoinModel &cm, uint64_t m, uint32_t l, uint64_t *rmask,
                              uint64_t *fmask, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_live_masks<<<grid_for(m, 256), 256, 0, s>>>(rrow, rcol, rhe, rtm1, rev2fwd, cm, m, l, rmask, fmask);
    return cudaGetLastError();
}
cudaError_t launch_live_count(const uint32_t *rptr, const uint64_t *rmask, uint32_t n, uint32_t l, uint64_t *off,
                              cudaStream_t s) {
    note_launch();
    k_live_count<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(rptr, rmask, n, l, off);
    return cudaGetLastError();
}
cudaError_t launch_live_fill(const uint32_t *rptr, const uint32_t *rcol, const uint64_t *rmask, uint32_t n, uint32_t l,
                             const uint64_t *off, uint32_t *live, cudaStream_t s) {
    note_launch();
    k_live_fill<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(rptr, rcol, rmask, n, l, off, live);
    return cudaGetLastError();
}

cudaError_t launch_max_degree(const uint32_t *ptr, uint32_t n, unsigned long long *out, cudaStream_t s) {
    note_launch();
    k_max_degree<<<grid_for(n, 256), 256, 0, s>>>(ptr, n, out);
    return cudaGetLastError();
}

cudaError_t launch_node_graph(const uint32_t *node_off, uint32_t count, uint32_t *node_graph, cudaStream_t s) {
    note_launch();
    k_node_graph<<<count < 4096 ? count : 4096, 256, 0, s>>>(node_off, count, node_graph);
    return cudaGetLastError();
}
cudaError_t launch_edge_states_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, const BatchDesc &b,
                                     int reverse, uint64_t *he, cudaStream_t s) {
    note_launch();
    k_edge_states_batch<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(ptr, col, n, b, reverse, he);
    return cudaGetLastError();
}
cudaError_t launch_edge_tm1_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, const BatchDesc &b,
                                  const uint64_t *thr_wc, int reverse, uint64_t *tm1, cudaStream_t s) {
    note_launch();
    k_edge_tm1_batch<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(ptr, col, n, b, thr_wc, reverse, tm1);
    return cudaGetLastError();
}
cudaError_t launch_rank_bases(const BatchDesc &b, uint32_t n, uint32_t l, uint64_t *rbase, cudaStream_t s) {
    note_launch();
    k_rank_bases<<<grid_for(n, 256), 256, 0, s>>>(b, n, l, rbase);
    return cudaGetLastError();
}

namespace {

struct SortSpace {
    uint64_t *cnt, *off;
    unsigned *fill;
    uint32_t *tmp;
    void *scan;
};

size_t sort_space_bytes(uint64_t nb, uint64_t total) {
    size_t b = (nb + 1) * sizeof(uint64_t) * 2 + nb * sizeof(unsigned) + total * sizeof(uint32_t);
    return b + scan_workspace_bytes(nb + 1) + 1024;
}

SortSpace carve(void *ws, uint64_t nb, uint64_t total) {
    SortSpace sp;
    char *p = static_cast<char *>(ws);
    sp.cnt = reinterpret_cast<uint64_t *>(p); p += (nb + 1) * sizeof(uint64_t);
    sp.off = reinterpret_cast<uint64_t *>(p); p += (nb + 1) * sizeof(uint64_t);
    sp.fill = reinterpret_cast<unsigned *>(p); p += nb * sizeof(unsigned);
    sp.tmp = reinterpret_cast<uint32_t *>(p); p += total * sizeof(uint32_t);
    sp.scan = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(p) + 255) & ~static_cast<uintptr_t>(255));
    return sp;
}

template <class K>
cudaError_t bucket_sort_all(const K &kf, uint64_t total, uint64_t nb, const SortSpace &sp, uint64_t *sorted_rank,
                            uint32_t *sorted_pair, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sp.cnt, 0, (nb + 1) * sizeof(uint64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sp.fill, 0, nb * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_count<<<grid_for(total, 256), 256, 0, s>>>(kf, total, reinterpret_cast<unsigned long long *>(sp.cnt));
    // off[b] = exclusive prefix; off[nb] = total (scan over nb+1 entries with cnt[nb] = 0)
    e = exclusive_scan_u64(sp.cnt, sp.off, nb + 1, nullptr, sp.scan, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_scatter<<<grid_for(total, 256), 256, 0, s>>>(kf, total, sp.off, sp.fill, sp.tmp);
    note_launch();
    k_bucket_sort<<<static_cast<unsigned>(nb), kBucketThreads, 0, s>>>(kf, sp.off, sp.tmp, sorted_rank, sorted_pair);
    return cudaGetLastError();
}

}  // namespace

size_t rank_sort_workspace_bytes(uint64_t nl) { return sort_space_bytes(1ull << bucket_bits(nl), nl); }

cudaError_t rank_sort(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t nl, uint64_t *sorted_rank,
                      uint32_t *sorted_pair, void *ws, cudaStream_t s) {
    if (nl == 0) return cudaSuccess;
    const int bb = bucket_bits(nl);
    const uint64_t nb = 1ull << bb;
    UniformKeys kf{rank_key, rbase, l, bb};
    return bucket_sort_all(kf, nl, nb, carve(ws, nb, nl), sorted_rank, sorted_pair, s);
}

uint64_t perm_key(uint64_t rank_key) { return fmix(rank_key ^ kPermSalt); }

size_t perm_sort_workspace_bytes(uint32_t n, uint32_t l, uint32_t chunks, bool ic) {
    const uint64_t nb = static_cast<uint64_t>(chunks) << bucket_bits(n);
    const uint64_t total = static_cast<uint64_t>(chunks) * n;
    return sort_space_bytes(nb, total) + (ic ? 0 : static_cast<size_t>(n) * l) + 256;
}

cudaError_t perm_sort(uint64_t rank_key, uint32_t n, uint32_t l, uint32_t chunks, bool ic, uint64_t *sorted_rank,
                      uint32_t *sorted_pair, void *ws, cudaStream_t s) {
    const uint64_t total = static_cast<uint64_t>(chunks) * n;
    if (total == 0) return cudaSuccess;
    const int bb = bucket_bits(n);
    const uint64_t nb = static_cast<uint64_t>(chunks) << bb;
    uint8_t *sigma = nullptr;
    char *rest = static_cast<char *>(ws);
    if (!ic) {
        sigma = reinterpret_cast<uint8_t *>(rest);
        rest += (static_cast<size_t>(n) * l + 255) & ~static_cast<size_t>(255);
        note_launch();
        k_perm_sigma<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(rank_key, n, l, sigma);
    }
    ChunkKeys kf{perm_key(rank_key), n, l, bb, sigma};
    return bucket_sort_all(kf, total, nb, carve(rest, nb, total), sorted_rank, sorted_pair, s);
}

}  // namespace skim

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

// Keys for the reverse CSR: (src << 32 | dst).  The input is sorted by
// (src, dst), so a stable sort on the dst bits alone yields (dst, src) order.
__global__ void k_make_rev_keys(const uint32_t *src, const uint32_t *dst, uint64_t m, uint64_t *key, uint32_t *val) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        key[e] = (static_cast<uint64_t>(src[e]) << 32) | dst[e];
        val[e] = static_cast<uint32_t>(e);  // forward CSR position
    }
}

// reverse CSR from the (dst, src)-ordered keys: column (src), row (dst) and the
// edge's forward CSR position
__global__ void k_split_rev(const uint64_t *key, const uint32_t *val, uint64_t m, uint32_t *rcol, uint32_t *rrow,
                            uint32_t *rev2fwd) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        rcol[e] = static_cast<uint32_t>(key[e] >> 32);
        rrow[e] = static_cast<uint32_t>(key[e]);
        rev2fwd[e] = val[e];
    }
}

// CSR row pointers of a row-sorted edge array: ptr[v] = the first edge whose
// row is at least v (a binary search per node), ptr[n] = m.
__global__ void k_row_ptr(const uint32_t *row, uint64_t m, uint32_t n, uint32_t *ptr) {
    for (uint64_t v = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; v <= n;
         v += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (row[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        ptr[v] = static_cast<uint32_t>(lo);
    }
}

// Per-edge coin states of both CSR orders from the reverse one: an edge's
// state depends on (src, dst) only.
__global__ void k_edge_states_both(const uint32_t *rcol, const uint32_t *rrow, const uint32_t *rev2fwd, uint64_t m,
                                   uint64_t coin_key, uint64_t *rhe, uint64_t *fhe) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t h = edge_state(coin_key, rcol[e], rrow[e]);
        rhe[e] = h;
        fhe[rev2fwd[e]] = h;
    }
}

__global__ void k_wc_thresholds(const uint32_t *rptr, uint32_t n, uint64_t *thr) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = rptr[v + 1] - rptr[v];
        thr[v] = d ? (~0ull) / d : 0ull;
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

// Live rows from the masks.  A warp walks edges [e0, e1) of a row in tiles of
// 32 (one per lane); for instance b the tile holds popc(ballot(bit b)) live
// edges.  Lane b % 32 keeps the counts (or write cursors) of instances b < 32
// (c0) and b >= 32 (c1).  Rows of up to kBigRow edges take one warp; longer
// rows take a block of 8 warps on contiguous slices (kernels *_big).
constexpr uint32_t kBigRow = 2048;

// Rows longer than kBigRow are cut into pieces of kBigRow edges, one warp per
// piece: the row's pieces get consecutive ids (in edge order) when the count
// pass meets the row; each piece's per-instance counts are summed per row into
// off, with the exclusive prefix of every piece kept for the fill pass.
struct Pieces {
    uint32_t *row;      // node of each piece
    uint32_t *e0;       // first edge of each piece
    uint64_t *cnt;      // 64 per piece: live edges of each instance, then the prefix within the row
    unsigned *count;    // pieces in use
    uint32_t cap;
};

SKIM_DEV void claim_pieces(const Pieces &P, uint32_t v, uint32_t e0, uint32_t e1) {
    const uint32_t np = (e1 - e0 + kBigRow - 1) / kBigRow;
    const unsigned base = atomicAdd(P.count, np);
    for (uint32_t q = 0; q < np && base + q < P.cap; q++) {
        P.row[base + q] = v;
        P.e0[base + q] = e0 + q * kBigRow;
    }
}

// A tile of 32 edges (lane q holds edge q's 64-bit live mask) is turned into
// one word per instance by transposing the two 32 x 32 bit matrices across
// the warp: afterwards lane b holds, in bit q, whether edge q is live in
// instance b (lo) and in instance b + 32 (hi).  Step j swaps the off-diagonal
// j x j blocks of every 2j x 2j block: a lane without bit j keeps its columns
// without bit j and takes its partner's others shifted up, the partner the
// reverse.
SKIM_DEV uint32_t warp_transpose32(uint32_t x) {
    const uint32_t lane = threadIdx.x & 31;
    constexpr uint32_t lo_cols[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const uint32_t j = 16u >> s, lo = lo_cols[s];
        const uint32_t y = __shfl_xor_sync(kFull, x, j);
        x = (lane & j) ? ((x & ~lo) | ((y >> j) & lo)) : ((x & lo) | ((y << j) & ~lo));
    }
    return x;
}

SKIM_DEV void warp_count(const uint64_t *mask, uint32_t e0, uint32_t e1, uint64_t &c0, uint64_t &c1) {
    const uint32_t lane = threadIdx.x & 31;
    for (; e0 < e1; e0 += 32) {
        const uint64_t mk = e0 + lane < e1 ? mask[e0 + lane] : 0;
        c0 += __popc(warp_transpose32(static_cast<uint32_t>(mk)));
        c1 += __popc(warp_transpose32(static_cast<uint32_t>(mk >> 32)));
    }
}

// Writes the tile's live edges of instances lane and lane + 32 at p0 and p1,
// in edge order; the warp loops as often as the fullest instance needs.
SKIM_DEV void warp_fill(const uint64_t *mask, const uint32_t *col, uint32_t e0, uint32_t e1, uint64_t &p0,
                        uint64_t &p1, uint32_t *live) {
    const uint32_t lane = threadIdx.x & 31;
    for (; e0 < e1; e0 += 32) {
        const bool in = e0 + lane < e1;
        const uint64_t mk = in ? mask[e0 + lane] : 0;
        const uint32_t w = in ? col[e0 + lane] : 0;
        uint32_t m0 = warp_transpose32(static_cast<uint32_t>(mk));
        uint32_t m1 = warp_transpose32(static_cast<uint32_t>(mk >> 32));
        while (__any_sync(kFull, (m0 | m1) != 0)) {
            const uint32_t x0 = __shfl_sync(kFull, w, m0 ? __ffs(m0) - 1 : 0);
            const uint32_t x1 = __shfl_sync(kFull, w, m1 ? __ffs(m1) - 1 : 0);
            if (m0) {
                live[p0++] = x0;
                m0 &= m0 - 1;
            }
            if (m1) {
                live[p1++] = x1;
                m1 &= m1 - 1;
            }
        }
    }
}

// counts of live edges per (node, instance) into off[v*l + i], rows up to kBigRow
__global__ void k_live_count(const uint32_t *ptr, const uint64_t *mask, uint32_t n, uint32_t l, uint64_t *off,
                             Pieces P) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t e0 = ptr[v], e1 = ptr[v + 1];
        if (e1 - e0 > kBigRow) {  // counted by pieces (k_piece_*)
            if (lane == 0) claim_pieces(P, v, e0, e1);
            continue;
        }
        uint64_t c0 = 0, c1 = 0;
        warp_count(mask, e0, e1, c0, c1);
        const uint64_t base = static_cast<uint64_t>(v) * l;
        if (lane < l) off[base + lane] = c0;
        if (lane + 32 < l) off[base + lane + 32] = c1;
    }
}

// the live edges of (v, i) written in row order from off[v*l + i], rows up to kBigRow
__global__ void k_live_fill(const uint32_t *ptr, const uint32_t *col, const uint64_t *mask, uint32_t n, uint32_t l,
                            const uint64_t *off, uint32_t *live) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t e0 = ptr[v], e1 = ptr[v + 1];
        if (e1 - e0 > kBigRow) continue;
        const uint64_t base = static_cast<uint64_t>(v) * l;
        uint64_t p0 = lane < l ? off[base + lane] : 0, p1 = lane + 32 < l ? off[base + lane + 32] : 0;
        warp_fill(mask, col, e0, e1, p0, p1, live);
    }
}

__global__ void k_piece_count(const uint32_t *ptr, const uint64_t *mask, Pieces P) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t np = min(*P.count, P.cap);
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t v = P.row[p], e0 = P.e0[p], e1 = min(ptr[v + 1], e0 + kBigRow);
        uint64_t c0 = 0, c1 = 0;
        warp_count(mask, e0, e1, c0, c1);
        P.cnt[static_cast<uint64_t>(p) * 64 + lane] = c0;
        P.cnt[static_cast<uint64_t>(p) * 64 + lane + 32] = c1;
    }
}

// one warp per row (its first piece): per instance, the row's total into off
// and each piece's count replaced by the sum over the row's earlier pieces
__global__ void k_piece_rows(const uint32_t *ptr, uint32_t l, uint64_t *off, Pieces P) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t np = min(*P.count, P.cap);
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t v = P.row[p];
        if (P.e0[p] != ptr[v]) continue;  // not the row's first piece
        uint64_t r0 = 0, r1 = 0;
        for (uint32_t q = p; q < np && P.row[q] == v; q++) {
            uint64_t *c = P.cnt + static_cast<uint64_t>(q) * 64;
            const uint64_t a0 = c[lane], a1 = c[lane + 32];
            c[lane] = r0;
            c[lane + 32] = r1;
            r0 += a0;
            r1 += a1;
        }
        const uint64_t base = static_cast<uint64_t>(v) * l;
        if (lane < l) off[base + lane] = r0;
        if (lane + 32 < l) off[base + lane + 32] = r1;
    }
}

__global__ void k_piece_fill(const uint32_t *ptr, const uint32_t *col, const uint64_t *mask, uint32_t l,
                             const uint64_t *off, uint32_t *live, Pieces P) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t np = min(*P.count, P.cap);
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t v = P.row[p], e0 = P.e0[p], e1 = min(ptr[v + 1], e0 + kBigRow);
        const uint64_t base = static_cast<uint64_t>(v) * l;
        const uint64_t *c = P.cnt + static_cast<uint64_t>(p) * 64;
        uint64_t p0 = lane < l ? off[base + lane] + c[lane] : 0;
        uint64_t p1 = lane + 32 < l ? off[base + lane + 32] + c[lane + 32] : 0;
        warp_fill(mask, col, e0, e1, p0, p1, live);
    }
}

// ---- rank order ---------------------------------------------------------
constexpr int kBucketCap = 2048;     // pairs sorted in shared memory per bucket
constexpr int kBucketThreads = 256;
constexpr int kSubBits = 11;         // counting sort of a bucket on the next 11 key bits
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
    SKIM_DEV uint32_t sub(uint64_t key) const { return static_cast<uint32_t>((key << bb) >> (64 - kSubBits)); }
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
    SKIM_DEV uint32_t sub(uint64_t key) const { return static_cast<uint32_t>((key << bb) >> (64 - kSubBits)); }
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
// x) and uniform, so a bucket of up to kBucketCap elements is placed by a
// counting sort on the next kSubBits bits below the bucket's own, after which
// the few elements sharing a sub-bucket are put in order one sub-bucket per
// thread; all of it on a permutation in shared memory, so that the bucket is
// written to memory once.  A larger bucket is placed by counting smaller keys; that path is
// correct for any size and only its speed depends on the bucket sizes.
template <class K>
__global__ void __launch_bounds__(kBucketThreads) k_bucket_sort(K kf, const uint64_t *off, const uint32_t *tmp,
                                                                uint64_t *sorted_rank, uint32_t *sorted_pair) {
    constexpr int kSub = 1 << kSubBits;
    __shared__ uint64_t key[kBucketCap];
    __shared__ uint32_t val[kBucketCap];
    __shared__ uint32_t cnt[kSub];
    __shared__ uint16_t perm[kBucketCap];
    __shared__ uint32_t wsum[kBucketThreads / 32];
    const uint64_t b0 = off[blockIdx.x], b1 = off[blockIdx.x + 1];
    const uint32_t s = static_cast<uint32_t>(b1 - b0);
    if (s == 0) return;
    if (s <= kBucketCap) {
        for (uint32_t i = threadIdx.x; i < kSub; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
            const uint32_t x = tmp[b0 + i];
            const uint64_t kx = kf.key(x);
            val[i] = x;
            key[i] = kx;
            atomicAdd(&cnt[kf.sub(kx)], 1u);
        }
        __syncthreads();
        // exclusive scan of cnt: each thread owns kSub / blockDim.x consecutive counters
        constexpr int per = kSub / kBucketThreads;
        uint32_t loc[per], tot = 0;
#pragma unroll
        for (int q = 0; q < per; q++) {
            loc[q] = tot;
            tot += cnt[threadIdx.x * per + q];
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if ((threadIdx.x & 31) >= static_cast<unsigned>(o)) inc += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = inc;
        __syncthreads();
        uint32_t wbase = 0;
        for (uint32_t w = 0; w < (threadIdx.x >> 5); w++) wbase += wsum[w];
        const uint32_t tbase = wbase + inc - tot;
#pragma unroll
        for (int q = 0; q < per; q++) cnt[threadIdx.x * per + q] = tbase + loc[q];
        __syncthreads();
        // scatter positions (a permutation in shared memory); cnt[b] ends as
        // the end of sub-bucket b
        for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
            const uint32_t pos = atomicAdd(&cnt[kf.sub(key[i])], 1u);
            perm[pos] = static_cast<uint16_t>(i);
        }
        __syncthreads();
        // order inside the sub-buckets that hold more than one element
        for (uint32_t b = threadIdx.x; b < kSub; b += blockDim.x) {
            const uint32_t lo = b ? cnt[b - 1] : 0, hi = cnt[b];
            for (uint32_t i = lo + 1; i < hi; i++) {
                const uint16_t pi = perm[i];
                const uint64_t kx = key[pi];
                uint32_t j = i;
                for (; j > lo && key[perm[j - 1]] > kx; j--) perm[j] = perm[j - 1];
                perm[j] = pi;
            }
        }
        __syncthreads();
        // one coalesced write of the bucket
        for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
            const uint16_t pi = perm[i];
            sorted_rank[b0 + i] = kf.out_rank(b0 + i, key[pi]);
            sorted_pair[b0 + i] = kf.out_pair(val[pi]);
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
cudaError_t launch_row_ptr(const uint32_t *row, uint64_t m, uint32_t n, uint32_t *ptr, cudaStream_t s) {
    note_launch();
    k_row_ptr<<<grid_for(static_cast<size_t>(n) + 1, 256), 256, 0, s>>>(row, m, n, ptr);
    return cudaGetLastError();
}
cudaError_t launch_edge_states_both(const uint32_t *rcol, const uint32_t *rrow, const uint32_t *rev2fwd, uint64_t m,
                                    uint64_t coin_key, uint64_t *rhe, uint64_t *fhe, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_edge_states_both<<<grid_for(m, 256), 256, 0, s>>>(rcol, rrow, rev2fwd, m, coin_key, rhe, fhe);
    return cudaGetLastError();
}
cudaError_t launch_wc_thresholds(const uint32_t *rptr, uint32_t n, uint64_t *thr, cudaStream_t s) {
    note_launch();
    k_wc_thresholds<<<grid_for(n, 256), 256, 0, s>>>(rptr, n, thr);
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
size_t live_pieces_bytes(uint64_t m) {
    const uint64_t cap = 2 * (m / kBigRow) + 2;
    return cap * (4 + 4 + 64 * 8) + 256;
}

namespace {
Pieces carve_pieces(void *ws, uint64_t m) {
    Pieces P;
    const uint64_t cap = 2 * (m / kBigRow) + 2;
    char *p = static_cast<char *>(ws);
    P.cnt = reinterpret_cast<uint64_t *>(p); p += cap * 64 * 8;
    P.row = reinterpret_cast<uint32_t *>(p); p += cap * 4;
    P.e0 = reinterpret_cast<uint32_t *>(p); p += cap * 4;
    P.count = reinterpret_cast<unsigned *>((reinterpret_cast<uintptr_t>(p) + 15) & ~static_cast<uintptr_t>(15));
    P.cap = static_cast<uint32_t>(cap);
    return P;
}
unsigned piece_grid(uint64_t m) { return grid_for((2 * (m / kBigRow) + 2) * 32, 256, 152 * 8); }
}  // namespace

cudaError_t launch_live_count(const uint32_t *ptr, const uint64_t *mask, uint32_t n, uint64_t m, uint32_t l,
                              uint64_t *off, void *pieces_ws, cudaStream_t s) {
    const Pieces P = carve_pieces(pieces_ws, m);
    cudaError_t e = cudaMemsetAsync(P.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_live_count<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(ptr, mask, n, l, off, P);
    note_launch();
    k_piece_count<<<piece_grid(m), 256, 0, s>>>(ptr, mask, P);
    note_launch();
    k_piece_rows<<<piece_grid(m), 256, 0, s>>>(ptr, l, off, P);
    return cudaGetLastError();
}
cudaError_t launch_live_fill(const uint32_t *ptr, const uint32_t *col, const uint64_t *mask, uint32_t n, uint64_t m,
                             uint32_t l, const uint64_t *off, uint32_t *live, void *pieces_ws, cudaStream_t s) {
    const Pieces P = carve_pieces(pieces_ws, m);
    note_launch();
    k_live_fill<<<grid_for(static_cast<size_t>(n) * 32, 256), 256, 0, s>>>(ptr, col, mask, n, l, off, live);
    note_launch();
    k_piece_fill<<<piece_grid(m), 256, 0, s>>>(ptr, col, mask, l, off, live, P);
    return cudaGetLastError();
}

namespace {
__global__ void k_offsets_u32(const uint64_t *off, uint64_t count, uint32_t *off32) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r <= count;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        off32[r] = static_cast<uint32_t>(off[r]);
}
__global__ void k_clear_row_flags(uint32_t *off32, uint64_t count) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < count;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        off32[r] &= kRowMask;
}
}  // namespace

cudaError_t launch_offsets_u32(const uint64_t *off, uint64_t count, uint32_t *off32, cudaStream_t s) {
    note_launch();
    k_offsets_u32<<<grid_for(count + 1, 256), 256, 0, s>>>(off, count, off32);
    return cudaGetLastError();
}

cudaError_t launch_clear_row_flags(uint32_t *off32, uint64_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    note_launch();
    k_clear_row_flags<<<grid_for(count, 256), 256, 0, s>>>(off32, count);
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

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
        val[e] = 0;
    }
}

__global__ void k_split_rev(const uint64_t *key, uint64_t m, uint32_t *rcol) {
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < m;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        rcol[e] = static_cast<uint32_t>(key[e]);
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

__global__ void k_rank_count(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t nl, int bb,
                             unsigned long long *cnt) {
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < nl;
         x += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t r = rank_of(rank_key, rbase, l, x);
        uint64_t b = bb ? (r >> (64 - bb)) : 0;
        atomicAdd(&cnt[b], 1ull);
    }
}

__global__ void k_rank_scatter(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t nl, int bb,
                               const uint64_t *off, unsigned *fill, uint32_t *tmp) {
    for (uint64_t x = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; x < nl;
         x += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t r = rank_of(rank_key, rbase, l, x);
        uint64_t b = bb ? (r >> (64 - bb)) : 0;
        unsigned p = atomicAdd(&fill[b], 1u);
        tmp[off[b] + p] = static_cast<uint32_t>(x);
    }
}

// Sort one bucket by rank.  Ranks are distinct (the pair -> rank map is a
// bijection), so a bucket larger than the shared-memory capacity can be
// placed by counting smaller keys; that path is correct for any size and
// only its speed depends on the (uniform) bucket sizes.
__global__ void __launch_bounds__(kBucketThreads) k_bucket_sort(uint64_t rank_key, const uint64_t *rbase, uint32_t l,
                                                                const uint64_t *off, const uint32_t *tmp,
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
                key[i] = rank_of(rank_key, rbase, l, x);
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
            sorted_rank[b0 + i] = key[i];
            sorted_pair[b0 + i] = val[i];
        }
        return;
    }
    // oversize bucket: ranks to the output rank slots, then place pairs by count
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) sorted_rank[b0 + i] = rank_of(rank_key, rbase, l, tmp[b0 + i]);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) {
        uint64_t r = sorted_rank[b0 + i];
        uint32_t pos = 0;
        for (uint32_t j = 0; j < s; j++) pos += sorted_rank[b0 + j] < r;
        sorted_pair[b0 + pos] = tmp[b0 + i];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x)
        sorted_rank[b0 + i] = rank_of(rank_key, rbase, l, sorted_pair[b0 + i]);
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
cudaError_t launch_split_rev(const uint64_t *key, uint64_t m, uint32_t *rcol, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    note_launch();
    k_split_rev<<<grid_for(m, 256), 256, 0, s>>>(key, m, rcol);
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

size_t rank_sort_workspace_bytes(uint64_t nl) {
    uint64_t nb = 1ull << bucket_bits(nl);
    size_t b = (nb + 1) * sizeof(uint64_t) * 2 + nb * sizeof(unsigned) + nl * sizeof(uint32_t);
    return b + scan_workspace_bytes(nb + 1) + 1024;
}

cudaError_t rank_sort(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t nl, uint64_t *sorted_rank,
                      uint32_t *sorted_pair, void *ws, cudaStream_t s) {
    if (nl == 0) return cudaSuccess;
    const int bb = bucket_bits(nl);
    const uint64_t nb = 1ull << bb;
    char *p = static_cast<char *>(ws);
    uint64_t *cnt = reinterpret_cast<uint64_t *>(p); p += (nb + 1) * sizeof(uint64_t);
    uint64_t *off = reinterpret_cast<uint64_t *>(p); p += (nb + 1) * sizeof(uint64_t);
    unsigned *fill = reinterpret_cast<unsigned *>(p); p += nb * sizeof(unsigned);
    uint32_t *tmp = reinterpret_cast<uint32_t *>(p); p += nl * sizeof(uint32_t);
    p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(p) + 255) & ~static_cast<uintptr_t>(255));
    void *sws = p;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (nb + 1) * sizeof(uint64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, nb * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_count<<<grid_for(nl, 256), 256, 0, s>>>(rank_key, rbase, l, nl, bb, reinterpret_cast<unsigned long long *>(cnt));
    // off[b] = exclusive prefix; off[nb] = nl (scan over nb+1 entries with cnt[nb] = 0)
    e = exclusive_scan_u64(cnt, off, nb + 1, nullptr, sws, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_scatter<<<grid_for(nl, 256), 256, 0, s>>>(rank_key, rbase, l, nl, bb, off, fill, tmp);
    note_launch();
    k_bucket_sort<<<static_cast<unsigned>(nb), kBucketThreads, 0, s>>>(rank_key, rbase, l, off, tmp, sorted_rank,
                                                                   sorted_pair);
    return cudaGetLastError();
}

}  // namespace skim

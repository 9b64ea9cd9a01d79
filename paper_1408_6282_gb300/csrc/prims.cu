// prims.cu -- exclusive scan and stable LSD radix sort.
#include "common.cuh"
#include "prims.cuh"

namespace skim {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

__global__ void __launch_bounds__(kScanThreads) k_block_sums(const uint64_t *in, size_t n, uint64_t *bsum) {
    __shared__ uint64_t red[kScanThreads / 32];
    const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile;
    uint64_t s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        size_t i = base + it * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = t;
    }
}

// Scan one tile: striped load into shared memory, blocked per-thread scan,
// block-wide scan of thread totals, write out with the block offset.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const uint64_t *in, uint64_t *out, size_t n,
                                                            const uint64_t *block_off, uint64_t *total) {
    __shared__ uint64_t buf[kScanTile];
    __shared__ uint64_t wsum[kScanThreads / 32];
    const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        int j = it * kScanThreads + threadIdx.x;
        size_t i = base + j;
        buf[j] = i < n ? in[i] : 0;
    }
    __syncthreads();
    uint64_t v[kScanItems];
    uint64_t tsum = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        v[it] = buf[threadIdx.x * kScanItems + it];
        tsum += v[it];
    }
    // block exclusive scan of tsum
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kScanThreads / 32 ? wsum[lane] : 0;
        uint64_t z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, z, o);
            if (lane >= o) z += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = z - w;  // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1 && total) *total = z + (block_off ? block_off[blockIdx.x] : 0);
    }
    __syncthreads();
    uint64_t run = (block_off ? block_off[blockIdx.x] : 0) + wsum[warp] + (x - tsum);
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        buf[threadIdx.x * kScanItems + it] = run;
        run += v[it];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        int j = it * kScanThreads + threadIdx.x;
        size_t i = base + j;
        if (i < n) out[i] = buf[j];
    }
}

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t *keys, size_t n, int shift, uint64_t *hist,
                                                        size_t ntiles) {
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = static_cast<size_t>(blockIdx.x) * kRsTile;
#pragma unroll
    for (int it = 0; it < kRsItems; it++) {
        size_t i = base + it * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[static_cast<size_t>(threadIdx.x) * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t *keys, const uint32_t *vals, uint64_t *okeys,
                                                           uint32_t *ovals, size_t n, int shift, const uint64_t *offs,
                                                           size_t ntiles) {
    __shared__ unsigned wcnt[kRsWarps][256];
    __shared__ uint64_t goff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    goff[threadIdx.x] = offs[static_cast<size_t>(threadIdx.x) * ntiles + blockIdx.x];
    __syncwarp();
    const size_t base = static_cast<size_t>(blockIdx.x) * kRsTile + warp * (32 * kRsItems);
    uint64_t k[kRsItems];
    uint32_t val[kRsItems];
    unsigned pos[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; it++) {
        size_t i = base + it * 32 + lane;
        bool ok = i < n;
        k[it] = ok ? keys[i] : 0;
        val[it] = ok ? vals[i] : 0;
        unsigned d = ok ? static_cast<unsigned>((k[it] >> shift) & 0xff) : (0x100u + lane);
        unsigned peers = __match_any_sync(kFull, d);
        unsigned pre = ok ? wcnt[warp][d] : 0;
        __syncwarp();
        if (ok && (peers & lanemask_lt()) == 0) wcnt[warp][d] = pre + __popc(peers);
        __syncwarp();
        pos[it] = pre + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    {   // exclusive offsets across warps, one digit per thread
        unsigned run = 0;
        const int d = threadIdx.x;
#pragma unroll
        for (int w = 0; w < kRsWarps; w++) {
            unsigned c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; it++) {
        size_t i = base + it * 32 + lane;
        if (i < n) {
            unsigned d = static_cast<unsigned>((k[it] >> shift) & 0xff);
            size_t o = goff[d] + wcnt[warp][d] + pos[it];
            okeys[o] = k[it];
            ovals[o] = val[it];
        }
    }
}

inline size_t cdiv(size_t a, size_t b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_workspace_bytes(size_t n) {
    size_t total = 0;
    while (n > static_cast<size_t>(kScanTile)) {
        n = cdiv(n, kScanTile);
        total += n * sizeof(uint64_t);
    }
    return total + 256;
}

cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, size_t n, uint64_t *total, void *ws,
                               cudaStream_t s) {
    if (n == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
        return cudaSuccess;
    }
    size_t nb = cdiv(n, kScanTile);
    if (nb == 1) {
        note_launch();
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total);
        return cudaGetLastError();
    }
    uint64_t *bsum = static_cast<uint64_t *>(ws);
    note_launch();
    k_block_sums<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, bsum);
    cudaError_t e = exclusive_scan_u64(bsum, bsum, nb, total, bsum + nb, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_scan_tile<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, out, n, bsum, nullptr);
    return cudaGetLastError();
}

size_t radix_workspace_bytes(size_t n) {
    size_t ntiles = cdiv(n ? n : 1, kRsTile);
    size_t h = 256 * ntiles;
    return h * sizeof(uint64_t) + scan_workspace_bytes(h);
}

cudaError_t radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *alt_keys, uint32_t *alt_vals, size_t n,
                             int bits, void *ws, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    size_t ntiles = cdiv(n, kRsTile);
    uint64_t *hist = static_cast<uint64_t *>(ws);
    void *sws = hist + 256 * ntiles;
    uint64_t *sk = keys, *dk = alt_keys;
    uint32_t *sv = vals, *dv = alt_vals;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = p * 8;
        note_launch();
        k_rs_hist<<<static_cast<unsigned>(ntiles), kRsThreads, 0, s>>>(sk, n, shift, hist, ntiles);
        cudaError_t e = exclusive_scan_u64(hist, hist, 256 * ntiles, nullptr, sws, s);
        if (e != cudaSuccess) return e;
        note_launch();
        k_rs_scatter<<<static_cast<unsigned>(ntiles), kRsThreads, 0, s>>>(sk, sv, dk, dv, n, shift, hist, ntiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t *tk = sk; sk = dk; dk = tk;
        uint32_t *tv = sv; sv = dv; dv = tv;
    }
    if (sk != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, sk, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(vals, sv, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace skim

// query.cu -- influence oracle queries (Section 5.1, Eq. unionest).
//
// For a seed set S, every rank z of X_u minus {tau_u} (u in S) is charged
// 1/max{tau_u : z in X_u minus {tau_u}}; the sum estimates |union of R_u| and
// is divided by l.  tau_u is the k-th smallest rank of a full sketch and 1 for
// a sketch with fewer than k ranks (Eq. combinedthresh).
//
// A hash table per query in global scratch keeps, per distinct z, the
// largest tau (as a 64-bit integer; the integer order equals the order of
// the reals h/2^64 and the rounding to double is monotone).  Each term 1/tau is
// formed in double exactly as h -> double -> scale by 2^-64 -> 1/x, then added
// exactly in 192-bit fixed point (64 fraction bits suffice: every term is >= 1
// with a 53-bit significand) and the total is rounded to double once, to
// nearest-even.  The result therefore does not depend on the order in which
// ranks are visited, and a query gives the same bits alone or in a batch.
// With permutation ranks (Sections 3.1, 3.2) a sketch holds positions and a
// threshold q becomes the term (n*l - 1)/q, or n/q in the IC model, each
// formed as one double division (terms are at least 1/k >= 2^-8, so 64
// fraction bits still hold them exactly).
#include <algorithm>

#include "internal.cuh"

namespace skim {

namespace {

constexpr int kQThreads = 512;

struct U192 {
    uint64_t w[3];
};

SKIM_DEV void add192(U192 &a, const U192 &b) {
    uint64_t s0 = a.w[0] + b.w[0];
    uint64_t c0 = s0 < a.w[0];
    uint64_t s1 = a.w[1] + b.w[1];
    uint64_t c1 = s1 < a.w[1];
    s1 += c0;
    c1 |= (s1 < c0);
    a.w[0] = s0;
    a.w[1] = s1;
    a.w[2] = a.w[2] + b.w[2] + c1;
}

// term 1/tau for the integer threshold h (h = ~0 stands for tau = 1)
SKIM_DEV double inv_tau(uint64_t h) {
    double tau = ldexp(__ull2double_rn(h), -64);
    return 1.0 / tau;
}

// term of a threshold h under the context's rank reading (QueryTerms)
SKIM_DEV double term_of(const QueryTerms &t, uint64_t h) {
    if (t.mode == 0) return inv_tau(h);
    if (h == ~0ull) return t.mode == 2 ? 0.0 : 1.0;
    return t.num / __ull2double_rn(h);
}

// exact fixed-point image (value * 2^64) of a double in [2^-12, 2^64]
SKIM_DEV U192 to_fixed(double v) {
    uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
    int e = static_cast<int>((bits >> 52) & 0x7ff) - 1023;
    uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = e + 12;  // value * 2^64 = mant * 2^(e - 52 + 64)
    U192 r{{0, 0, 0}};
    int q = sh >> 6, rb = sh & 63;
    r.w[q] = mant << rb;
    if (rb && q + 1 < 3) r.w[q + 1] = mant >> (64 - rb);
    return r;
}

SKIM_DEV int top_bit(const U192 &a) {
    for (int i = 2; i >= 0; i--)
        if (a.w[i]) return i * 64 + 63 - __clzll(static_cast<long long>(a.w[i]));
    return -1;
}

SKIM_DEV uint64_t bit_at(const U192 &a, int p) { return (a.w[p >> 6] >> (p & 63)) & 1ull; }

SKIM_DEV bool any_below(const U192 &a, int p) {  // any bit set strictly below position p
    for (int i = 0; i < 3; i++) {
        int lo = i * 64;
        if (p <= lo) break;
        uint64_t m = (p - lo >= 64) ? ~0ull : ((1ull << (p - lo)) - 1);
        if (a.w[i] & m) return true;
    }
    return false;
}

// round (a * 2^-64) to the nearest double, ties to even
SKIM_DEV double fixed_to_double(const U192 &a) {
    int p = top_bit(a);
    if (p < 0) return 0.0;
    if (p <= 52) return ldexp(static_cast<double>(a.w[0]), -64);
    int sh = p - 52;
    uint64_t mant = 0;
    for (int b = 0; b < 53; b++) mant |= bit_at(a, sh + b) << b;
    bool rnd = bit_at(a, sh - 1);
    bool sticky = any_below(a, sh - 1);
    if (rnd && (sticky || (mant & 1ull))) {
        mant++;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            sh++;
        }
    }
    return ldexp(static_cast<double>(mant), sh - 64);
}

// ---- multi-block form: the work of a group of queries is spread over the
// whole GPU.  Each query owns a hash table of H_q slots (a power of two) in
// one scratch array; table q is cut into chunks of kQChunk slots whose
// partial sums (exact, 192-bit) are added per query at the end.

constexpr uint32_t kQChunk = 2048;

SKIM_DEV uint32_t upper_bound_u64(const uint64_t *a, uint32_t n, uint64_t x) {  // first i with a[i] > x
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_q_clear(uint64_t *hkeys, uint64_t *hvals, uint64_t total, unsigned long long *top_tau,
                          unsigned *top_used, uint32_t q) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        hkeys[i] = kEmptyKey;
        hvals[i] = 0;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        top_tau[i] = 0;
        top_used[i] = 0;
    }
}

__global__ void k_q_insert(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, const uint32_t *seeds,
                           const uint64_t *offsets, const uint64_t *table_off, uint32_t q, uint64_t *hkeys,
                           uint64_t *hvals, unsigned long long *top_tau, unsigned *top_used, unsigned *err) {
    const uint64_t total = offsets[q] * k;
    for (uint64_t e = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t j = e / k;
        const uint32_t pos = static_cast<uint32_t>(e % k);
        const uint32_t u = seeds[j];
        if (u >= n) {
            atomicOr(err, 1u);
            continue;
        }
        const uint32_t ln = xlen[u];
        const uint32_t body = ln == k ? k - 1 : ln;
        if (pos >= body) continue;
        const uint32_t qi = upper_bound_u64(offsets + 1, q, j);  // query holding seed j
        const uint64_t z = X[static_cast<uint64_t>(u) * k + pos];
        const uint64_t tau = ln == k ? X[static_cast<uint64_t>(u) * k + k - 1] : ~0ull;
        if (z == kEmptyKey) {
            atomicMax(&top_tau[qi], static_cast<unsigned long long>(tau));
            top_used[qi] = 1;
            continue;
        }
        const uint64_t base = table_off[qi], H = table_off[qi + 1] - base;
        uint64_t *tk = hkeys + base;
        uint64_t *tv = hvals + base;
        uint64_t h = fmix(z) & (H - 1);
        for (uint64_t p = 0; p < H; p++) {
            unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long *>(&tk[h]),
                                                static_cast<unsigned long long>(kEmptyKey),
                                                static_cast<unsigned long long>(z));
            if (prev == kEmptyKey || prev == z) {
                atomicMax(reinterpret_cast<unsigned long long *>(&tv[h]), static_cast<unsigned long long>(tau));
                break;
            }
            h = (h + 1) & (H - 1);
        }
    }
}

// one block per chunk: partial[c] = exact sum of the chunk's terms
__global__ void __launch_bounds__(256) k_q_sum(const uint64_t *hkeys, const uint64_t *hvals, const uint64_t *table_off,
                                               const uint64_t *chunk_off, uint32_t q,
                                               const unsigned long long *top_tau, const unsigned *top_used,
                                               QueryTerms terms, U192 *partial) {
    __shared__ U192 wsum[8];
    const uint32_t c = blockIdx.x;
    const uint32_t qi = upper_bound_u64(chunk_off + 1, q, c);
    const uint64_t first = chunk_off[qi];
    const uint64_t lo = table_off[qi] + (c - first) * kQChunk;
    const uint64_t hi = min(lo + kQChunk, table_off[qi + 1]);
    U192 acc{{0, 0, 0}};
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        if (hkeys[i] != kEmptyKey) {
            const double v = term_of(terms, hvals[i]);
            if (v != 0.0) add192(acc, to_fixed(v));
        }
    if (c == first && threadIdx.x == 0 && top_used[qi]) {
        const double v = term_of(terms, top_tau[qi]);
        if (v != 0.0) add192(acc, to_fixed(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        U192 other;
        for (int w = 0; w < 3; w++) other.w[w] = __shfl_down_sync(kFull, acc.w[w], o);
        add192(acc, other);
    }
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        U192 tot{{0, 0, 0}};
        for (int w = 0; w < 8; w++) add192(tot, wsum[w]);
        partial[c] = tot;
    }
}

__global__ void k_q_final(const U192 *partial, const uint64_t *chunk_off, uint32_t q, double div, double *out) {
    for (uint32_t qi = blockIdx.x * blockDim.x + threadIdx.x; qi < q; qi += gridDim.x * blockDim.x) {
        U192 tot{{0, 0, 0}};
        for (uint64_t c = chunk_off[qi]; c < chunk_off[qi + 1]; c++) add192(tot, partial[c]);
        out[qi] = fixed_to_double(tot) / div;
    }
}

// Single-node influence estimates from each node's own sketch: the bottom-k
// estimator (k-1)/tau of Section 3 (mode 0), the permutation estimator
// 1 + (k-1)(D-1)/(T-1) of Section 3.1 (mode 1) and n(k-1)/(T-1) of Section 3.2
// (mode 2); |X_v| (mode 0, 1) or 0 (mode 2) for a sketch that is not full.
__global__ void k_node_estimates(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, uint32_t l,
                                 int mode, double *out) {
    const double dl = static_cast<double>(l), k1 = static_cast<double>(k - 1);
    const double d1 = static_cast<double>(static_cast<uint64_t>(n) * l - 1);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t lv = xlen[v];
        double e;
        if (lv < k) {
            e = mode == 2 ? 0.0 : static_cast<double>(lv) / dl;
        } else {
            const double q = __ull2double_rn(X[static_cast<uint64_t>(v) * k + k - 1]);
            if (mode == 0) e = k1 / ldexp(q, -64) / dl;
            else if (mode == 1) e = (1.0 + k1 * d1 / q) / dl;
            else e = static_cast<double>(n) * k1 / q;
        }
        out[v] = e;
    }
}

}  // namespace

uint32_t query_chunks(uint64_t table_slots) { return static_cast<uint32_t>((table_slots + kQChunk - 1) / kQChunk); }

size_t query_partial_bytes() { return sizeof(U192); }

cudaError_t launch_node_estimates(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, uint32_t l,
                                  int mode, double *out, cudaStream_t s) {
    note_launch();
    const unsigned g = static_cast<unsigned>(std::min<uint64_t>((n + 255) / 256, 152 * 16));
    k_node_estimates<<<g ? g : 1, 256, 0, s>>>(X, xlen, n, k, l, mode, out);
    return cudaGetLastError();
}

cudaError_t launch_query_multi(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, const QueryTerms &terms,
                               const uint32_t *seeds, const uint64_t *offsets, const uint64_t *table_off,
                               const uint64_t *chunk_off, uint32_t q, uint64_t total_slots, uint64_t total_seeds,
                               uint32_t total_chunks, const QueryScratch &qs, double *out, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    auto grid = [](uint64_t work) {
        uint64_t g = (work + 255) / 256;
        return static_cast<unsigned>(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
    };
    unsigned long long *top_tau = reinterpret_cast<unsigned long long *>(qs.top_tau);
    note_launch();
    k_q_clear<<<grid(total_slots), 256, 0, s>>>(qs.hkeys, qs.hvals, total_slots, top_tau, qs.top_used, q);
    note_launch();
    k_q_insert<<<grid(total_seeds * k), 256, 0, s>>>(X, xlen, n, k, seeds, offsets, table_off, q, qs.hkeys, qs.hvals,
                                                     top_tau, qs.top_used, qs.err);
    note_launch();
    k_q_sum<<<total_chunks, 256, 0, s>>>(qs.hkeys, qs.hvals, table_off, chunk_off, q, top_tau, qs.top_used, terms,
                                         static_cast<U192 *>(qs.partial));
    note_launch();
    k_q_final<<<grid(q), 256, 0, s>>>(static_cast<const U192 *>(qs.partial), chunk_off, q, terms.div, out);
    return cudaGetLastError();
}

}  // namespace skim

// ---------------------------------------------------------------------------
// Allocation-free variant for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool, inside a region where allocation would break a
// memory budget, or in processes whose allocator is owned by someone else.
// This entry point keeps the query's scratch hash table in a fixed array of
// static device memory instead (every GPU that loads the library holds it
// until the process exits).  The caller still passes the sketches, the seed
// list and the output.  All calls on a device share the one array, so calls
// whose work overlaps on the GPU race with each other; the kernel clears the
// part of the table it uses before every query.
// ---------------------------------------------------------------------------
#include <mutex>

#include "skim.h"

namespace skim {
namespace {

constexpr uint64_t kStaticSlots = 1ull << 18;  // hash slots: 2^18 keys + 2^18 values = 4 MiB
static __device__ __align__(256) uint64_t g_static_table[2 * kStaticSlots];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
uint64_t *g_static_ptr[kMaxDevices] = {};  // device address of g_static_table, per device

__global__ void __launch_bounds__(kQThreads) k_query_static(const uint64_t *X, const uint32_t *xlen, uint32_t n,
                                                            uint32_t k, QueryTerms terms, const uint32_t *seeds,
                                                            uint32_t s, uint64_t *table, uint64_t H, double *out) {
    __shared__ unsigned long long top_tau;
    __shared__ int top_used, bad;
    __shared__ U192 wsum[kQThreads / 32];
    uint64_t *tk = table;
    uint64_t *tv = table + H;
    if (threadIdx.x == 0) {
        top_tau = 0;
        top_used = 0;
        bad = 0;
    }
    for (uint64_t i = threadIdx.x; i < H; i += blockDim.x) {
        tk[i] = kEmptyKey;
        tv[i] = 0;
    }
    __syncthreads();
    const uint64_t hmask = H - 1;
    const uint64_t work = static_cast<uint64_t>(s) * k;
    for (uint64_t e = threadIdx.x; e < work; e += blockDim.x) {
        const uint32_t u = seeds[e / k];
        const uint32_t pos = static_cast<uint32_t>(e % k);
        if (u >= n) {
            bad = 1;
            continue;
        }
        const uint32_t ln = xlen[u];
        const uint32_t body = ln == k ? k - 1 : ln;
        if (pos >= body) continue;
        const uint64_t z = X[static_cast<uint64_t>(u) * k + pos];
        const uint64_t tau = ln == k ? X[static_cast<uint64_t>(u) * k + k - 1] : ~0ull;
        if (z == kEmptyKey) {
            atomicMax(&top_tau, static_cast<unsigned long long>(tau));
            top_used = 1;
            continue;
        }
        uint64_t h = fmix(z) & hmask;
        for (uint64_t p = 0; p < H; p++) {
            unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long *>(&tk[h]),
                                                static_cast<unsigned long long>(kEmptyKey),
                                                static_cast<unsigned long long>(z));
            if (prev == kEmptyKey || prev == z) {
                atomicMax(reinterpret_cast<unsigned long long *>(&tv[h]), static_cast<unsigned long long>(tau));
                break;
            }
            h = (h + 1) & hmask;
        }
    }
    __syncthreads();
    U192 acc{{0, 0, 0}};
    for (uint64_t i = threadIdx.x; i < H; i += blockDim.x)
        if (tk[i] != kEmptyKey) {
            const double v = term_of(terms, tv[i]);
            if (v != 0.0) add192(acc, to_fixed(v));
        }
    if (threadIdx.x == 0 && top_used) {
        const double v = term_of(terms, top_tau);
        if (v != 0.0) add192(acc, to_fixed(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        U192 other;
        for (int w = 0; w < 3; w++) other.w[w] = __shfl_down_sync(kFull, acc.w[w], o);
        add192(acc, other);
    }
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        U192 tot{{0, 0, 0}};
        for (int w = 0; w < kQThreads / 32; w++) add192(tot, wsum[w]);
        out[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : fixed_to_double(tot) / terms.div;
    }
}

}  // namespace
}  // namespace skim

extern "C" int skim_union_estimate_static(const uint64_t *x_dev, const uint32_t *len_dev, uint32_t n, uint32_t k,
                                          uint32_t l, uint32_t rank_mode, const uint32_t *seeds_dev,
                                          uint32_t n_seeds, double *est_dev, void *stream) {
    using namespace skim;
    if (!x_dev || !len_dev || !est_dev || (n_seeds && !seeds_dev)) return SKIM_EINVAL;
    if (n == 0 || k < 2 || k > 255 || l == 0 || l > 64) return SKIM_EINVAL;
    if (rank_mode > SKIM_RANKS_IC_MODEL || (rank_mode == SKIM_RANKS_IC_MODEL && l != 1)) return SKIM_EINVAL;
    // the same reading of a threshold as the context queries (query_terms_of)
    QueryTerms terms{0, 0.0, static_cast<double>(l)};
    if (rank_mode == SKIM_RANKS_PERMUTATION)
        terms = QueryTerms{1, static_cast<double>(static_cast<uint64_t>(n) * l - 1), static_cast<double>(l)};
    else if (rank_mode == SKIM_RANKS_IC_MODEL)
        terms = QueryTerms{2, static_cast<double>(n), 1.0};
    uint64_t H = 64;
    const uint64_t need = 2ull * n_seeds * (k - 1) + 2;
    while (H < need) H <<= 1;
    if (H > kStaticSlots) return SKIM_ERANGE;  // the static table holds 2^18 slots
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SKIM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SKIM_ERANGE;
    uint64_t *table = nullptr;
    {
        // once per device, with that device current: the device address of
        // the static array (its name in host code is only a stand-in)
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_table) != cudaSuccess || !p) return SKIM_ECUDA;
            g_static_ptr[dev] = static_cast<uint64_t *>(p);
        }
        table = g_static_ptr[dev];
    }
    // An error left pending by the caller's earlier work is not ours to
    // consume: report it and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return SKIM_ECUDA;
    note_launch();
    k_query_static<<<1, kQThreads, 0, static_cast<cudaStream_t>(stream)>>>(x_dev, len_dev, n, k, terms, seeds_dev,
                                                                           n_seeds, table, H, est_dev);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();  // the launch's own error
        return SKIM_ECUDA;
    }
    return SKIM_OK;
}

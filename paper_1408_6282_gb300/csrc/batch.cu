// batch.cu -- per-batch steps after a reverse search has marked, for every
// visited (node, lane word), the lanes that reached the node.  Visit records
// (node << tbits | word, table slot) arrive sorted by key, so each node's
// words form one run in increasing rank order.
//
// Algorithm 2 acceptance (Section 5.2): for node v and instance i the first
// k - lcnt[v][i] lanes of instance i (in rank order) join v's local sketch;
// the ranks that join also enter the global sketch X_v while it holds fewer
// than k ranks.  Batches advance in increasing rank order, so X_v is filled
// in increasing order and needs no merge: appending is the bottom-k merge of
// Algorithm 2.  Pruning in the search used the counts at the start of the
// batch, so every lane whose rank belongs in a local sketch did reach it.
//
// SKIM (Algorithm 1): size[v] counts the processed, uncovered ranks that reach
// v.  The batch's stop lane is the earliest lane at which some node's size
// reaches k (smallest node id on ties); lanes up to it are committed (sizes
// and the inverted index), the rest stay valid for the next step because a
// search from an uncovered pair never meets a covered node.
#include "internal.cuh"

namespace skim {

namespace {

inline unsigned grid_for(size_t n, int threads, unsigned cap = 152 * 32) {
    size_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g ? g : 1);
}

// Instance of every lane and the offset of its coin stream, (i + 1) * G.
// Instance and coin-stream offset of every lane: instance i = pair % l, or in
// the IC model (lane_rank given) a fresh instance numbered by the position.
__global__ void k_lane_inst(const uint32_t *lane_pair, const uint64_t *lane_rank, uint32_t B, uint32_t l,
                            uint8_t *lane_inst, uint64_t *lane_g) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < B; j += gridDim.x * blockDim.x) {
        if (lane_rank) {
            lane_inst[j] = 0;
            lane_g[j] = kGolden * (lane_rank[j] + 1);
            continue;
        }
        const uint32_t i = lane_pair[j] % l;
        lane_inst[j] = static_cast<uint8_t>(i);
        lane_g[j] = kGolden * static_cast<uint64_t>(i + 1);
    }
}

SKIM_DEV bool run_start(const uint64_t *rec_key, uint64_t r, uint32_t tbits) {
    return r == 0 || (rec_key[r] >> tbits) != (rec_key[r - 1] >> tbits);
}

// Algorithm 2's acceptance for the records of one batch, sorted by key so that
// a node's records are adjacent and in word (= rank) order.  Per (node v,
// instance i) the first k - lcnt[v,i] offers are accepted (the instance-local
// sketch), and accepted ranks are appended to X_v while it holds fewer than k.
//
// Records are split into windows of 32; a warp owns the nodes whose runs start
// in its window and walks their records 32 at a time, past the window's end
// for the last one.  The offers (record, lane bit) are taken 32 per step in
// rank order.  An offer of (v, i) with rank rho among the step's offers of
// (v, i) is accepted iff lcnt[v,i] + rho < k, which is the sequential rule;
// its place in X_v is xlen[v] plus the accepted offers of v before it in the
// step.  Counts, lengths and full bits are written back after every step, so
// the next step reads them current.

// One step: offer `has` of node v at batch lane ln (one per warp lane).
SKIM_DEV void accept_step(bool has, uint32_t v, uint64_t ln, const uint8_t *__restrict__ lane_inst,
                          const uint64_t *__restrict__ lane_rank, uint32_t l, uint32_t k, uint8_t *lcnt,
                          uint64_t *full, uint32_t *row_flag, uint64_t *X, uint32_t *xlen, unsigned long long &ins) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t i = 0, lc0 = 0, len0 = 0;
    if (has) {
        i = lane_inst[ln];
        lc0 = lcnt[static_cast<uint64_t>(v) * l + i];
        len0 = xlen[v];
    }
    // peers in (v, i) and in v; idle lanes get keys no offer has
    const unsigned pvi = __match_any_sync(kFull, has ? (static_cast<uint64_t>(v) << 6 | i) : ~0ull - lane);
    const unsigned pv = __match_any_sync(kFull, has ? static_cast<uint64_t>(v) : (1ull << 32 | lane));
    const uint32_t rho = __popc(pvi & lanemask_lt());
    const bool acc = has && lc0 + rho < k;
    const unsigned ab = __ballot_sync(kFull, acc);
    if (acc) {
        const uint32_t pos = len0 + __popc(ab & pv & lanemask_lt());
        if (pos < k) X[static_cast<uint64_t>(v) * k + pos] = lane_rank[ln];
        ins++;
    }
    __syncwarp();
    if (has && rho == 0 && lc0 < k) {  // one lane per (v, i)
        const uint32_t c = min(k, lc0 + __popc(pvi));
        lcnt[static_cast<uint64_t>(v) * l + i] = static_cast<uint8_t>(c);
        if (c == k) {
            atomicOr(reinterpret_cast<unsigned long long *>(&full[v]), 1ull << i);
            if (row_flag) atomicOr(&row_flag[static_cast<uint64_t>(v) * l + i], kRowFull);
        }
    }
    if (has && (pv & lanemask_lt()) == 0) {  // one lane per v
        const uint32_t len = min(k, len0 + __popc(ab & pv));
        if (len != len0) xlen[v] = len;
    }
    __syncwarp();
}

// Record r's lane bits are those of its table slot, hvals[2 * rec_val[r]].
__global__ void __launch_bounds__(256)
    k_accept(const uint64_t *__restrict__ rec_key, const uint32_t *__restrict__ rec_val,
             const uint64_t *__restrict__ hvals, uint64_t R, uint32_t tbits,
             const uint8_t *__restrict__ lane_inst, const uint64_t *__restrict__ lane_rank, uint32_t l, uint32_t k,
             uint8_t *lcnt, uint64_t *full, uint32_t *row_flag, uint64_t *X, uint32_t *xlen, DevCtl *ctl) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t tmask = (1ull << tbits) - 1;
    unsigned long long ins = 0;
    const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const uint64_t nwin = (R + 31) / 32;
    for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < nwin; w += warps) {
        const uint64_t W0 = w * 32, W1 = min(R, W0 + 32);
        bool st = false;
        if (W0 + lane < W1) st = run_start(rec_key, W0 + lane, tbits);
        const unsigned sb = __ballot_sync(kFull, st);
        if (!sb) continue;  // the window lies inside a run owned by an earlier warp
        const uint64_t s0 = W0 + __ffs(sb) - 1;
        const uint64_t last = rec_key[W1 - 1] >> tbits;
        for (uint64_t c0 = s0;; c0 += 32) {
            // the warp's records form one stretch [s0, end of last's run)
            const uint64_t rr = c0 + lane;
            uint64_t key = 0, m = 0;
            bool act = false;
            if (rr < R) {
                key = rec_key[rr];
                act = rr < W1 || (key >> tbits) == last;
            }
            const unsigned actb = __ballot_sync(kFull, act);
            if (!actb) break;
            if (act) m = hvals[2ull * rec_val[rr]];
            const uint32_t vr = static_cast<uint32_t>(key >> tbits);
            const uint64_t tr = key & tmask;
            if (!__any_sync(kFull, __popcll(m) > 1)) {
                // one offer per record (the common case)
                const bool has = m != 0;
                accept_step(has, vr, tr * 64 + (has ? __ffsll(m) - 1 : 0), lane_inst, lane_rank, l, k, lcnt, full,
                            row_flag, X, xlen, ins);
            } else {
                // offer o is bit (o - pre_s) of record s with pre_s <= o < pre_s + cnt_s
                const uint32_t cnt = __popcll(m);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= static_cast<unsigned>(o)) incl += y;
                }
                const uint32_t pre = incl - cnt, total = __shfl_sync(kFull, incl, 31);
                for (uint32_t g = 0; g < total; g += 32) {
                    const uint32_t o = g + lane;
                    const bool has = o < total;
                    uint32_t src = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const uint32_t cand = src + step;
                        const uint32_t pc = __shfl_sync(kFull, pre, cand);
                        if (has && pc <= o) src = cand;
                    }
                    const uint64_t ms = __shfl_sync(kFull, m, src), ts = __shfl_sync(kFull, tr, src);
                    const uint32_t ps = __shfl_sync(kFull, pre, src), vs = __shfl_sync(kFull, vr, src);
                    uint64_t ln = 0;
                    if (has) {
                        uint64_t x = ms;
                        for (uint32_t skip = o - ps; skip; skip--) x &= x - 1;
                        ln = ts * 64 + (__ffsll(x) - 1);
                    }
                    accept_step(has, vs, ln, lane_inst, lane_rank, l, k, lcnt, full, row_flag, X, xlen, ins);
                }
            }
            if (actb != kFull) break;
        }
    }
    warp_add(&ctl->stats[kStInsert], ins);
}

// lanes of word t inside [lo, hi] (inclusive), lo <= hi
SKIM_DEV uint64_t range_mask(uint64_t t, uint32_t lo, uint32_t hi) {
    const uint64_t w0 = t * 64, w1 = w0 + 63;
    if (w1 < lo || w0 > hi) return 0;
    uint64_t m = ~0ull;
    if (lo > w0) m &= ~0ull << (lo - w0);
    if (hi < w1) m &= ~0ull >> (w1 - hi);
    return m;
}

// SKIM batches read a record's lane bits in every candidate scan and in both
// commit passes: they are gathered once from the visited table, next to the
// records, after the records are put in order.
__global__ void k_gather_bits(const uint32_t *__restrict__ rec_val, const uint64_t *__restrict__ hvals, uint64_t R,
                              uint64_t *__restrict__ rbits) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        rbits[r] = hvals[2ull * rec_val[r]];
}

// SKIM's stop: per node v the lane at which size[v] reaches k, i.e. the
// need = k - size[v]-th uncovered lane bit (from lane lo on) of v's records in
// rank order (a node already at k stops at its first record).  Warps own the
// runs that start in 32-record windows, as in the acceptance; a segmented
// scan over the lanes counts each node's bits in order.
__global__ void k_candidates(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                             const uint64_t *alive, uint32_t lo, const uint32_t *size, uint32_t k, DevCtl *ctl) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t tmask = (1ull << tbits) - 1;
    const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const uint64_t nwin = (R + 31) / 32;
    for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < nwin; w += warps) {
        const uint64_t W0 = w * 32, W1 = min(R, W0 + 32);
        bool st = false;
        if (W0 + lane < W1) st = run_start(rec_key, W0 + lane, tbits);
        const unsigned sb = __ballot_sync(kFull, st);
        if (!sb) continue;
        const uint64_t s0 = W0 + __ffs(sb) - 1;
        const uint64_t last = rec_key[W1 - 1] >> tbits;
        uint64_t cv = ~0ull;  // node that continues from the previous chunk, and its count so far
        uint32_t ccum = 0;
        for (uint64_t c0 = s0;; c0 += 32) {
            const uint64_t rr = c0 + lane;
            uint64_t key = 0, m = 0;
            bool act = false;
            if (rr < R) {
                key = rec_key[rr];
                act = rr < W1 || (key >> tbits) == last;
            }
            const unsigned actb = __ballot_sync(kFull, act);
            if (!actb) break;
            const uint64_t v = key >> tbits, t = key & tmask;
            // lanes of the record's word from lo on; its lane bits only when
            // some are left
            if (act) {
                m = range_mask(t, lo, 0xffffffffu);
                if (m) m &= rbits[rr] & alive[t];
            }
            const uint32_t c = __popcll(m);
            // inclusive count of v's bits up to this record (runs are contiguous)
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, o);
                const uint64_t vo = __shfl_up_sync(kFull, v, o);
                if (lane >= static_cast<unsigned>(o) && vo == v) incl += y;
            }
            if (v == cv) incl += ccum;
            if (act) {
                const uint32_t excl = incl - c, need = k - size[v];
                const bool hit = need == 0 ? run_start(rec_key, rr, tbits) : (excl < need && incl >= need);
                if (hit) {
                    const uint64_t p = t * 64 + nth_set_bit(m, static_cast<int>(need - excl - 1));
                    atomicMin(&ctl->best, (p << 32) | v);
                }
            }
            const int ll = 31 - __clz(actb);
            cv = __shfl_sync(kFull, v, ll);
            ccum = __shfl_sync(kFull, incl, ll);
            if (actb != kFull) break;
        }
    }
}

// Commit of lanes [lo, hi]: size[v] += the committed uncovered lane bits of
// v's records, and per lane the number of nodes it reaches (the index
// segment lengths).  Additive, so one thread per record.
__global__ void k_commit_count(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                               const uint64_t *alive, uint32_t lo, uint32_t hi, uint32_t *size,
                               unsigned long long *lane_cnt, DevCtl *ctl) {
    const uint64_t tmask = (1ull << tbits) - 1;
    unsigned long long ins = 0;
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t key = rec_key[r];
        const uint64_t t = key & tmask;
        uint64_t m = range_mask(t, lo, hi);
        if (!m) continue;
        m &= rbits[r] & alive[t];
        if (!m) continue;
        const uint32_t c = __popcll(m);
        atomicAdd(&size[key >> tbits], c);
        ins += c;
        while (m) {
            const int j = __ffsll(m) - 1;
            m &= m - 1;
            atomicAdd(&lane_cnt[t * 64 + j], 1ull);
        }
    }
    warp_add(&ctl->stats[kStInsert], ins);
}

__global__ void k_commit_scatter(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                                 const uint64_t *alive, uint32_t lo, uint32_t hi, const uint64_t *lane_off,
                                 uint32_t *lane_fill, const uint64_t *idx_ctr, uint32_t *idx_nodes) {
    const uint64_t tmask = (1ull << tbits) - 1;
    const uint64_t idx_base = idx_ctr[0];
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < R;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t v = rec_key[r] >> tbits;
        const uint64_t t = rec_key[r] & tmask;
        uint64_t m = range_mask(t, lo, hi);
        if (m) m &= rbits[r] & alive[t];
        while (m) {
            int j = __ffsll(m) - 1;
            m &= m - 1;
            const uint64_t lane = t * 64 + j;
            uint32_t pos = atomicAdd(&lane_fill[lane], 1u);
            idx_nodes[idx_base + lane_off[lane] + pos] = static_cast<uint32_t>(v);
        }
    }
}

__global__ void k_commit_segments(const uint32_t *lane_pair, uint32_t lo, uint32_t hi, const uint64_t *lane_cnt,
                                  const uint64_t *lane_off, const uint64_t *idx_ctr, uint64_t *seg_start,
                                  uint32_t *seg_len) {
    const uint64_t idx_base = idx_ctr[0];
    for (uint64_t j = lo + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j <= hi;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t c = lane_cnt[j];
        if (c) {
            uint32_t pr = lane_pair[j];
            seg_start[pr] = idx_base + lane_off[j];
            seg_len[pr] = static_cast<uint32_t>(c);
        }
    }
}

// After a commit of `total` index entries: idx_ctr[1] = the commit's first
// entry, idx_ctr[0] = the next free one.
__global__ void k_idx_advance(uint64_t *idx_ctr, const unsigned long long *total) {
    idx_ctr[1] = idx_ctr[0];
    idx_ctr[0] += *total;
}

__global__ void k_refilter(const uint32_t *lane_pair, uint32_t lo, uint32_t B, uint32_t l, const uint64_t *covered,
                           uint64_t *alive) {
    for (uint32_t j = lo + blockIdx.x * blockDim.x + threadIdx.x; j < B; j += gridDim.x * blockDim.x) {
        const uint64_t bit = 1ull << (j & 63);
        if (!(alive[j >> 6] & bit)) continue;
        uint32_t pr = lane_pair[j];
        uint32_t u = pr / l, i = pr % l;
        if ((covered[u] >> i) & 1ull) atomicAnd(reinterpret_cast<unsigned long long *>(&alive[j >> 6]), ~bit);
    }
}

// Section 4.3.2: add delta to the size of every node in the committed index
// list of lane p (each node appears once in a lane's list).
__global__ void k_lane_size_add(const uint32_t *idx_nodes, const uint64_t *idx_base, const uint64_t *lane_off,
                                const uint64_t *lane_cnt, uint32_t p, uint32_t *size, int delta) {
    const uint64_t off = *idx_base + lane_off[p], cnt = lane_cnt[p];
    for (uint64_t j = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; j < cnt;
         j += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        size[idx_nodes[off + j]] += static_cast<uint32_t>(delta);
}

// k' of Section 4.3.2: the largest size among nodes other than x.
__global__ void k_max_size_except(const uint32_t *size, uint32_t n, uint32_t x, uint32_t *out) {
    uint32_t best = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (v != x) best = max(best, size[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

__global__ void k_argmax_size(const uint32_t *size, uint32_t n, DevCtl *ctl) {
    unsigned long long best = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        unsigned long long key = (static_cast<unsigned long long>(size[v]) << 32) | (0xffffffffu - v);
        best = max(best, key);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ctl->argmax, best);
}

__global__ void k_min_unchosen(const uint8_t *chosen, uint32_t n, DevCtl *ctl) {
    unsigned long long best = ~0ull;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (!chosen[v]) best = min(best, static_cast<unsigned long long>(v));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(kFull, best, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&ctl->best, best);
}

}  // namespace

cudaError_t launch_lane_inst(const uint32_t *lane_pair, const uint64_t *lane_rank, uint32_t B, uint32_t l,
                             uint8_t *lane_inst, uint64_t *lane_g, cudaStream_t s) {
    note_launch();
    k_lane_inst<<<grid_for(B, 256), 256, 0, s>>>(lane_pair, lane_rank, B, l, lane_inst, lane_g);
    return cudaGetLastError();
}
cudaError_t launch_accept(const uint64_t *rec_key, const uint32_t *rec_val, const uint64_t *hvals, uint64_t R,
                          uint32_t tbits, const uint8_t *lane_inst, const uint64_t *lane_rank, uint32_t l, uint32_t k,
                          uint8_t *lcnt, uint64_t *full, uint32_t *row_flag, uint64_t *X, uint32_t *xlen, DevCtl *ctl,
                          cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    note_launch();
    k_accept<<<grid_for(R, 256), 256, 0, s>>>(rec_key, rec_val, hvals, R, tbits, lane_inst, lane_rank, l, k,
                                               lcnt, full, row_flag, X, xlen, ctl);
    return cudaGetLastError();
}
cudaError_t launch_gather_bits(const uint32_t *rec_val, const uint64_t *hvals, uint64_t R, uint64_t *rbits,
                               cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    note_launch();
    k_gather_bits<<<grid_for(R, 256), 256, 0, s>>>(rec_val, hvals, R, rbits);
    return cudaGetLastError();
}
cudaError_t launch_candidates(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                              const uint64_t *alive, uint32_t lo, const uint32_t *size, uint32_t k, DevCtl *ctl,
                              cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    note_launch();
    k_candidates<<<grid_for(R, 256), 256, 0, s>>>(rec_key, rbits, R, tbits, alive, lo, size, k, ctl);
    return cudaGetLastError();
}
cudaError_t launch_commit_count(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                                const uint64_t *alive, uint32_t lo, uint32_t hi, uint32_t *size, uint64_t *lane_cnt,
                                DevCtl *ctl, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    note_launch();
    k_commit_count<<<grid_for(R, 256), 256, 0, s>>>(rec_key, rbits, R, tbits, alive, lo, hi, size,
                                                    reinterpret_cast<unsigned long long *>(lane_cnt), ctl);
    return cudaGetLastError();
}
cudaError_t launch_commit_scatter(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                                  const uint64_t *alive, uint32_t lo, uint32_t hi, const uint64_t *lane_off,
                                  uint32_t *lane_fill, const uint64_t *idx_ctr, uint32_t *idx_nodes, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    note_launch();
    k_commit_scatter<<<grid_for(R, 256), 256, 0, s>>>(rec_key, rbits, R, tbits, alive, lo, hi, lane_off, lane_fill,
                                                      idx_ctr, idx_nodes);
    return cudaGetLastError();
}
cudaError_t launch_commit_segments(const uint32_t *lane_pair, uint32_t lo, uint32_t hi, const uint64_t *lane_cnt,
                                   const uint64_t *lane_off, const uint64_t *idx_ctr, uint64_t *seg_start,
                                   uint32_t *seg_len, cudaStream_t s) {
    note_launch();
    k_commit_segments<<<grid_for(hi - lo + 1, 256), 256, 0, s>>>(lane_pair, lo, hi, lane_cnt, lane_off, idx_ctr,
                                                                 seg_start, seg_len);
    return cudaGetLastError();
}
cudaError_t launch_refilter(const uint32_t *lane_pair, uint32_t lo, uint32_t B, uint32_t l, const uint64_t *covered,
                            uint64_t *alive, cudaStream_t s) {
    if (lo >= B) return cudaSuccess;
    note_launch();
    k_refilter<<<grid_for(B - lo, 256), 256, 0, s>>>(lane_pair, lo, B, l, covered, alive);
    return cudaGetLastError();
}
cudaError_t launch_argmax_size(const uint32_t *size, uint32_t n, DevCtl *ctl, cudaStream_t s) {
    note_launch();
    k_argmax_size<<<grid_for(n, 256), 256, 0, s>>>(size, n, ctl);
    return cudaGetLastError();
}
cudaError_t launch_second_size(const uint32_t *idx_nodes, const uint64_t *idx_base, const uint64_t *lane_off,
                               const uint64_t *lane_cnt, uint32_t p, uint32_t *size, uint32_t n, uint32_t x,
                               uint32_t *out, cudaStream_t s) {
    // the stop lane's list holds at most n nodes (its length is on the device)
    const unsigned g = grid_for(n, 256, 1024);
    note_launch();
    k_lane_size_add<<<g, 256, 0, s>>>(idx_nodes, idx_base, lane_off, lane_cnt, p, size, -1);
    note_launch();
    k_max_size_except<<<grid_for(n, 256), 256, 0, s>>>(size, n, x, out);
    note_launch();
    k_lane_size_add<<<g, 256, 0, s>>>(idx_nodes, idx_base, lane_off, lane_cnt, p, size, 1);
    return cudaGetLastError();
}
cudaError_t launch_idx_advance(uint64_t *idx_ctr, const unsigned long long *total, cudaStream_t s) {
    note_launch();
    k_idx_advance<<<1, 1, 0, s>>>(idx_ctr, total);
    return cudaGetLastError();
}
cudaError_t launch_min_unchosen(const uint8_t *chosen, uint32_t n, DevCtl *ctl, cudaStream_t s) {
    note_launch();
    k_min_unchosen<<<grid_for(n, 256), 256, 0, s>>>(chosen, n, ctl);
    return cudaGetLastError();
}

}  // namespace skim

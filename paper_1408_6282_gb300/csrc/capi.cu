// capi.cu -- libskim C ABI: context, graph and rank setup, the rank-batched
// sketch build (Algorithm 2), SKIM (Algorithm 1) and influence queries
// (Eq. unionest).  Host code orchestrates; all per-element work runs in the
// kernels of graph.cu, traverse.cu, batch.cu and query.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"
#include "prims.cuh"
#include "skim.h"

using namespace skim;

struct skim_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool broken = false;
    uint32_t n = 0;
    uint64_t m = 0;
    uint32_t l = 0, k = 0;
    uint64_t nl = 0;
    CoinModel cm{};
    uint32_t batch_cfg = 0;
    // switches of the rank-batched search (skim_set_tuning): per-warp queues
    // for batches of at most ring_rpl expected records per lane; records
    // placed by node buckets when buckets <= node_density * records
    double ring_rpl = 0;
    uint32_t node_density = 0;
    // graph
    uint32_t *fptr = nullptr, *fcol = nullptr, *rptr = nullptr, *rcol = nullptr;
    uint64_t *thr_wc = nullptr;
    uint64_t *rhe = nullptr, *fhe = nullptr;  // per-edge coin-stream states
    // rank order
    uint64_t *srank = nullptr;
    uint32_t *spair = nullptr;
    void *rank_ws = nullptr;
    // rank order: SKIM_RANKS_* mode, positions in the order, and how many of
    // them the sketch build processes
    int rank_mode = 0;
    uint64_t npos = 0, nbuild = 0;
    // materialised instances (Section 2): per-edge live masks in both CSR
    // orders and the node-major live in-neighbour rows of every (v, i)
    bool mat = false;
    bool mat_wanted = true;  // skim_set_live_rows: walk materialised live rows when they exist
    bool live_ready = false;  // the live rows of both directions are filled
    uint64_t *rmask = nullptr, *fmask = nullptr;
    uint32_t *loff = nullptr, *foff = nullptr;  // live-row offsets (kRowFull flags on loff)
    uint32_t *rlive = nullptr, *flive = nullptr;  // live in- and out-neighbour rows
    uint32_t *rrow = nullptr, *rev2fwd = nullptr;  // per reverse CSR edge: head, forward position
    void *pieces = nullptr;                         // workspace of the long-row passes
    uint64_t rlive_cap = 0, live_total = 0;
    uint64_t rank_key = 0;
    // graphs of a batch (skim_create_batch): per-node rank bases, per-edge
    // thresholds, node offsets of the graphs
    uint64_t *rbase = nullptr, *rtm1 = nullptr, *ftm1 = nullptr;
    uint32_t batch_count = 0;
    // control
    DevCtl *ctl = nullptr;
    DevCtl *hctl = nullptr;  // pinned mirror
    unsigned *dflag = nullptr;
    // traversal scratch
    Item *q = nullptr;
    uint64_t qcap = 0;
    uint64_t *hkeys = nullptr, *hvals = nullptr, *pend = nullptr;
    uint64_t hcap = 0;
    uint64_t *rkey = nullptr, *rkey2 = nullptr;
    uint32_t *rval = nullptr, *rval2 = nullptr;
    // a SKIM batch's lane bits per record, gathered after the record order
    // (the order's scratch rkey2, free until the next batch)
    uint64_t *rbits = nullptr;
    uint64_t rcap = 0;
    // per-node placement of a batch's records (recsort.cu): counters (all
    // zero between batches), node offsets, node lists
    uint64_t *ncnt = nullptr, *noff = nullptr;
    uint32_t *nlist = nullptr;
    unsigned *nlist_cnt = nullptr;
    bool bnode = false;  // the active batch's records were placed per node
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint8_t *lane_inst = nullptr;
    uint64_t *lane_g = nullptr;
    uint64_t *alive = nullptr, *lane_cnt = nullptr, *lane_off = nullptr;
    uint32_t *lane_fill = nullptr;
    uint32_t lane_cap = 0;
    int grid_rev = 0, grid_fwd = 0, grid_ring = 0;
    uint64_t timeout_ns = 2000000000ull;
    // sketches
    uint8_t *lcnt = nullptr;
    uint64_t *full = nullptr, *X = nullptr;
    uint32_t *xlen = nullptr;
    bool built = false;
    // SKIM
    bool sk_init = false;
    uint64_t *covered = nullptr, *seg_start = nullptr, *pend_trav = nullptr, *pend_erase = nullptr;
    uint32_t *size = nullptr, *seg_len = nullptr, *idx = nullptr;
    uint8_t *chosen = nullptr;
    uint64_t idx_cap = 0;
    // inverted index fill: on the device [0] entries used, [1] first entry of
    // the last commit; on the host an upper bound of [0] (the visit bits of
    // the SKIM batches so far), which sizes the index without a read-back
    uint64_t *idx_ctr = nullptr;
    uint64_t idx_bound = 0, vis_seen = 0;
    uint64_t cursor = 0;
    uint32_t nseeds = 0;
    bool batch_active = false;
    uint64_t bp0 = 0;
    uint32_t bB = 0, btbits = 0, blo = 0;
    uint64_t bR = 0;
    uint32_t skim_B = 0;
    uint32_t retry_run = 0;  // consecutive SKIM batch re-runs
    // SKIM batch sizing: ranks consumed since the last seed, and the gap (in
    // ranks) between the last two seeds
    uint64_t since_stop = 0, last_gap = 0;
    double vpl_est = 0;  // visit records per lane of the last SKIM batch
    uint32_t last_B = 0;
    // Section 4.3.2 records of the current skim_greedy_ex call (device):
    // per seed the threshold rank and k'; null when not asked for
    uint64_t *rec_tau = nullptr;
    uint32_t *rec_kp = nullptr;
    uint32_t rec_j = 0;
    // the residual search of the last seed, launched and not read back yet:
    // the next read of the control block finishes it and stores its count of
    // newly covered pairs at *pend_cov
    bool pend_res = false;
    uint64_t *pend_cov = nullptr;
    // queries
    uint64_t *qk = nullptr, *qv = nullptr;
    uint64_t qtcap = 0;
    uint32_t *qseeds = nullptr;
    uint64_t qseeds_cap = 0;
    uint64_t *qoff = nullptr;  // seed, table and chunk offsets (3 x (q+1))
    double *qout = nullptr;
    uint64_t qmeta_cap = 0;
    uint64_t *qtop = nullptr;
    unsigned *qtopu = nullptr;
    void *qpart = nullptr;
    uint64_t qpart_cap = 0;
    // counters of the last build/greedy call
    uint64_t hstats[SKIM_STAT_COUNT] = {0};
    // kernel timing (CUDA events on the context stream)
    bool timing = false;
    double kms[SKIM_K_COUNT] = {0};
    uint64_t klaunch[SKIM_K_COUNT] = {0};
    struct Pend { cudaEvent_t a, b; int kind; };
    std::vector<Pend> kpend;
    std::vector<cudaEvent_t> kpool;
};

namespace {

int fail_cuda(skim_ctx *c, cudaError_t e) {
    if (c) c->broken = true;
    if (getenv("SKIM_DEBUG")) fprintf(stderr, "libskim: CUDA error %s\n", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SKIM_ENOMEM : SKIM_ECUDA;
}

#define CK(c, x)                                       \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return fail_cuda(c, e_); \
    } while (0)

#define RC(x)                 \
    do {                      \
        int r_ = (x);         \
        if (r_ != SKIM_OK) return r_; \
    } while (0)

// Device memory of every context comes from one stream-ordered pool per
// device that keeps the blocks freed by skim_destroy (release threshold: never)
// for the next context, so a context per graph or per request does not pay
// for cudaMalloc and cudaFree of its gigabytes of scratch each time.
// Allocations and frees are ordered on the context's stream.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t device_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

int dalloc_bytes(skim_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, c->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SKIM_ENOMEM : fail_cuda(c, e);
    }
    return SKIM_OK;
}

template <class T>
int dalloc(skim_ctx *c, T **p, size_t count) {
    return dalloc_bytes(c, reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T));
}

template <class T>
void dfree(skim_ctx *c, T *&p) {
    if (p) cudaFreeAsync(p, c->st);
    p = nullptr;
}

int bitlen(uint64_t x) {  // bits needed to hold values 0..x
    int b = 0;
    while (b < 64 && (x >> b)) b++;
    return b;
}

uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

uint64_t tm1_of(double p) {
    if (p >= 1.0) return ~0ull;
    return static_cast<uint64_t>(std::ldexp(p, 64)) - 1ull;
}

cudaEvent_t ev_get(skim_ctx *c) {
    if (!c->kpool.empty()) {
        cudaEvent_t e = c->kpool.back();
        c->kpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket a launch group with events; resolved at the next synchronisation.
struct KTimer {
    skim_ctx *c;
    int kind;
    cudaEvent_t a = nullptr;
    KTimer(skim_ctx *cc, int k) : c(cc), kind(k) {
        if (c->timing) {
            a = ev_get(c);
            cudaEventRecord(a, c->st);
        }
    }
    ~KTimer() {
        if (c->timing && a) {
            cudaEvent_t b = ev_get(c);
            cudaEventRecord(b, c->st);
            c->kpend.push_back({a, b, kind});
            c->klaunch[kind]++;
        }
    }
};

void resolve_timers(skim_ctx *c) {
    for (auto &p : c->kpend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->kms[p.kind] += ms;
        c->kpool.push_back(p.a);
        c->kpool.push_back(p.b);
    }
    c->kpend.clear();
}

int sync_ctl(skim_ctx *c) {
    CK(c, cudaMemcpyAsync(c->hctl, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    resolve_timers(c);
    return SKIM_OK;
}

// zero the queue/control fields of DevCtl, keep the statistics
int reset_ctl(skim_ctx *c) {
    CK(c, cudaMemsetAsync(c->ctl, 0, offsetof(DevCtl, stats), c->st));
    CK(c, cudaMemsetAsync(&c->ctl->err, 0, sizeof(unsigned) * 4, c->st));
    return SKIM_OK;
}

// the first `slots` visited-table slots empty (key and lane bits zero)
cudaError_t clear_table(skim_ctx *c, uint64_t slots) {
    return cudaMemsetAsync(c->hkeys, 0, std::min(slots, c->hcap) * 2 * sizeof(uint64_t), c->st);
}

// empty the work queue (cursors and slots) before another traversal round
int reset_queue(skim_ctx *c, uint64_t used) {
    uint64_t u = std::min(used, c->qcap);
    if (u) CK(c, cudaMemsetAsync(c->q, 0, u * sizeof(Item), c->st));
    CK(c, cudaMemsetAsync(&c->ctl->q_head, 0, 3 * sizeof(HotCounter), c->st));
    CK(c, cudaMemsetAsync(&c->ctl->spill, 0, sizeof(unsigned), c->st));
    return SKIM_OK;
}

TravArgs base_args(skim_ctx *c, bool forward) {
    TravArgs a{};
    a.ptr = forward ? c->fptr : c->rptr;
    a.col = c->mat ? (forward ? c->flive : c->rlive) : (forward ? c->fcol : c->rcol);
    a.mat = c->mat ? 1 : 0;
    a.loff = forward ? c->foff : c->loff;
    a.lmask = forward ? c->fmask : nullptr;
    a.cm = c->cm;
    a.q = c->q;
    a.qcap = c->qcap;
    a.ctl = c->ctl;
    a.timeout_ns = c->timeout_ns;
    a.hkeys = c->hkeys;
    a.hvals = c->hvals;
    a.hmask = c->hcap - 1;
    a.rec_key = c->rkey;
    a.rec_val = c->rval;
    a.rcap = c->rcap;
    a.lane_inst = c->lane_inst;
    a.lane_g = c->lane_g;
    a.he = forward ? c->fhe : c->rhe;
    a.tm1e = forward ? c->ftm1 : c->rtm1;
    a.full = c->full;
    a.pend = c->pend;
    a.covered = c->covered;
    a.seg_start = c->seg_start;
    a.seg_len = c->seg_len;
    a.size = c->size;
    a.idx_nodes = c->idx;
    a.l = c->l;
    a.pend_trav = c->pend_trav;
    a.pend_erase = c->pend_erase;
    return a;
}

// Source lanes of a reverse batch taken by the per-warp-queue search.
struct RevSources {
    const uint32_t *lane_pair;
    uint32_t B;
    const uint64_t *covered;
    uint64_t *alive;
};

// Run traversal rounds until the queue drains with nothing spilled.  With
// `rs`, the reverse search over materialised rows (per-warp queues) takes the
// batch's sources in its first round.
int run_traversal(skim_ctx *c, TravArgs &a, bool forward, uint64_t *R_out, const RevSources *rs = nullptr) {
    for (bool first = true;; first = false) {
        {
            KTimer kt(c, forward ? SKIM_K_FWD : SKIM_K_REV);
            if (rs)
                CK(c, launch_rev_ring(a, rs->lane_pair, rs->B, c->l, rs->covered, rs->alive, first, c->grid_ring,
                                      c->st));
            else
                CK(c, launch_traverse(a, forward, forward ? c->grid_fwd : c->grid_rev, c->st));
        }
        RC(sync_ctl(c));
        const DevCtl &h = *c->hctl;
        if (h.err & kErrTimeout) {
            c->broken = true;
            return SKIM_ETIMEOUT;
        }
        if (R_out) *R_out = h.rec_count.v;
        if (h.err & kErrRetryable) return SKIM_OK;  // caller re-runs the batch
        if (!h.spill) return SKIM_OK;
        c->hstats[SKIM_STAT_REQUEUES]++;
        RC(reset_queue(c, h.q_tail.v));
        KTimer kt(c, forward ? SKIM_K_FWD : SKIM_K_REV);
        if (forward)
            CK(c, launch_respill_fwd(a, c->n, c->st));
        else
            CK(c, launch_respill_rev(a, h.rec_count.v, c->st));
    }
}

// A batch's records are placed by node (or node bucket) when there are at
// least a quarter as many of them as buckets; below that the pass over the
// counters costs more than a radix sort of the records.
constexpr uint64_t kNodeSortDensity = 4;
// widest low key part the per-node placement orders (its block pass marks
// 2^kPlaceBits bits in shared memory)
#ifndef SKIM_PLACE_BITS
#define SKIM_PLACE_BITS 19
#endif
constexpr uint32_t kPlaceBits = SKIM_PLACE_BITS;

#ifndef SKIM_TABLE_SLOTS
#define SKIM_TABLE_SLOTS 4
#endif
// visited-table slots per expected visit record of a batch, and per lane when
// the records per lane are not known yet
constexpr double kTableSlots = SKIM_TABLE_SLOTS;
#ifndef SKIM_RING_RECORDS_PER_LANE
#define SKIM_RING_RECORDS_PER_LANE 8
#endif
constexpr double kRingRecordsPerLane = SKIM_RING_RECORDS_PER_LANE;
#ifndef SKIM_NODE_HASH_WORDS
#define SKIM_NODE_HASH_WORDS 64
#endif
// batches of at most this many lane words place a node's visited-table
// entries side by side (traverse.cu: table_slot)
constexpr uint32_t kNodeHashWords = SKIM_NODE_HASH_WORDS;

int ensure_idx(skim_ctx *c, uint64_t need);

bool trace_batches() {
    static const bool on = getenv("SKIM_TRACE_BATCHES") != nullptr;
    return on;
}

// Buffers of the per-node record placement; the counters start at zero.
int node_buffers(skim_ctx *c) {
    if (c->ncnt) return SKIM_OK;
    RC(dalloc(c, &c->ncnt, static_cast<size_t>(c->n) + 1));
    RC(dalloc(c, &c->noff, static_cast<size_t>(c->n) + 1));
    RC(dalloc(c, &c->nlist, c->n));
    RC(dalloc(c, &c->nlist_cnt, 2));
    CK(c, cudaMemsetAsync(c->ncnt, 0, (static_cast<size_t>(c->n) + 1) * sizeof(uint64_t), c->st));
    return SKIM_OK;
}

// Reverse search of the batch of ranks [p0, p0+B).  mode_build: Algorithm 2
// (pruned by local counts); otherwise SKIM (covered sources skipped).
// est_per_lane: expected visit records per lane (0 or negative = unknown, or
// a re-run after an overflow: the whole table).  The visited table used is a
// power of two of about 4 slots per expected record, zeroed before the batch
// (a batch touches only its own prefix of the table, and no slot needs a
// generation tag).  A batch of searches that stay small (at most the tuned
// ring_rpl expected records per lane) runs on the per-warp queues;
// larger searches -- a lane that reaches thousands of nodes, as in the first
// batches or on hub-heavy graphs -- spread over the whole GPU through the
// global queue, whose atomic claims keep every warp fed.  Returns SKIM_OK
// with *retry set if the batch overflowed its tables.
int rev_batch(skim_ctx *c, uint64_t p0, uint32_t B, bool mode_build, bool *retry, double est_per_lane) {
    *retry = false;
    const uint32_t T = (B + 63) / 64;
    const uint32_t tbits = bitlen(T - 1);
    RC(reset_ctl(c));
    CK(c, launch_lane_inst(c->spair + p0, c->rank_mode == SKIM_RANKS_IC_MODEL ? c->srank + p0 : nullptr, B, c->l,
                           c->lane_inst, c->lane_g, c->st));
    if (!mode_build) CK(c, cudaMemsetAsync(c->alive, 0, T * sizeof(uint64_t), c->st));
    TravArgs a = base_args(c, false);
    a.tbits = tbits;
    a.hnode = T <= kNodeHashWords ? 1 : 0;
    {
        uint64_t want = c->hcap;
        if (est_per_lane > 0)
            want = static_cast<uint64_t>(kTableSlots * est_per_lane * static_cast<double>(B));
        want = pow2_at_least(std::max<uint64_t>(1ull << 16, want));
        a.hmask = std::min(want, c->hcap) - 1;
        CK(c, clear_table(c, a.hmask + 1));
    }
    // IC-model searches are never pruned: every lane is its own instance
    a.prune = mode_build && c->rank_mode != SKIM_RANKS_IC_MODEL ? 1 : 0;
    uint64_t R = 0;
#ifndef SKIM_REV_RING
#define SKIM_REV_RING 1
#endif
    // SKIM_TRACE_BATCHES=1 in the environment: one line per batch on stderr
    // (search kernel, lanes, records, visits, device time of its searches and
    // of its record sort)
    const bool trace = trace_batches();
    cudaEvent_t tr0 = nullptr, tr1 = nullptr, tr2 = nullptr;
    if (trace) {
        cudaEventCreate(&tr0);
        cudaEventCreate(&tr1);
        cudaEventCreate(&tr2);
        cudaEventRecord(tr0, c->st);
    }
    const bool use_ring = c->mat && SKIM_REV_RING && est_per_lane > 0 && est_per_lane <= c->ring_rpl;
    if (use_ring) {
        const RevSources rs{c->spair + p0, B, mode_build ? nullptr : c->covered, mode_build ? nullptr : c->alive};
        RC(run_traversal(c, a, false, &R, &rs));
    } else {
        {
            KTimer kt(c, SKIM_K_SOURCES);
            CK(c, launch_rev_sources(a, c->spair + p0, B, c->l, mode_build ? nullptr : c->covered,
                                     mode_build ? nullptr : c->alive, c->st));
        }
        RC(run_traversal(c, a, false, &R));
    }
    if (trace) cudaEventRecord(tr1, c->st);
    const auto trace_line = [&]() {
        if (!trace) return;
        cudaEventRecord(tr2, c->st);
        cudaEventSynchronize(tr2);
        float ms = 0.f, ms_sort = 0.f;
        cudaEventElapsedTime(&ms, tr0, tr1);
        cudaEventElapsedTime(&ms_sort, tr1, tr2);
        fprintf(stderr, "skim batch %s %s p0=%llu B=%u records=%llu visits=%llu ms=%.4f sort_ms=%.4f\n",
                mode_build ? "build" : "skim", use_ring ? "ring" : "queue", static_cast<unsigned long long>(p0), B,
                static_cast<unsigned long long>(R), static_cast<unsigned long long>(c->hctl->stats[kStRevVisits]), ms,
                ms_sort);
        cudaEventDestroy(tr0);
        cudaEventDestroy(tr1);
        cudaEventDestroy(tr2);
    };
    const DevCtl &h = *c->hctl;
    if (h.err & kErrRetryable) {
        *retry = true;
        RC(reset_queue(c, h.q_tail.v));
        CK(c, cudaMemsetAsync(c->pend, 0, c->hcap * sizeof(uint64_t), c->st));
        c->hstats[SKIM_STAT_RETRIES]++;
        trace_line();
        return SKIM_OK;
    }
    RC(reset_queue(c, h.q_tail.v));
    if (!mode_build) {  // SKIM: the batch's commits add at most its visit bits to the index
        const uint64_t vis = h.stats[kStRevVisits] - c->vis_seen;
        c->vis_seen = h.stats[kStRevVisits];
        RC(ensure_idx(c, c->idx_bound + vis));
        c->idx_bound += vis;
    }
    const int bits = bitlen(c->n - 1) + static_cast<int>(tbits);
    // Records are placed node by node (one pass over per-node counters) when
    // they are dense over the nodes.  Sparser batches are placed by buckets of
    // 2^sb consecutive nodes instead, about one bucket per record: a bucket's
    // records are put in (node, word) order as a node's are in word order,
    // the key's low tbits + sb bits playing the word (at most kPlaceBits, the
    // block pass's bitmap).  The rest is radix-sorted over the key bits.
    uint32_t sb = 0;
    while (sb + tbits < kPlaceBits && (static_cast<uint64_t>(c->n) >> sb) > std::max<uint64_t>(R, 1)) sb++;
    const uint32_t nb = static_cast<uint32_t>((static_cast<uint64_t>(c->n) + (1ull << sb) - 1) >> sb);
    c->bnode = static_cast<uint64_t>(nb) <= static_cast<uint64_t>(c->node_density) * R;
    if (c->bnode) RC(node_buffers(c));
    {
        KTimer kt(c, SKIM_K_SORT);
        if (c->bnode)
            CK(c, launch_node_sort(c->rkey, c->rval, R, tbits + sb, nb, c->ncnt, c->noff, c->rkey2, c->nlist,
                                   c->nlist_cnt, c->ws, c->st));
        else
            CK(c, radix_sort_pairs(c->rkey, c->rval, c->rkey2, c->rval2, R, bits, c->ws, c->st));
    }
    if (!mode_build) {
        c->rbits = c->rkey2;
        KTimer kt(c, SKIM_K_SORT);
        CK(c, launch_gather_bits(c->rval, c->hvals, R, c->rbits, c->st));
    }
    c->bR = R;
    c->btbits = tbits;
    c->hstats[SKIM_STAT_BATCHES]++;
    trace_line();
    return SKIM_OK;
}

// Release the active batch's records (the next batch zeroes the part of the
// visited table it uses).
int clear_batch(skim_ctx *c) {
    c->bR = 0;
    c->bnode = false;
    return SKIM_OK;
}

int pull_stats(skim_ctx *c) {
    RC(sync_ctl(c));
    c->hstats[SKIM_STAT_REV_VISITS] = c->hctl->stats[kStRevVisits];
    c->hstats[SKIM_STAT_REV_COINS] = c->hctl->stats[kStRevCoins];
    c->hstats[SKIM_STAT_INSERTIONS] = c->hctl->stats[kStInsert];
    c->hstats[SKIM_STAT_FWD_VISITS] = c->hctl->stats[kStFwdVisits];
    c->hstats[SKIM_STAT_FWD_COINS] = c->hctl->stats[kStFwdCoins];
    c->hstats[SKIM_STAT_REV_EDGES] = c->hctl->stats[kStRevEdges];
    c->hstats[SKIM_STAT_FWD_EDGES] = c->hctl->stats[kStFwdEdges];
    return SKIM_OK;
}

int reset_stats(skim_ctx *c) {
    CK(c, cudaMemsetAsync(c->ctl->stats, 0, sizeof(c->ctl->stats), c->st));
    std::fill(c->hstats, c->hstats + SKIM_STAT_COUNT, 0);
    c->vis_seen = 0;
    return SKIM_OK;
}

#ifndef SKIM_VISIT_BUDGET
#define SKIM_VISIT_BUDGET 4.0e6
#endif
constexpr double kSkimVisitBudget = SKIM_VISIT_BUDGET;  // visits a SKIM batch aims at
#ifndef SKIM_BUILD_GROWTH
#define SKIM_BUILD_GROWTH 32
#endif
constexpr uint64_t kBuildGrowth = SKIM_BUILD_GROWTH;  // lanes of a build batch over the last one, at most
#ifndef SKIM_BUILD_FIRST
#define SKIM_BUILD_FIRST 256
#endif
constexpr uint32_t kBuildFirst = SKIM_BUILD_FIRST;  // lanes of the first build batch

// Lanes of a rank batch when the caller sets none: 2M, and 4M on graphs of
// 2^23 nodes or more, whose batches of small searches are sparse over the
// nodes (R-MAT 24 p = 0.01: sketches and 200 seeds 1.75 -> 1.69 s; R-MAT 20
// keeps 2M: a 4M-lane batch's records take longer to order than its search
// saves).
uint64_t auto_lanes(uint64_t n) { return n >= (1ull << 23) ? (1ull << 22) : (1ull << 21); }

uint32_t default_lanes(skim_ctx *c) {
    uint64_t b = c->batch_cfg ? c->batch_cfg : auto_lanes(c->n);
    b = std::min<uint64_t>(b, static_cast<uint64_t>(kMaxWords) * 64);
    b = std::min<uint64_t>(b, c->lane_cap);
    return static_cast<uint32_t>(std::max<uint64_t>(64, b));
}

// ---- SKIM steps ------------------------------------------------------------

int skim_state_init(skim_ctx *c) {
    if (!c->covered) {
        RC(dalloc(c, &c->covered, c->n));
        RC(dalloc(c, &c->size, c->n));
        RC(dalloc(c, &c->seg_start, c->nl));
        RC(dalloc(c, &c->seg_len, c->nl));
        RC(dalloc(c, &c->chosen, c->n));
        RC(dalloc(c, &c->pend_trav, c->n));
        RC(dalloc(c, &c->pend_erase, c->n));
        RC(dalloc(c, &c->idx_ctr, 2));
    }
    CK(c, cudaMemsetAsync(c->covered, 0, c->n * sizeof(uint64_t), c->st));
    CK(c, cudaMemsetAsync(c->size, 0, c->n * sizeof(uint32_t), c->st));
    CK(c, cudaMemsetAsync(c->seg_len, 0, c->nl * sizeof(uint32_t), c->st));
    CK(c, cudaMemsetAsync(c->chosen, 0, c->n, c->st));
    CK(c, cudaMemsetAsync(c->pend_trav, 0, c->n * sizeof(uint64_t), c->st));
    CK(c, cudaMemsetAsync(c->pend_erase, 0, c->n * sizeof(uint64_t), c->st));
    if (c->batch_active) RC(clear_batch(c));
    CK(c, cudaMemsetAsync(c->idx_ctr, 0, 2 * sizeof(uint64_t), c->st));
    c->idx_bound = 0;
    c->cursor = 0;
    c->nseeds = 0;
    c->batch_active = false;
    c->skim_B = 0;
    c->since_stop = 0;
    c->last_gap = 0;
    c->vpl_est = 0;
    c->last_B = 0;
    c->sk_init = true;
    return SKIM_OK;
}

int ensure_idx(skim_ctx *c, uint64_t need) {
    if (need <= c->idx_cap) return SKIM_OK;
    uint64_t cap = std::max<uint64_t>(need + need / 2, 1ull << 22);
    uint32_t *nb = nullptr;
    RC(dalloc(c, &nb, cap));
    // every committed entry lies below idx_bound (the frees are stream-ordered)
    if (c->idx && c->idx_bound)
        CK(c, cudaMemcpyAsync(nb, c->idx, std::min(c->idx_bound, c->idx_cap) * sizeof(uint32_t),
                              cudaMemcpyDeviceToDevice, c->st));
    dfree(c, c->idx);
    c->idx = nb;
    c->idx_cap = cap;
    return SKIM_OK;
}

// Commit lanes [lo, hi] of the active batch: sizes and the inverted index.
// The index was sized for the whole batch when it was searched, and its fill
// offset stays on the device, so a commit needs no read-back.
int commit_lanes(skim_ctx *c, uint32_t lo, uint32_t hi) {
    if (lo > hi) return SKIM_OK;
    const uint32_t cnt = hi - lo + 1;
    CK(c, cudaMemsetAsync(c->lane_cnt + lo, 0, cnt * sizeof(uint64_t), c->st));
    CK(c, cudaMemsetAsync(c->lane_fill + lo, 0, cnt * sizeof(uint32_t), c->st));
    KTimer kt(c, SKIM_K_STEP);
    CK(c, launch_commit_count(c->rkey, c->rbits, c->bR, c->btbits, c->alive, lo, hi, c->size, c->lane_cnt,
                              c->ctl, c->st));
    CK(c, exclusive_scan_u64(c->lane_cnt + lo, c->lane_off + lo, cnt, reinterpret_cast<uint64_t *>(&c->ctl->total),
                             c->ws, c->st));
    CK(c, launch_commit_scatter(c->rkey, c->rbits, c->bR, c->btbits, c->alive, lo, hi, c->lane_off,
                                c->lane_fill, c->idx_ctr, c->idx, c->st));
    CK(c, launch_commit_segments(c->spair + c->bp0, lo, hi, c->lane_cnt, c->lane_off, c->idx_ctr, c->seg_start,
                                 c->seg_len, c->st));
    CK(c, launch_idx_advance(c->idx_ctr, &c->ctl->total, c->st));
    return SKIM_OK;
}

// Finish the pending residual search, after a read of the control block that
// followed it.  A search that parked work (its queue overflowed) resumes until
// the queue drains; the lane filter launched after it then runs again, and
// *again tells the caller that what it read back (stop candidate, argmax) was
// computed before the search had finished.  Then the search's count of newly
// covered pairs goes out and the queue is emptied.
int finish_residual(skim_ctx *c, bool *again) {
    *again = false;
    if (!c->pend_res) return SKIM_OK;
    c->pend_res = false;
    const DevCtl &h = *c->hctl;
    if (h.err & kErrTimeout) {
        c->broken = true;
        return SKIM_ETIMEOUT;
    }
    if (h.spill && !(h.err & kErrRetryable)) {
        *again = true;
        c->hstats[SKIM_STAT_REQUEUES]++;
        RC(reset_queue(c, h.q_tail.v));
        TravArgs a = base_args(c, true);
        {
            KTimer kt(c, SKIM_K_FWD);
            CK(c, launch_respill_fwd(a, c->n, c->st));
        }
        RC(run_traversal(c, a, true, nullptr));
        if (c->batch_active)
            CK(c, launch_refilter(c->spair + c->bp0, c->blo, c->bB, c->l, c->covered, c->alive, c->st));
    }
    *c->pend_cov = c->hctl->ix_cov;
    RC(reset_queue(c, c->hctl->q_tail.v));
    return SKIM_OK;
}

// Wait for the pending residual search, if any, and finish it.
int settle_residual(skim_ctx *c) {
    if (!c->pend_res) return SKIM_OK;
    RC(sync_ctl(c));
    bool again = false;
    return finish_residual(c, &again);
}

// Residual problem for seed x: forward search in every instance.  The search
// is launched and not waited for: the host goes on to queue the next seed's
// scan behind it, and the read-back of that scan finishes the search
// (finish_residual), storing its count of newly covered pairs at *cov.
int residual(skim_ctx *c, uint32_t x, uint64_t *cov) {
    RC(reset_ctl(c));
    TravArgs a = base_args(c, true);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    const uint64_t v0 = trace_batches() ? c->hctl->stats[kStFwdVisits] : 0;
    if (trace_batches()) {
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaEventRecord(t0, c->st);
    }
    CK(c, launch_fwd_source(a, x, c->st));
    {
        KTimer kt(c, SKIM_K_FWD);
        CK(c, launch_traverse(a, true, c->grid_fwd, c->st));
    }
    CK(c, cudaMemsetAsync(c->chosen + x, 1, 1, c->st));
    c->pend_res = true;
    c->pend_cov = cov;
    if (trace_batches()) {  // one line per residual search, waited for
        RC(settle_residual(c));
        cudaEventRecord(t1, c->st);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        fprintf(stderr, "skim residual seed=%u visits=%llu edges=%llu cov=%llu ms=%.4f\n", x,
                static_cast<unsigned long long>(c->hctl->stats[kStFwdVisits] - v0),
                static_cast<unsigned long long>(c->hctl->stats[kStFwdEdges]), static_cast<unsigned long long>(*cov),
                ms);
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    return SKIM_OK;
}

int next_seed(skim_ctx *c, uint32_t *x_out, uint64_t *cov_out) {
    for (;;) {
        if (c->batch_active) {
            CK(c, cudaMemsetAsync(&c->ctl->best, 0xff, sizeof(unsigned long long), c->st));
            {
                KTimer kt(c, SKIM_K_STEP);
                CK(c, launch_candidates(c->rkey, c->rbits, c->bR, c->btbits, c->alive, c->blo, c->size,
                                        c->k, c->ctl, c->st));
            }
            RC(sync_ctl(c));
            {
                bool again = false;
                RC(finish_residual(c, &again));
                if (again) continue;  // the scan ran before the last seed's search had finished
            }
            const uint64_t best = c->hctl->best;
            if (best != ~0ull) {
                const uint32_t p = static_cast<uint32_t>(best >> 32);
                const uint32_t x = static_cast<uint32_t>(best & 0xffffffffu);
                RC(commit_lanes(c, c->blo, p));
                if (c->rec_tau) {
                    CK(c, cudaMemcpyAsync(c->rec_tau + c->rec_j, c->srank + c->bp0 + p, sizeof(uint64_t),
                                          cudaMemcpyDeviceToDevice, c->st));
                    CK(c, launch_second_size(c->idx, c->idx_ctr + 1, c->lane_off, c->lane_cnt, p, c->size, c->n, x,
                                             c->rec_kp + c->rec_j, c->st));
                }
                RC(residual(c, x, cov_out));
                {
                    const uint64_t after = c->bB - 1 - p;  // batch lanes not yet consumed
                    c->last_gap = c->since_stop - after;
                    c->since_stop = after;
                }
                c->blo = p + 1;
                CK(c, launch_refilter(c->spair + c->bp0, c->blo, c->bB, c->l, c->covered, c->alive, c->st));
                *x_out = x;
                return SKIM_OK;
            }
            RC(commit_lanes(c, c->blo, c->bB - 1));
            RC(clear_batch(c));
            c->batch_active = false;
            continue;
        }
        if (c->cursor < c->nl) {
            RC(settle_residual(c));  // a new batch resets the control block
            // A lane can cost a whole reverse search of a giant component,
            // and lanes past the next stop are wasted if the new seed covers
            // their source.  So a batch is sized to about kSkimVisitBudget
            // visits, from the visits per lane of the previous batch (64
            // lanes first; at most 16x growth per batch), and to at most four
            // times the last gap between seeds (or the ranks consumed since the
            // last seed, if that is longer).
            uint64_t want = 64;
            if (c->vpl_est > 0) {
                want = static_cast<uint64_t>(kSkimVisitBudget / c->vpl_est);
                want = std::min<uint64_t>(want, 16ull * std::max<uint32_t>(c->last_B, 64));
                // each stop re-scans the batch for candidates: about four
                // seeds' worth of ranks per batch once the gap is known
                if (c->last_gap) want = std::min<uint64_t>(want, 4 * std::max(c->last_gap, c->since_stop));
                want = std::max<uint64_t>(want, 64);
            }
            if (c->skim_B && c->skim_B < want) want = c->skim_B;  // shrunk after an overflow
            want = std::min<uint64_t>(want, default_lanes(c));
            uint32_t B = static_cast<uint32_t>(std::min<uint64_t>(want, c->nl - c->cursor));
            bool retry = false;
            RC(rev_batch(c, c->cursor, B, false, &retry, c->vpl_est));
            if (retry) {
                if (++c->retry_run > 48) return SKIM_ENOMEM;  // the tables cannot hold even small batches
                c->skim_B = std::max<uint32_t>(64, B / 2);
                // more records than expected: a larger table too (the whole
                // table when there was no estimate yet)
                c->vpl_est = c->vpl_est > 0 ? c->vpl_est * 4 : -1.0;
                continue;
            }
            c->retry_run = 0;
            c->skim_B = 0;
            c->batch_active = true;
            c->bp0 = c->cursor;
            c->bB = B;
            c->blo = 0;
            c->cursor += B;
            c->hstats[SKIM_STAT_RANKS] += B;
            c->since_stop += B;
            c->last_B = B;
            c->vpl_est = static_cast<double>(c->bR ? c->bR : 1) / B;  // records ~ visits (one lane per entry)
            continue;
        }
        // ranks exhausted: the largest partial sketch (ties to the smallest id)
        CK(c, cudaMemsetAsync(&c->ctl->argmax, 0, sizeof(unsigned long long), c->st));
        CK(c, launch_argmax_size(c->size, c->n, c->ctl, c->st));
        RC(sync_ctl(c));
        {
            bool again = false;
            RC(finish_residual(c, &again));
            if (again) continue;  // the sizes were read before the last seed's search had finished
        }
        uint64_t am = c->hctl->argmax;
        uint32_t x = 0xffffffffu - static_cast<uint32_t>(am & 0xffffffffu);
        if ((am >> 32) == 0) {
            CK(c, cudaMemsetAsync(&c->ctl->best, 0xff, sizeof(unsigned long long), c->st));
            CK(c, launch_min_unchosen(c->chosen, c->n, c->ctl, c->st));
            RC(sync_ctl(c));
            x = static_cast<uint32_t>(c->hctl->best);
        }
        if (c->rec_tau) {  // exact residual counts: recorded as k' = -1, tau = 0
            CK(c, cudaMemsetAsync(c->rec_kp + c->rec_j, 0xff, sizeof(uint32_t), c->st));
            CK(c, cudaMemsetAsync(c->rec_tau + c->rec_j, 0, sizeof(uint64_t), c->st));
        }
        RC(residual(c, x, cov_out));
        *x_out = x;
        return SKIM_OK;
    }
}

// Materialise the l live-edge instances (Section 2: Algorithms 1 and 2 take a
// set of instances): every edge's coins once per instance, then the live
// in-neighbour rows.  The IC model has an instance per position and keeps
// drawing coins during the searches; so does a context whose live pairs would
// not fit 32-bit row offsets.
int make_instances(skim_ctx *c) {
    c->mat = false;
    c->live_ready = false;
    if (c->rank_mode == SKIM_RANKS_IC_MODEL) return SKIM_OK;
    KTimer kt(c, SKIM_K_INSTANCES);
    if (!c->loff) {
        RC(dalloc(c, &c->rmask, std::max<uint64_t>(c->m, 1)));
        RC(dalloc(c, &c->fmask, std::max<uint64_t>(c->m, 1)));
        RC(dalloc(c, &c->loff, c->nl + 1));
        RC(dalloc(c, &c->foff, c->nl + 1));
        RC(dalloc_bytes(c, &c->pieces, live_pieces_bytes(c->m)));
    }
    // counts per (v, i) scanned into 64-bit offsets, kept as 32-bit offsets
    uint64_t *off = nullptr;
    RC(dalloc(c, &off, c->nl + 1));
    CK(c, launch_live_masks(c->rrow, c->rcol, c->rhe, c->rtm1, c->rev2fwd, c->cm, c->m, c->l, c->rmask, c->fmask,
                            c->st));
    CK(c, launch_live_count(c->rptr, c->rmask, c->n, c->m, c->l, off, c->pieces, c->st));
    CK(c, cudaMemsetAsync(off + c->nl, 0, sizeof(uint64_t), c->st));
    CK(c, exclusive_scan_u64(off, off, c->nl + 1, nullptr, c->ws, c->st));
    CK(c, cudaMemcpyAsync(&c->live_total, off + c->nl, sizeof(uint64_t), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (c->live_total > kRowMask) {  // offsets would not fit 31 bits: coins are drawn in the searches
        dfree(c, off);
        return SKIM_OK;
    }
    if (c->live_total > c->rlive_cap) {
        dfree(c, c->rlive);
        dfree(c, c->flive);
        c->rlive_cap = 0;
        RC(dalloc(c, &c->rlive, c->live_total));
        RC(dalloc(c, &c->flive, c->live_total));
        c->rlive_cap = c->live_total;
    }
    CK(c, launch_live_fill(c->rptr, c->rcol, c->rmask, c->n, c->m, c->l, off, c->rlive, c->pieces, c->st));
    CK(c, launch_offsets_u32(off, c->nl, c->loff, c->st));
    // the same live pairs by tail: rows of live out-neighbours for the residual
    CK(c, launch_live_count(c->fptr, c->fmask, c->n, c->m, c->l, off, c->pieces, c->st));
    CK(c, cudaMemsetAsync(off + c->nl, 0, sizeof(uint64_t), c->st));
    CK(c, exclusive_scan_u64(off, off, c->nl + 1, nullptr, c->ws, c->st));
    CK(c, launch_live_fill(c->fptr, c->fcol, c->fmask, c->n, c->m, c->l, off, c->flive, c->pieces, c->st));
    CK(c, launch_offsets_u32(off, c->nl, c->foff, c->st));
    dfree(c, off);
    c->live_ready = true;
    c->mat = c->mat_wanted;
    return SKIM_OK;
}

int rank_order(skim_ctx *c) {
    {
        KTimer kt(c, SKIM_K_RANKS);
        if (c->rank_mode == SKIM_RANKS_UNIFORM)
            CK(c, rank_sort(c->rank_key, c->rbase, c->l, c->nl, c->srank, c->spair, c->rank_ws, c->st));
        else
            CK(c, perm_sort(c->rank_key, c->n, c->l, static_cast<uint32_t>(c->npos / c->n),
                            c->rank_mode == SKIM_RANKS_IC_MODEL, c->srank, c->spair, c->rank_ws, c->st));
    }
    CK(c, cudaStreamSynchronize(c->st));
    resolve_timers(c);
    return SKIM_OK;
}

int ensure_query_space(skim_ctx *c, uint64_t seeds, uint64_t q, uint64_t table, uint64_t chunks) {
    if (chunks > c->qpart_cap) {
        dfree(c, c->qpart);
        c->qpart_cap = std::max<uint64_t>(chunks, 1024);
        const int rc = dalloc_bytes(c, &c->qpart, c->qpart_cap * query_partial_bytes());
        if (rc != SKIM_OK) {
            c->qpart_cap = 0;
            return rc;
        }
    }
    if (seeds > c->qseeds_cap) {
        dfree(c, c->qseeds);
        c->qseeds_cap = std::max<uint64_t>(seeds, 4096);
        RC(dalloc(c, &c->qseeds, c->qseeds_cap));
    }
    if (q + 1 > c->qmeta_cap) {
        dfree(c, c->qoff);
        dfree(c, c->qout);
        dfree(c, c->qtop);
        dfree(c, c->qtopu);
        c->qmeta_cap = std::max<uint64_t>(q + 1, 1024);
        RC(dalloc(c, &c->qoff, 3 * c->qmeta_cap));  // seed, table and chunk offsets in one upload
        RC(dalloc(c, &c->qout, c->qmeta_cap));
        RC(dalloc(c, &c->qtop, c->qmeta_cap));
        RC(dalloc(c, &c->qtopu, c->qmeta_cap));
    }
    if (table > c->qtcap) {
        dfree(c, c->qk);
        dfree(c, c->qv);
        c->qtcap = std::max<uint64_t>(table, 1ull << 16);
        RC(dalloc(c, &c->qk, c->qtcap));
        RC(dalloc(c, &c->qv, c->qtcap));
    }
    return SKIM_OK;
}

uint64_t query_table(uint64_t s, uint32_t k) { return pow2_at_least(std::max<uint64_t>(64, 2 * s * (k - 1) + 2)); }

}  // namespace

QueryTerms skim::query_terms_of(const skim_ctx *c) {
    if (c->rank_mode == SKIM_RANKS_PERMUTATION)
        return QueryTerms{1, static_cast<double>(c->nl - 1), static_cast<double>(c->l)};
    if (c->rank_mode == SKIM_RANKS_IC_MODEL) return QueryTerms{2, static_cast<double>(c->n), 1.0};
    return QueryTerms{0, 0.0, static_cast<double>(c->l)};
}

extern "C" {

const char *skim_strerror(int code) {
    switch (code) {
        case SKIM_OK: return "ok";
        case SKIM_EINVAL: return "invalid argument";
        case SKIM_ENOMEM: return "out of memory";
        case SKIM_ENOTBUILT: return "sketches not built";
        case SKIM_ETIMEOUT: return "device wait timed out";
        case SKIM_ECUDA: return "CUDA error";
        case SKIM_EGRAPH: return "edge list not canonical";
        case SKIM_ERANGE: return "size out of range";
        default: return "unknown error";
    }
}

int skim_destroy(skim_ctx *c) {
    if (!c) return SKIM_EINVAL;
    cudaStreamSynchronize(c->st);
    dfree(c, c->fptr); dfree(c, c->fcol); dfree(c, c->rptr); dfree(c, c->rcol); dfree(c, c->thr_wc);
    dfree(c, c->rhe); dfree(c, c->fhe);
    dfree(c, c->srank); dfree(c, c->spair);
    dfree(c, c->rank_ws);
    dfree(c, c->rbase); dfree(c, c->rtm1); dfree(c, c->ftm1);
    dfree(c, c->ctl); dfree(c, c->dflag);
    if (c->hctl) cudaFreeHost(c->hctl);
    dfree(c, c->q); dfree(c, c->hkeys); dfree(c, c->pend);
    c->hvals = nullptr;
    dfree(c, c->rkey); dfree(c, c->rkey2); dfree(c, c->rval); dfree(c, c->rval2);
    dfree(c, c->ncnt); dfree(c, c->noff); dfree(c, c->nlist); dfree(c, c->nlist_cnt);
    dfree(c, c->ws);
    dfree(c, c->lane_inst); dfree(c, c->lane_g); dfree(c, c->alive); dfree(c, c->lane_cnt); dfree(c, c->lane_off); dfree(c, c->lane_fill);
    dfree(c, c->lcnt); dfree(c, c->full); dfree(c, c->X); dfree(c, c->xlen);
    dfree(c, c->covered); dfree(c, c->seg_start); dfree(c, c->pend_trav); dfree(c, c->pend_erase);
    dfree(c, c->size); dfree(c, c->seg_len); dfree(c, c->idx); dfree(c, c->chosen);
    dfree(c, c->rec_tau); dfree(c, c->rec_kp); dfree(c, c->idx_ctr);
    dfree(c, c->rmask); dfree(c, c->fmask); dfree(c, c->loff); dfree(c, c->rlive); dfree(c, c->rrow); dfree(c, c->rev2fwd);
    dfree(c, c->foff); dfree(c, c->flive);
    dfree(c, c->pieces);
    dfree(c, c->qk); dfree(c, c->qv); dfree(c, c->qseeds); dfree(c, c->qoff); dfree(c, c->qout);
    dfree(c, c->qtop); dfree(c, c->qtopu);
    dfree(c, c->qpart);
    for (auto &p : c->kpend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->kpool) cudaEventDestroy(e);
    delete c;
    return SKIM_OK;
}

int skim_release_memory(void) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < kMaxDevices; d++)
        if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) {
            cudaGetLastError();
            return SKIM_ECUDA;
        }
    return SKIM_OK;
}

int skim_create(const skim_graph *g, const skim_params *prm, void *stream, skim_ctx **out) {
    if (!g || !prm || !out) return SKIM_EINVAL;
    *out = nullptr;
    if (g->n == 0 || prm->l == 0 || prm->l > 64 || prm->k < 2 || prm->k > 255) return SKIM_EINVAL;
    if (prm->prob_model < 0 || prm->prob_model > 2) return SKIM_EINVAL;
    if (prm->prob_model == 0 && !(prm->p > 0.0 && prm->p <= 1.0)) return SKIM_EINVAL;
    if (prm->prob_model == 0 && prm->p < 1.0 && static_cast<uint64_t>(std::ldexp(prm->p, 64)) == 0) return SKIM_EINVAL;
    if (g->m && (!g->src || !g->dst)) return SKIM_EINVAL;
    if (g->m >= (1ull << 32)) return SKIM_ERANGE;
    if (prm->rank_mode > SKIM_RANKS_IC_MODEL) return SKIM_EINVAL;
    if (prm->rank_mode == SKIM_RANKS_IC_MODEL && prm->l != 1) return SKIM_EINVAL;
    const uint64_t nl = static_cast<uint64_t>(g->n) * prm->l;
    if (nl > 0xffffffffull) return SKIM_ERANGE;
    // positions of the rank order, and those the sketch build needs (with
    // permutation ranks every node owns one position per chunk, so no position
    // past min(k, l) chunks can enter a sketch)
    uint64_t npos = nl, nbuild = nl;
    if (prm->rank_mode == SKIM_RANKS_PERMUTATION) nbuild = static_cast<uint64_t>(std::min(prm->k, prm->l)) * g->n;
    if (prm->rank_mode == SKIM_RANKS_IC_MODEL) npos = nbuild = static_cast<uint64_t>(prm->k) * g->n;
    if (npos > 0xffffffffull) return SKIM_ERANGE;

    skim_ctx *c = new (std::nothrow) skim_ctx();
    if (!c) return SKIM_ENOMEM;
    cudaGetDevice(&c->device);
    c->st = static_cast<cudaStream_t>(stream);
    c->n = g->n;
    c->m = g->m;
    c->l = prm->l;
    c->k = prm->k;
    c->nl = nl;
    c->rank_mode = static_cast<int>(prm->rank_mode);
    c->npos = npos;
    c->nbuild = nbuild;
    c->batch_cfg = prm->batch_lanes;
    c->ring_rpl = kRingRecordsPerLane;
    c->node_density = static_cast<uint32_t>(kNodeSortDensity);
    c->cm.model = prm->prob_model;
    c->cm.tm1_uniform = prm->prob_model == 0 ? tm1_of(prm->p) : 0;
    c->cm.tm1_class[0] = tm1_of(0.1);
    c->cm.tm1_class[1] = tm1_of(0.01);
    c->cm.tm1_class[2] = tm1_of(0.001);
    c->cm.coin_key = prm->coin_key;
    c->cm.prob_key = prm->prob_key;
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    int rc = SKIM_OK;
#define TRY(x)                       \
    do {                             \
        rc = (x);                    \
        if (rc != SKIM_OK) goto fail; \
    } while (0)
#define TRYC(x)                                  \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) {                 \
            rc = fail_cuda(c, e_);               \
            goto fail;                           \
        }                                        \
    } while (0)
    {
        TRY(dalloc(c, &c->ctl, 1));
        TRYC(cudaMallocHost(reinterpret_cast<void **>(&c->hctl), sizeof(DevCtl)));
        TRYC(cudaMemsetAsync(c->ctl, 0, sizeof(DevCtl), c->st));
        TRY(dalloc(c, &c->dflag, 1));
        // edges on the device
        uint32_t *dsrc = nullptr, *ddst = nullptr;
        bool own_edges = !g->on_device;
        if (own_edges) {
            TRY(dalloc(c, &dsrc, m));
            TRY(dalloc(c, &ddst, m));
            if (m) {
                TRYC(cudaMemcpyAsync(dsrc, g->src, m * sizeof(uint32_t), cudaMemcpyHostToDevice, c->st));
                TRYC(cudaMemcpyAsync(ddst, g->dst, m * sizeof(uint32_t), cudaMemcpyHostToDevice, c->st));
            }
        } else {
            dsrc = const_cast<uint32_t *>(g->src);
            ddst = const_cast<uint32_t *>(g->dst);
        }
        TRYC(cudaMemsetAsync(c->dflag, 0, sizeof(unsigned), c->st));
        TRYC(launch_check_edges(dsrc, ddst, m, n, c->dflag, c->st));
        unsigned bad = 0;
        TRYC(cudaMemcpyAsync(&bad, c->dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
        TRYC(cudaStreamSynchronize(c->st));
        if (bad) {
            if (own_edges) { dfree(c, dsrc); dfree(c, ddst); }
            rc = SKIM_EGRAPH;
            goto fail;
        }
        // workspace for scans and sorts
        // visit records per batch: a few per lane; sized generously so that
        // re-running a batch with fewer lanes stays rare
        const uint64_t lanes_max = std::min<uint64_t>(npos, prm->batch_lanes ? prm->batch_lanes : auto_lanes(g->n));
#ifndef SKIM_RECORDS_PER_LANE
#define SKIM_RECORDS_PER_LANE 16
#endif
        uint64_t rcap =
            std::min<uint64_t>(std::max<uint64_t>(SKIM_RECORDS_PER_LANE * lanes_max, 1u << 20), 1ull << 26);
        // SKIM_RECORD_ITEMS in the environment (a test hook): that many visit
        // records (and twice as many table slots), so that batches overflow
        // and are re-run with fewer lanes
        if (const char *ri = getenv("SKIM_RECORD_ITEMS")) rcap = std::max<uint64_t>(64, strtoull(ri, nullptr, 10));
        size_t ws = std::max({scan_workspace_bytes(static_cast<size_t>(n) + 1), scan_workspace_bytes(nl + 1),
                              scan_workspace_bytes(rcap + 1),
                              radix_workspace_bytes(m),
                              radix_workspace_bytes(rcap), scan_workspace_bytes(static_cast<size_t>(kMaxWords) * 64)});
        c->ws_bytes = ws;
        TRY(dalloc_bytes(c, &c->ws, ws));
        // forward CSR: rows of the (src,dst)-sorted list
        TRY(dalloc(c, &c->fptr, static_cast<size_t>(n) + 1));
        TRY(dalloc(c, &c->rptr, static_cast<size_t>(n) + 1));
        TRY(dalloc(c, &c->fcol, m));
        TRY(dalloc(c, &c->rcol, m));
        TRY(dalloc(c, &c->rrow, m));
        TRY(dalloc(c, &c->rev2fwd, m));
        TRYC(launch_row_ptr(dsrc, m, n, c->fptr, c->st));
        if (m) TRYC(cudaMemcpyAsync(c->fcol, ddst, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->st));
        // reverse CSR: (dst, src) order, by a stable sort on the dst bits
        if (m) {
            uint64_t *k1 = nullptr, *k2 = nullptr;
            uint32_t *v1 = nullptr, *v2 = nullptr;
            TRY(dalloc(c, &k1, m));
            TRY(dalloc(c, &k2, m));
            TRY(dalloc(c, &v1, m));
            TRY(dalloc(c, &v2, m));
            TRYC(launch_make_rev_keys(dsrc, ddst, m, k1, v1, c->st));
            TRYC(radix_sort_pairs(k1, v1, k2, v2, m, std::max(1, bitlen(n - 1)), c->ws, c->st));
            TRYC(launch_split_rev(k1, v1, m, c->rcol, c->rrow, c->rev2fwd, c->st));
            dfree(c, k1); dfree(c, k2); dfree(c, v1); dfree(c, v2);  // (stream-ordered)
        }
        TRYC(launch_row_ptr(c->rrow, m, n, c->rptr, c->st));
        if (own_edges) { dfree(c, dsrc); dfree(c, ddst); }
        TRYC(cudaMemsetAsync(c->ctl, 0, sizeof(DevCtl), c->st));
        TRY(dalloc(c, &c->rhe, m));
        TRY(dalloc(c, &c->fhe, m));
        TRYC(launch_edge_states_both(c->rcol, c->rrow, c->rev2fwd, m, prm->coin_key, c->rhe, c->fhe, c->st));
        if (prm->prob_model == 1) {
            TRY(dalloc(c, &c->thr_wc, n));
            TRYC(launch_wc_thresholds(c->rptr, n, c->thr_wc, c->st));
        }
        c->cm.thr_wc = c->thr_wc;
        TRY(make_instances(c));
        // rank order of the n*l pairs
        TRY(dalloc(c, &c->srank, npos));
        TRY(dalloc(c, &c->spair, npos));
        TRY(dalloc_bytes(c, &c->rank_ws, c->rank_mode == SKIM_RANKS_UNIFORM
                                             ? rank_sort_workspace_bytes(nl)
                                             : perm_sort_workspace_bytes(n, c->l, static_cast<uint32_t>(npos / n),
                                                                         c->rank_mode == SKIM_RANKS_IC_MODEL)));
        c->rank_key = prm->rank_key;
        TRY(rank_order(c));
        // traversal scratch
        c->lane_cap = static_cast<uint32_t>(std::min<uint64_t>(pow2_at_least(std::min<uint64_t>(npos, kMaxWords * 64ull)),
                                                               kMaxWords * 64ull));
        if (c->lane_cap < 64) c->lane_cap = 64;
        c->rcap = rcap;
        c->hcap = pow2_at_least(2 * rcap);
        c->qcap = std::max<uint64_t>(rcap, 1u << 22);
        // SKIM_QUEUE_ITEMS in the environment (a test hook): a queue of that
        // many items, so that searches overflow it and park their work in
        // the pending masks, which are re-queued after the queue drains
        if (const char *qi = getenv("SKIM_QUEUE_ITEMS"))
            c->qcap = std::max<uint64_t>(64, strtoull(qi, nullptr, 10));
        TRY(dalloc(c, &c->q, c->qcap));
        TRYC(cudaMemsetAsync(c->q, 0, c->qcap * sizeof(Item), c->st));
        // one array of 16-byte slots: key at [2h], lane bits at [2h + 1]
        TRY(dalloc(c, &c->hkeys, 2 * c->hcap));
        c->hvals = c->hkeys + 1;
        TRY(dalloc(c, &c->pend, c->hcap));
        TRYC(clear_table(c, c->hcap));
        TRYC(cudaMemsetAsync(c->pend, 0, c->hcap * sizeof(uint64_t), c->st));
        TRY(dalloc(c, &c->rkey, c->rcap));
        TRY(dalloc(c, &c->rkey2, c->rcap + 1));  // radix sort's alternate keys; node placement's scratch
        TRY(dalloc(c, &c->rval, c->rcap));
        TRY(dalloc(c, &c->rval2, c->rcap + 1));
        TRY(dalloc(c, &c->lane_inst, c->lane_cap));
        TRYC(cudaMemsetAsync(c->lane_inst, 0, c->lane_cap, c->st));
        TRY(dalloc(c, &c->lane_g, c->lane_cap));
        TRY(dalloc(c, &c->alive, c->lane_cap / 64 + 1));
        TRY(dalloc(c, &c->lane_cnt, c->lane_cap));
        TRY(dalloc(c, &c->lane_off, c->lane_cap));
        TRY(dalloc(c, &c->lane_fill, c->lane_cap));
        c->grid_rev = traverse_grid(false);
        c->grid_ring = rev_ring_grid();
        c->grid_fwd = traverse_grid(true);
        TRYC(cudaStreamSynchronize(c->st));
    }
#undef TRY
#undef TRYC
    *out = c;
    return SKIM_OK;
fail:
    skim_destroy(c);
    return rc;
}

int skim_create_batch(const skim_graph *graphs, const skim_params *prm, uint32_t count, void *stream,
                      skim_ctx **out) {
    if (!graphs || !prm || !out || count == 0) return SKIM_EINVAL;
    *out = nullptr;
    const uint32_t l = prm[0].l, k = prm[0].k;
    uint64_t n_tot = 0, m_tot = 0;
    std::vector<uint32_t> node_off(count + 1, 0);
    std::vector<uint64_t> ck(count), rk(count), pk(count), tu(count);
    std::vector<int> model(count);
    for (uint32_t g = 0; g < count; g++) {
        const skim_params &p = prm[g];
        if (graphs[g].on_device) return SKIM_EINVAL;  // host edge lists only
        if (graphs[g].n == 0 || p.l != l || p.k != k) return SKIM_EINVAL;
        if (p.rank_mode != SKIM_RANKS_UNIFORM) return SKIM_EINVAL;  // per-graph rank bases are uniform ranks
        if (p.prob_model < 0 || p.prob_model > 2) return SKIM_EINVAL;
        if (p.prob_model == 0 && !(p.p > 0.0 && p.p <= 1.0)) return SKIM_EINVAL;
        if (graphs[g].m && (!graphs[g].src || !graphs[g].dst)) return SKIM_EINVAL;
        node_off[g] = static_cast<uint32_t>(n_tot);
        n_tot += graphs[g].n;
        m_tot += graphs[g].m;
        if (n_tot >= (1ull << 32) || m_tot >= (1ull << 32)) return SKIM_ERANGE;
        ck[g] = p.coin_key;
        rk[g] = p.rank_key;
        pk[g] = p.prob_key;
        model[g] = p.prob_model;
        tu[g] = p.prob_model == 0 ? tm1_of(p.p) : 0;
    }
    node_off[count] = static_cast<uint32_t>(n_tot);
    // the disjoint union: graph g's node v becomes node_off[g] + v (the
    // concatenated lists stay sorted)
    std::vector<uint32_t> us(m_tot), ud(m_tot);
    uint64_t e = 0;
    for (uint32_t g = 0; g < count; g++) {
        for (uint64_t j = 0; j < graphs[g].m; j++, e++) {
            if (graphs[g].src[j] >= graphs[g].n || graphs[g].dst[j] >= graphs[g].n) return SKIM_EGRAPH;
            us[e] = graphs[g].src[j] + node_off[g];
            ud[e] = graphs[g].dst[j] + node_off[g];
        }
    }
    skim_graph ug{static_cast<uint32_t>(n_tot), m_tot, us.data(), ud.data(), 0};
    skim_params up = prm[0];
    up.prob_model = 1;  // builds the per-node 1/indeg thresholds; replaced by per-edge thresholds below
    skim_ctx *c = nullptr;
    int rc = skim_create(&ug, &up, stream, &c);
    if (rc) return rc;
    auto fail = [&](int r) {
        skim_destroy(c);
        return r;
    };
    // per-graph tables on the device
    uint32_t *d_off = nullptr, *d_ng = nullptr;
    uint64_t *d_keys = nullptr;
    int *d_model = nullptr;
    if ((rc = dalloc(c, &d_off, count + 1)) || (rc = dalloc(c, &d_ng, n_tot)) || (rc = dalloc(c, &d_keys, 4ull * count)) ||
        (rc = dalloc(c, &d_model, count)))
        return fail(rc);
    std::vector<uint64_t> keys;
    keys.insert(keys.end(), ck.begin(), ck.end());
    keys.insert(keys.end(), rk.begin(), rk.end());
    keys.insert(keys.end(), pk.begin(), pk.end());
    keys.insert(keys.end(), tu.begin(), tu.end());
    BatchDesc b{count, d_ng, d_off, d_keys, d_keys + count, d_keys + 2 * count, d_keys + 3 * count, d_model,
                {tm1_of(0.1), tm1_of(0.01), tm1_of(0.001)}};
    bool ok = cudaMemcpyAsync(d_off, node_off.data(), (count + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, c->st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(d_keys, keys.data(), keys.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, c->st) ==
                  cudaSuccess &&
              cudaMemcpyAsync(d_model, model.data(), count * sizeof(int), cudaMemcpyHostToDevice, c->st) == cudaSuccess &&
              launch_node_graph(d_off, count, d_ng, c->st) == cudaSuccess;
    if (ok) {
        if ((rc = dalloc(c, &c->rbase, n_tot)) || (rc = dalloc(c, &c->rtm1, m_tot)) || (rc = dalloc(c, &c->ftm1, m_tot)))
            return fail(rc);
        ok = launch_edge_states_batch(c->rptr, c->rcol, c->n, b, 1, c->rhe, c->st) == cudaSuccess &&
             launch_edge_states_batch(c->fptr, c->fcol, c->n, b, 0, c->fhe, c->st) == cudaSuccess &&
             launch_edge_tm1_batch(c->rptr, c->rcol, c->n, b, c->thr_wc, 1, c->rtm1, c->st) == cudaSuccess &&
             launch_edge_tm1_batch(c->fptr, c->fcol, c->n, b, c->thr_wc, 0, c->ftm1, c->st) == cudaSuccess &&
             launch_rank_bases(b, c->n, c->l, c->rbase, c->st) == cudaSuccess;
    }
    if (ok) ok = cudaStreamSynchronize(c->st) == cudaSuccess;
    dfree(c, d_off);
    dfree(c, d_ng);
    dfree(c, d_keys);
    dfree(c, d_model);
    if (!ok) return fail(fail_cuda(c, cudaGetLastError()));
    c->cm.model = 3;
    c->batch_count = count;
    if ((rc = make_instances(c))) return fail(rc);
    if ((rc = rank_order(c))) return fail(rc);
    *out = c;
    return SKIM_OK;
}

int skim_autotune_batch_lanes(skim_ctx *c, const uint32_t *candidates, uint32_t count, uint32_t *best,
                              double *seconds) {
    if (!c || !candidates || !count || !best) return SKIM_EINVAL;
    double best_t = 1e300;
    uint32_t best_b = c->batch_cfg;
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) return fail_cuda(c, cudaGetLastError());
    int rc = SKIM_OK;
    for (uint32_t i = 0; i < count && rc == SKIM_OK; i++) {
        c->batch_cfg = std::max<uint32_t>(64, candidates[i]);
        cudaEventRecord(a, c->st);
        rc = skim_build_sketches(c);
        cudaEventRecord(z, c->st);
        cudaEventSynchronize(z);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, z);
        if (seconds) seconds[i] = ms / 1000.0;
        if (rc == SKIM_OK && ms < best_t) {
            best_t = ms;
            best_b = c->batch_cfg;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    c->batch_cfg = best_b;
    *best = best_b;
    return rc;
}

int skim_get_tuning(skim_ctx *c, skim_tuning *out) {
    if (!c || !out) return SKIM_EINVAL;
    out->batch_lanes = c->batch_cfg;
    out->ring_records_per_lane = c->ring_rpl;
    out->node_sort_density = c->node_density;
    return SKIM_OK;
}

int skim_set_tuning(skim_ctx *c, const skim_tuning *t) {
    if (!c || !t) return SKIM_EINVAL;
    if (!(t->ring_records_per_lane >= 0.0)) return SKIM_EINVAL;
    c->batch_cfg = t->batch_lanes;
    c->ring_rpl = t->ring_records_per_lane;
    c->node_density = t->node_sort_density;
    return SKIM_OK;
}

int skim_autotune(skim_ctx *c, const skim_tuning *candidates, uint32_t count, uint32_t *best, double *seconds) {
    if (!c || !candidates || !count || !best) return SKIM_EINVAL;
    for (uint32_t i = 0; i < count; i++)
        if (!(candidates[i].ring_records_per_lane >= 0.0)) return SKIM_EINVAL;
    skim_tuning keep{};
    skim_get_tuning(c, &keep);
    double best_t = 1e300;
    uint32_t best_i = count;
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) return fail_cuda(c, cudaGetLastError());
    int rc = SKIM_OK;
    for (uint32_t i = 0; i < count && rc == SKIM_OK; i++) {
        skim_set_tuning(c, &candidates[i]);
        if (c->batch_cfg) c->batch_cfg = std::max<uint32_t>(64, c->batch_cfg);
        cudaEventRecord(a, c->st);
        rc = skim_build_sketches(c);
        cudaEventRecord(z, c->st);
        cudaEventSynchronize(z);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, z);
        if (seconds) seconds[i] = ms / 1000.0;
        if (rc == SKIM_OK && ms < best_t) {
            best_t = ms;
            best_i = i;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    skim_set_tuning(c, best_i < count ? &candidates[best_i] : &keep);
    if (c->batch_cfg) c->batch_cfg = std::max<uint32_t>(64, c->batch_cfg);
    *best = best_i;
    return rc;
}

int skim_rank_order(skim_ctx *c) {
    if (!c) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (c->batch_active) {
        RC(clear_batch(c));
        c->batch_active = false;
    }
    RC(rank_order(c));
    c->sk_init = false;
    return SKIM_OK;
}

int skim_instances(skim_ctx *c) {
    if (!c) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (c->batch_active) {
        RC(clear_batch(c));
        c->batch_active = false;
    }
    RC(make_instances(c));
    c->sk_init = false;
    return SKIM_OK;
}

int skim_instance_stats(skim_ctx *c, uint64_t *live_pairs, int *materialised) {
    if (!c || !live_pairs || !materialised) return SKIM_EINVAL;
    *live_pairs = c->live_total;
    *materialised = c->mat ? 1 : 0;
    return SKIM_OK;
}

int skim_build_sketches(skim_ctx *c) {
    if (!c) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (!c->X) {
        RC(dalloc(c, &c->lcnt, c->nl));
        RC(dalloc(c, &c->full, c->n));
        RC(dalloc(c, &c->X, static_cast<size_t>(c->n) * c->k));
        RC(dalloc(c, &c->xlen, c->n));
    }
    if (c->batch_active) {  // a SKIM batch holds the visited table: release it
        RC(commit_lanes(c, c->blo, c->bB - 1));
        RC(clear_batch(c));
        c->batch_active = false;
    }
    CK(c, cudaMemsetAsync(c->lcnt, 0, c->nl, c->st));
    CK(c, cudaMemsetAsync(c->full, 0, c->n * sizeof(uint64_t), c->st));
    if (c->mat) CK(c, launch_clear_row_flags(c->loff, c->nl, c->st));
    CK(c, cudaMemsetAsync(c->X, 0, static_cast<size_t>(c->n) * c->k * sizeof(uint64_t), c->st));
    CK(c, cudaMemsetAsync(c->xlen, 0, c->n * sizeof(uint32_t), c->st));
    RC(reset_stats(c));
    c->built = false;
    const uint32_t Bmax = default_lanes(c);
    // The first batch is small: the searches of the lowest ranks can each
    // reach a large part of the graph (thousands of records per lane on
    // hub-heavy graphs), and the next batch is sized from this one.
    uint32_t B = std::min<uint32_t>(Bmax, kBuildFirst);
    uint64_t p0 = 0;
    double rpl = 0;  // records per lane of the last batch (0: unknown)
    while (p0 < c->nbuild) {
        uint32_t b = static_cast<uint32_t>(std::min<uint64_t>(B, c->nbuild - p0));
        bool retry = false;
        RC(rev_batch(c, p0, b, true, &retry, rpl));
        if (retry) {
            if (b <= 64) return SKIM_ENOMEM;  // even the smallest batch overflows the tables
            B = std::max<uint32_t>(64, b / 4);
            rpl = -1;  // the whole table for the re-run
            continue;
        }
        {
            KTimer kt(c, SKIM_K_ACCEPT);
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            if (trace_batches()) {
                cudaEventCreate(&t0);
                cudaEventCreate(&t1);
                cudaEventRecord(t0, c->st);
            }
            CK(c, launch_accept(c->rkey, c->rval, c->hvals, c->bR, c->btbits, c->lane_inst, c->srank + p0, c->l,
                                c->k, c->lcnt, c->full, c->mat ? c->loff : nullptr, c->X, c->xlen, c->ctl, c->st));
            if (trace_batches()) {
                cudaEventRecord(t1, c->st);
                cudaEventSynchronize(t1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                fprintf(stderr, "skim accept p0=%llu ms=%.4f\n", static_cast<unsigned long long>(p0), ms);
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
            }
        }
        const uint64_t recs = c->bR;
        RC(clear_batch(c));
        p0 += b;
        c->hstats[SKIM_STAT_RANKS] += b;
        // next batch: up to kBuildGrowth times larger, but keep the visit
        // records near a quarter of the table (dense instances can give
        // thousands of records per lane).  Each batch costs at least the
        // latency of its deepest search, so small batches are left quickly.
        const double per_lane = static_cast<double>(recs ? recs : 1) / b;
        rpl = per_lane;
#ifndef SKIM_BUILD_FILL
#define SKIM_BUILD_FILL 4.0
#endif
        const uint64_t fit = static_cast<uint64_t>(static_cast<double>(c->rcap) / SKIM_BUILD_FILL / per_lane);
        B = static_cast<uint32_t>(std::max<uint64_t>(64, std::min<uint64_t>({Bmax, kBuildGrowth * B, fit})));
    }
    uint64_t batches = c->hstats[SKIM_STAT_BATCHES], ranks = c->hstats[SKIM_STAT_RANKS],
             retries = c->hstats[SKIM_STAT_RETRIES];
    RC(pull_stats(c));
    c->hstats[SKIM_STAT_BATCHES] = batches;
    c->hstats[SKIM_STAT_RANKS] = ranks;
    c->hstats[SKIM_STAT_RETRIES] = retries;
    c->built = true;
    return SKIM_OK;
}

int skim_get_sketches(skim_ctx *c, uint64_t *x_out, uint32_t *len_out, int out_on_device) {
    if (!c || !x_out || !len_out) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (!c->built) return SKIM_ENOTBUILT;
    cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(c, cudaMemcpyAsync(x_out, c->X, static_cast<size_t>(c->n) * c->k * sizeof(uint64_t), kind, c->st));
    CK(c, cudaMemcpyAsync(len_out, c->xlen, c->n * sizeof(uint32_t), kind, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    return SKIM_OK;
}

int skim_get_sketch(skim_ctx *c, uint32_t v, uint64_t *out_k, uint32_t *out_len) {
    if (!c || !out_k || !out_len) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (!c->built) return SKIM_ENOTBUILT;
    if (v >= c->n) return SKIM_EINVAL;
    uint32_t len = 0;
    CK(c, cudaMemcpyAsync(&len, c->xlen + v, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    if (len > c->k) return fail_cuda(c, cudaErrorIllegalState);
    if (len)
        CK(c, cudaMemcpyAsync(out_k, c->X + static_cast<size_t>(v) * c->k, len * sizeof(uint64_t),
                              cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    *out_len = len;
    return SKIM_OK;
}

int skim_set_wait_limit_ns(skim_ctx *c, uint64_t ns) {
    if (!c || ns == 0) return SKIM_EINVAL;
    c->timeout_ns = ns;
    return SKIM_OK;
}

int skim_set_live_rows(skim_ctx *c, int on) {
    if (!c) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (c->batch_active) {
        RC(commit_lanes(c, c->blo, c->bB - 1));
        RC(clear_batch(c));
        c->batch_active = false;
    }
    c->mat_wanted = on != 0;
    // live rows exist only when they were generated (not for the IC model or
    // 2^31 or more live pairs); turning them on again needs nothing else
    c->mat = c->mat_wanted && c->live_ready;
    c->sk_init = false;
    return SKIM_OK;
}

int skim_sketch_pointers(skim_ctx *c, const uint64_t **x_dev, const uint32_t **len_dev) {
    if (!c || !x_dev || !len_dev) return SKIM_EINVAL;
    if (!c->built) return SKIM_ENOTBUILT;
    *x_dev = c->X;
    *len_dev = c->xlen;
    return SKIM_OK;
}

int skim_greedy_reset(skim_ctx *c) {
    if (!c) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    return skim_state_init(c);
}

namespace {

// cov_out[j] is stored when seed j's residual search is finished: by the
// read-back of seed j+1's scan, or before the call returns.
int greedy_loop(skim_ctx *c, uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out) {
    int rc = SKIM_OK;
    for (uint32_t j = 0; j < n_seeds; j++) {
        uint32_t x = 0;
        c->rec_j = j;
        rc = next_seed(c, &x, cov_out + j);
        if (rc != SKIM_OK) break;
        seeds_out[j] = x;
        c->nseeds++;
    }
    if (rc == SKIM_OK) rc = settle_residual(c);
    // an error return with a search still pending came from a failed CUDA
    // call or wait, after which the context refuses further work
    c->pend_res = false;
    return rc;
}

}  // namespace

int skim_greedy_ex(skim_ctx *c, uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out, uint64_t *tau_out,
                   int32_t *kprime_out) {
    if (!c || (n_seeds && (!seeds_out || !cov_out))) return SKIM_EINVAL;
    if (c->batch_count) return SKIM_EINVAL;  // a batch of graphs has no single seed sequence
    if (c->rank_mode == SKIM_RANKS_IC_MODEL) return SKIM_EINVAL;  // IC-model SKIM is not built
    if (c->broken) return SKIM_ECUDA;
    if (!c->sk_init) RC(skim_state_init(c));
    if (static_cast<uint64_t>(c->nseeds) + n_seeds > c->n) return SKIM_EINVAL;
    RC(reset_stats(c));
    if ((tau_out || kprime_out) && n_seeds) {
        RC(dalloc(c, &c->rec_tau, n_seeds));
        int rc = dalloc(c, &c->rec_kp, n_seeds);
        if (rc == SKIM_OK) {
            CK(c, cudaMemsetAsync(c->rec_kp, 0, n_seeds * sizeof(uint32_t), c->st));
            rc = greedy_loop(c, n_seeds, seeds_out, cov_out);
        }
        if (rc == SKIM_OK) {
            std::vector<uint64_t> t(n_seeds);
            std::vector<uint32_t> kp(n_seeds);
            CK(c, cudaMemcpyAsync(t.data(), c->rec_tau, n_seeds * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->st));
            CK(c, cudaMemcpyAsync(kp.data(), c->rec_kp, n_seeds * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
            CK(c, cudaStreamSynchronize(c->st));
            for (uint32_t j = 0; j < n_seeds; j++) {
                if (tau_out) tau_out[j] = t[j];
                if (kprime_out) kprime_out[j] = static_cast<int32_t>(kp[j]);
            }
        }
        dfree(c, c->rec_tau);
        dfree(c, c->rec_kp);
        RC(rc);
    } else {
        RC(greedy_loop(c, n_seeds, seeds_out, cov_out));
    }
    uint64_t keep[3] = {c->hstats[SKIM_STAT_BATCHES], c->hstats[SKIM_STAT_RANKS], c->hstats[SKIM_STAT_RETRIES]};
    RC(pull_stats(c));
    c->hstats[SKIM_STAT_BATCHES] = keep[0];
    c->hstats[SKIM_STAT_RANKS] = keep[1];
    c->hstats[SKIM_STAT_RETRIES] = keep[2];
    return SKIM_OK;
}

int skim_greedy(skim_ctx *c, uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out) {
    return skim_greedy_ex(c, n_seeds, seeds_out, cov_out, nullptr, nullptr);
}

int skim_oracle_query_batch(skim_ctx *c, const uint64_t *offsets, uint32_t q, const uint32_t *seeds, double *est_out,
                            int on_device) {
    if (!c || !offsets || (q && !est_out)) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (!c->built) return SKIM_ENOTBUILT;
    if (q == 0) return SKIM_OK;
    if (offsets[0] != 0) return SKIM_EINVAL;
    // one host block: seed offsets | table offsets | chunk offsets
    const size_t q1 = static_cast<size_t>(q) + 1;
    std::vector<uint64_t> meta(3 * q1, 0);
    uint64_t *toff = meta.data() + q1, *coff = meta.data() + 2 * q1;
    for (uint32_t i = 0; i < q; i++) {
        if (offsets[i + 1] < offsets[i]) return SKIM_EINVAL;
        const uint64_t H = query_table(offsets[i + 1] - offsets[i], c->k);
        toff[i + 1] = toff[i] + H;
        coff[i + 1] = coff[i] + query_chunks(H);
    }
    std::copy(offsets, offsets + q1, meta.data());
    const uint64_t total = offsets[q];
    if (total && !seeds) return SKIM_EINVAL;
    if (!on_device) {
        for (uint64_t i = 0; i < total; i++)
            if (seeds[i] >= c->n) return SKIM_EINVAL;
    }
    RC(ensure_query_space(c, total, q, toff[q], coff[q]));
    const uint32_t *dseeds = seeds;
    if (!on_device && total) {
        CK(c, cudaMemcpyAsync(c->qseeds, seeds, total * sizeof(uint32_t), cudaMemcpyHostToDevice, c->st));
        dseeds = c->qseeds;
    }
    uint64_t *d_off = c->qoff, *d_toff = c->qoff + q1, *d_coff = c->qoff + 2 * q1;
    CK(c, cudaMemcpyAsync(d_off, meta.data(), meta.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, c->st));
    CK(c, cudaMemsetAsync(c->dflag, 0, sizeof(unsigned), c->st));
    double *dout = on_device ? est_out : c->qout;
    {
        KTimer kt(c, SKIM_K_QUERY);
        QueryScratch qs{c->qk, c->qv, c->qtop, c->qtopu, c->qpart, c->dflag};
        CK(c, launch_query_multi(c->X, c->xlen, c->n, c->k, query_terms_of(c), dseeds, d_off, d_toff, d_coff, q, toff[q], total,
                                 static_cast<uint32_t>(coff[q]), qs, dout, c->st));
    }
    unsigned bad = 0;
    CK(c, cudaMemcpyAsync(&bad, c->dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    if (!on_device)
        CK(c, cudaMemcpyAsync(est_out, c->qout, q * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(c, cudaStreamSynchronize(c->st));
    resolve_timers(c);
    return bad ? SKIM_EINVAL : SKIM_OK;
}

int skim_oracle_query(skim_ctx *c, const uint32_t *seeds, uint32_t n_seeds, double *est_out) {
    if (!c || !est_out || (n_seeds && !seeds)) return SKIM_EINVAL;
    uint64_t off[2] = {0, n_seeds};
    return skim_oracle_query_batch(c, off, 1, seeds, est_out, 0);
}

int skim_kernel_launches(uint64_t *out) {
    if (!out) return SKIM_EINVAL;
    *out = g_kernel_launches.load();
    return SKIM_OK;
}

int skim_node_estimates(skim_ctx *c, double *out, int out_on_device) {
    if (!c || !out) return SKIM_EINVAL;
    if (c->broken) return SKIM_ECUDA;
    if (!c->built) return SKIM_ENOTBUILT;
    double *d = out;
    if (!out_on_device) RC(dalloc(c, &d, c->n));
    int rc = SKIM_OK;
    if (launch_node_estimates(c->X, c->xlen, c->n, c->k, c->l, c->rank_mode, d, c->st) != cudaSuccess ||
        (!out_on_device &&
         cudaMemcpyAsync(out, d, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->st) != cudaSuccess) ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
        rc = fail_cuda(c, cudaGetLastError());
    if (!out_on_device) dfree(c, d);
    return rc;
}

int skim_set_timing(skim_ctx *c, int on) {
    if (!c) return SKIM_EINVAL;
    c->timing = on != 0;
    // create the events up front: creating them inside a timed bracket would
    // leave the GPU waiting on the host there
    const size_t want = 2048;
    while (c->timing && c->kpool.size() + c->kpend.size() * 2 < want) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda(c, cudaGetLastError());
        c->kpool.push_back(e);
    }
    return SKIM_OK;
}

int skim_kernel_times(skim_ctx *c, double *ms_out, uint64_t *launches_out, uint32_t count, int reset) {
    if (!c) return SKIM_EINVAL;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return fail_cuda(c, cudaGetLastError());
    resolve_timers(c);
    for (uint32_t i = 0; i < count && i < SKIM_K_COUNT; i++) {
        if (ms_out) ms_out[i] = c->kms[i];
        if (launches_out) launches_out[i] = c->klaunch[i];
    }
    if (reset) {
        std::fill(c->kms, c->kms + SKIM_K_COUNT, 0.0);
        std::fill(c->klaunch, c->klaunch + SKIM_K_COUNT, 0);
    }
    return SKIM_OK;
}

int skim_context_shape(skim_ctx *c, uint32_t *n, uint32_t *k, uint32_t *l) {
    if (!c || !n || !k || !l) return SKIM_EINVAL;
    *n = c->n;
    *k = c->k;
    *l = c->l;
    return SKIM_OK;
}

int skim_get_stats(skim_ctx *c, uint64_t *out, uint32_t count) {
    if (!c || !out) return SKIM_EINVAL;
    for (uint32_t i = 0; i < count && i < SKIM_STAT_COUNT; i++) out[i] = c->hstats[i];
    return SKIM_OK;
}

}  // extern "C"

// traverse.cu -- asynchronous, worklist-driven graph searches.
//
// Reverse searches (Algorithm 2 sketch building, Section 5.2; Algorithm 1
// sketch building, Section 4): a batch of B consecutive ranks is searched at
// once.  Lane j of the batch is the j-th rank; lanes are packed 64 to a word
// and a visit is a (node, word, lane mask) triple.  Every (node, lane) pair is
// expanded at most once: a lane bit enters a node through an atomicOr on the
// node's visited word, and only newly set bits are pushed.  The live-edge coin
// of a lane is drawn in that lane's instance (Section 2, binary IC model).
// Algorithm 2's pruning -- skip a node whose local sketch of the lane's
// instance already holds k ranks -- is tested against the state at the start
// of the batch, which keeps the result exact (see the acceptance step).
//
// Residual searches (Algorithm 1, "Residual problem"): a forward search from
// the new seed with lanes = instances, pruned at covered pairs; each newly
// covered pair with an index entry queues the decrements of the sizes listed
// in that entry (the entry is erased).
//
// There are no BFS levels: warps claim items from one global queue, process
// them, and push new items; the search ends when every pushed item is done.
// Reverse searches of small batches use per-warp queues instead (k_rev_ring),
// and residual searches keep a few items per block in shared memory (FwdRing).
// Every wait is bounded by a timeout that sets an error flag.
#include <type_traits>

#include "internal.cuh"

namespace skim {

namespace {

constexpr int kTravThreads = 256;
constexpr int kMaxProbe = 512;  // the table is sized to a load of about 1/4: longer chains mean it is full

// Live threshold of CSR edge idx = (u -> v); tm1_head is the item's value
// for the models whose threshold depends on the head node only.
SKIM_DEV uint64_t edge_tm1_rev(const TravArgs &A, uint32_t idx, uint32_t u, uint32_t v, uint64_t tm1_head) {
    const CoinModel &cm = A.cm;
    if (cm.model == 3) return A.tm1e[idx];
    if (cm.model == 2) return cm.tm1_class[fmix(cm.prob_key ^ ((static_cast<uint64_t>(u) << 32) | v)) % 3u];
    return tm1_head;
}

SKIM_DEV uint64_t edge_tm1_fwd(const TravArgs &A, uint32_t idx, uint32_t u, uint32_t w) {
    const CoinModel &cm = A.cm;
    if (cm.model == 3) return A.tm1e[idx];
    if (cm.model == 0) return cm.tm1_uniform;
    if (cm.model == 1) return cm.thr_wc[w];
    return cm.tm1_class[fmix(cm.prob_key ^ ((static_cast<uint64_t>(u) << 32) | w)) % 3u];
}

// 16-byte compare-and-swap of a table slot {key, bits}: true if the slot held
// {ek, eb}; *ok, *ob = what it held.
SKIM_DEV bool cas_slot(uint64_t *slot, uint64_t ek, uint64_t eb, uint64_t nk, uint64_t nb, uint64_t *ok,
                       uint64_t *ob) {
    uint64_t lo, hi;
    asm volatile(
        "{\n\t.reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%2, %3};\n\t"
        "mov.b128 c, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(lo), "=l"(hi)
        : "l"(ek), "l"(eb), "l"(nk), "l"(nb), "l"(slot)
        : "memory");
    *ok = lo;
    *ob = hi;
    return lo == ek && hi == eb;
}

// Insert-or-merge of (key, bits) into the visited table.  Returns false if the
// probe limit is hit.  *old = bits present before, *slot = table slot,
// *first = this call created the entry.  Slot h keeps key + 1 at hkeys[2h] and
// its bits at hvals[2h] (hvals = hkeys + 1): both in one 16-byte sector.  The
// batch's part of the table is zeroed before the batch (0 = empty).  The
// caller has loaded the first slot (h, k, b): an empty slot is claimed by a
// 16-byte compare-and-swap that writes key and bits together (so no other lane
// can OR bits into a half-written entry); a slot with this key gets the bits
// ORed in (nothing to do when they are there already); another key moves the
// probe on.  Every pass (a lost CAS, a step) counts against the probe limit.
SKIM_DEV bool hash_or_from(uint64_t *hkeys, uint64_t *hvals, uint64_t hmask, uint64_t key, uint64_t bits,
                           uint64_t h, uint64_t k, uint64_t b, uint64_t *old, uint64_t *slot, bool *first) {
    const uint64_t stored = key + 1;
    for (int p = 0; p < kMaxProbe; p++) {
        if (k == 0) {
            uint64_t ok, ob;
            if (cas_slot(&hkeys[2 * h], 0, 0, stored, bits, &ok, &ob)) {
                *first = true;
                *slot = h;
                *old = 0;
                return true;
            }
            k = ok;  // someone else claimed it first: look at what it holds now
            b = ob;
            continue;
        }
        if (k == stored) {
            *first = false;
            *slot = h;
            *old = (b & bits) == bits ? b : atomicOr(reinterpret_cast<unsigned long long *>(&hvals[2 * h]), bits);
            return true;
        }
        h = (h + 1) & hmask;
        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(k), "=l"(b) : "l"(&hkeys[2 * h]) : "memory");
    }
    return false;
}

// First visited-table slot of entry key = u << tbits | t.  With hnode set
// (batches of few words) the entries of one node for different words lie
// side by side, so that the lanes of a batch that reach the same node touch
// one or two cache lines of the table rather than one each; a batch of many
// words hashes the whole key (a hub's entries would otherwise form long runs
// that other keys must probe across).
SKIM_DEV uint64_t table_slot(uint64_t key, uint32_t tbits, uint32_t hnode, uint64_t hmask) {
    if (hnode) return (fmix(key >> tbits) + (key & ((1ull << tbits) - 1))) & hmask;
    return fmix(key) & hmask;
}

SKIM_DEV void load_slot(const uint64_t *hkeys, uint64_t h, uint64_t *k, uint64_t *b) {
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(*k), "=l"(*b) : "l"(&hkeys[2 * h]) : "memory");
}

SKIM_DEV bool hash_or(uint64_t *hkeys, uint64_t *hvals, uint64_t hmask, uint32_t tbits, uint32_t hnode, uint64_t key,
                      uint64_t bits, uint64_t *old, uint64_t *slot, bool *first) {
    const uint64_t h = table_slot(key, tbits, hnode, hmask);
    uint64_t k, b;
    load_slot(hkeys, h, &k, &b);
    return hash_or_from(hkeys, hvals, hmask, key, bits, h, k, b, old, slot, first);
}

SKIM_DEV uint32_t n_chunks(uint32_t deg) { return (deg + kChunk - 1) / kChunk; }
SKIM_DEV uint32_t n_chunks(uint32_t deg, uint64_t mask) {
    const uint32_t ce = chunk_edges(deg, mask);
    return (deg + ce - 1) / ce;
}

// Per-lane counters, added to DevCtl once when a warp finishes.  `pushed`
// records that the lane reserved queue slots since the warp last reported
// items done.
struct Acc {
    unsigned long long visits = 0, coins = 0, cov = 0, edges = 0;
    bool pushed = false;
};

SKIM_DEV void flush_acc(const TravArgs &A, const Acc &acc, bool fwd) {
    warp_add(&A.ctl->stats[fwd ? kStFwdVisits : kStRevVisits], acc.visits);
    warp_add(&A.ctl->stats[fwd ? kStFwdCoins : kStRevCoins], acc.coins);
    if (fwd) warp_add(&A.ctl->ix_cov, acc.cov);
    warp_add(&A.ctl->stats[fwd ? kStFwdEdges : kStRevEdges], acc.edges);
}

// Reserve `cnt` queue slots per lane (warp-aggregated); returns the lane's
// first slot.  Slots at or beyond capacity never receive an item: they are
// counted as done at once, and the caller parks that work in a pending mask.
SKIM_DEV unsigned long long reserve_slots(const TravArgs &A, Acc &acc, uint32_t cnt) {
    if (cnt) acc.pushed = true;
    unsigned long long tot;
    unsigned long long ex = warp_excl_scan(cnt, &tot);
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0 && tot) base = atomicAdd(&A.ctl->q_tail.v, tot);
    base = __shfl_sync(kFull, base, 0);
    if ((threadIdx.x & 31) == 0 && tot && base + tot > A.qcap) {
        unsigned long long lost = base + tot - (base >= A.qcap ? base : A.qcap);
        atomicAdd(&A.ctl->q_done.v, lost);
    }
    return base + ex;
}

SKIM_DEV void write_item(const TravArgs &A, unsigned long long slot, uint32_t v, uint32_t w, uint64_t mask) {
    if (slot >= A.qcap) return;
    const uint64_t lo = (static_cast<uint64_t>(w + 1) << 32) | (v + 1);
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(&A.q[slot]), "l"(lo), "l"(mask) : "memory");
}

// Reads a slot; true once all of its fields have arrived.
SKIM_DEV bool read_item(const TravArgs &A, unsigned long long slot, Item *it) {
    uint64_t lo, m;
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(m) : "l"(&A.q[slot]) : "memory");
    const uint32_t v1 = static_cast<uint32_t>(lo), w1 = static_cast<uint32_t>(lo >> 32);
    if (v1 == 0 || w1 == 0 || m == 0) return false;
    it->v = v1 - 1;
    it->w = w1 - 1;
    it->mask = m;
    return true;
}

// A lane whose reservation does not fit fills its in-capacity slots with
// placeholders; returns true if the lane must park its work.
SKIM_DEV bool spill_if_full(const TravArgs &A, unsigned long long s, uint32_t ni) {
    if (s + ni <= A.qcap) return false;
    for (uint32_t c = 0; c < ni; c++) write_item(A, s + c, 0, kNopTag, 1);
    atomicOr(&A.ctl->spill, 1u);
    return true;
}

// ---- Block-local work ring of the residual searches ----
//
// A residual search starts at one seed and, on sparse live graphs, is a long
// and mostly narrow walk (tens of hops deep per instance), so its time is its
// depth times the latency of one hop.  Through the global queue a hop is a
// slot reservation, the item's write, a poll that finds it and its read, on
// top of the row read and the covering OR.  So a block of the search over
// materialised rows keeps up to kFwdKeep items in a ring in shared memory,
// taken by its own warps; the items that do not fit go to the global queue,
// which spreads a wide frontier over the grid.
//
// The ring is a bounded multi-producer multi-consumer queue: positions are
// handed out by compare-and-swap on `tail` (reserved) and `head` (taken), and
// slot i's sequence number says whether it is free for position p (seq = p)
// or holds the item of position p (seq = p + 1).
//
// The search still ends by the global queue's drain test (done == tail).
// While a ring holds unfinished items its block holds one reserved queue slot,
// the token, which is written with a placeholder only after the last of them
// is finished; whoever claims the slot counts it as done.  The token is
// reserved before the items it covers are pushed, and the items' own pushes
// are counted before they are finished, so the drain test cannot pass while a
// ring holds work.  A token outlives its ring's work until a warp of the block
// has found nothing to do for kFwdParkNs (the next items pushed to the ring
// reuse it, without a reservation on the queue); a warp that leaves releases
// it.  `state` packs the token with the count of unfinished items so that
// both change together.
#ifndef SKIM_FWD_KEEP
#define SKIM_FWD_KEEP 8
#endif
constexpr uint32_t kFwdKeep = SKIM_FWD_KEEP;  // items a block's ring may hold (0: no ring)
#ifndef SKIM_FWD_PARK_NS
#define SKIM_FWD_PARK_NS 2000
#endif
constexpr uint64_t kFwdParkNs = SKIM_FWD_PARK_NS;  // idle time after which a warp frees its block's token
constexpr unsigned long long kNoTok = 0xffffffffull;  // token field: none held
constexpr uint32_t kFwdCap = kFwdKeep <= 64 ? 64 : 512;  // ring slots (a power of two, at least kFwdKeep)
static_assert(kFwdKeep <= kFwdCap, "ring size");

struct FwdRing {
    ulonglong2 it[kFwdCap];    // .x = (w + 1) << 32 | (v + 1), .y = mask
    unsigned seq[kFwdCap];
    unsigned head, tail;
    unsigned long long state;  // token slot (kNoTok: none) << 32 | unfinished items
};

SKIM_DEV unsigned ld_vol(const unsigned *p) { return *reinterpret_cast<const volatile unsigned *>(p); }
SKIM_DEV void st_ring_item(ulonglong2 *p, uint64_t x, uint64_t y) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("st.volatile.shared.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(x), "l"(y) : "memory");
}
SKIM_DEV void ld_ring_item(const ulonglong2 *p, uint64_t *x, uint64_t *y) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
    asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];" : "=l"(*x), "=l"(*y) : "r"(a) : "memory");
}

SKIM_DEV void ring_init(FwdRing *R) {
    for (uint32_t i = threadIdx.x; i < kFwdCap; i += blockDim.x) R->seq[i] = i;
    if (threadIdx.x == 0) {
        R->head = R->tail = 0;
        R->state = kNoTok << 32;
    }
}

// Spin until *p == want; false (and the error flag) when the wait limit runs out.
SKIM_DEV bool ring_wait(const TravArgs &A, const unsigned *p, unsigned want) {
    if (ld_vol(p) == want) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned k = 1;; k++) {
        if (ld_vol(p) == want) return true;
        if ((k & 63) == 0 && globaltimer() - t0 > A.timeout_ns) {
            atomicOr(&A.ctl->err, kErrTimeout);
            return false;
        }
    }
}

// Lane 0: free the block's token if its ring has no unfinished items (a
// placeholder into its queue slot).
SKIM_DEV void ring_release(const TravArgs &A, FwdRing *R) {
    const unsigned long long s = *reinterpret_cast<volatile unsigned long long *>(&R->state);
    if ((s & 0xffffffffull) != 0 || (s >> 32) == kNoTok) return;
    if (atomicCAS(&R->state, s, kNoTok << 32) != s) return;
    __threadfence();  // the reservations of the finished items' own pushes come first
    write_item(A, s >> 32, 0, kNopTag, 1);
}

// Lane 0 finishes k of the ring's items.
SKIM_DEV void ring_finish(const TravArgs &A, FwdRing *R, unsigned k) {
    atomicAdd(&R->state, 0ull - k);
    if (kFwdParkNs == 0) ring_release(A, R);
}

// Lane 0 counts tot new ring items; the first of an empty ring takes a token
// unless the block still holds one.  False when no token can be had (the
// global queue is full).
SKIM_DEV bool ring_count(const TravArgs &A, FwdRing *R, unsigned long long tot) {
    unsigned long long s = *reinterpret_cast<volatile unsigned long long *>(&R->state), tok = kNoTok;
    for (int k = 0;; k++) {
        if (k == 4096) {  // contended for too long: the items go to the queue
            if (tok != kNoTok) write_item(A, tok, 0, kNopTag, 1);
            return false;
        }
        unsigned long long ns;
        const bool fresh = (s >> 32) == kNoTok;
        if (fresh) {
            if (tok == kNoTok) {
                tok = atomicAdd(&A.ctl->q_tail.v, 1ull);
                if (tok >= A.qcap) {  // beyond the queue: counted as done at once
                    atomicAdd(&A.ctl->q_done.v, 1ull);
                    return false;
                }
            }
            ns = (tok << 32) | tot;
        } else {
            ns = s + tot;
        }
        const unsigned long long o = atomicCAS(&R->state, s, ns);
        if (o == s) {
            if (!fresh && tok != kNoTok) write_item(A, tok, 0, kNopTag, 1);  // a token not needed after all
            return true;
        }
        s = o;
    }
}

// Warp-collective: tot ring positions for the warp's new items, all or none;
// *base = the first.
SKIM_DEV bool ring_reserve(const TravArgs &A, FwdRing *R, unsigned long long tot, unsigned *base) {
    int ok = 0;
    unsigned b = 0;
    if ((threadIdx.x & 31) == 0 && tot && tot <= kFwdKeep &&
        ld_vol(&R->tail) - ld_vol(&R->head) + tot <= kFwdKeep && ring_count(A, R, tot)) {
        unsigned t = ld_vol(&R->tail);
        for (int k = 0; k < 16; k++) {
            if (t - ld_vol(&R->head) + tot > kFwdKeep) break;
            const unsigned o = atomicCAS(&R->tail, t, t + static_cast<unsigned>(tot));
            if (o == t) {
                ok = 1;
                b = t;
                break;
            }
            t = o;
        }
        if (!ok) ring_finish(A, R, static_cast<unsigned>(tot));  // no room after all: uncount
    }
    *base = __shfl_sync(kFull, b, 0);
    return __shfl_sync(kFull, ok, 0) != 0;
}

// Write the item of ring position pos once its slot is free.
SKIM_DEV void ring_put(const TravArgs &A, FwdRing *R, unsigned pos, uint32_t v, uint32_t w, uint64_t mask) {
    const unsigned i = pos & (kFwdCap - 1);
    if (!ring_wait(A, &R->seq[i], pos)) return;
    const uint64_t lo = (static_cast<uint64_t>(w + 1) << 32) | (v + 1);
    st_ring_item(&R->it[i], lo, mask);
    __threadfence_block();
    *reinterpret_cast<volatile unsigned *>(&R->seq[i]) = pos + 1;
}

// Warp-collective: the lanes of `freel` take ring items, one each, as many as
// there are; returns the lanes that took one (an item lost to the wait limit
// is taken empty).
SKIM_DEV unsigned ring_take(const TravArgs &A, FwdRing *R, unsigned freel, bool &have, Item &it) {
    const int lane = threadIdx.x & 31;
    unsigned n = 0, b = 0;
    if (lane == 0) {
        unsigned h = ld_vol(&R->head);
        const unsigned want = __popc(freel);
        for (int k = 0; k < 16; k++) {
            const unsigned avail = ld_vol(&R->tail) - h;
            const unsigned m = avail < want ? avail : want;
            if (!m) break;
            const unsigned o = atomicCAS(&R->head, h, h + m);
            if (o == h) {
                n = m;
                b = h;
                break;
            }
            h = o;
        }
    }
    n = __shfl_sync(kFull, n, 0);
    if (!n) return 0;
    b = __shfl_sync(kFull, b, 0);
    const unsigned r = __popc(freel & lanemask_lt());
    const bool mine = ((freel >> lane) & 1u) && r < n;
    if (mine) {
        const unsigned pos = b + r, i = pos & (kFwdCap - 1);
        if (ring_wait(A, &R->seq[i], pos + 1)) {
            uint64_t x = 0, y = 0;
            ld_ring_item(&R->it[i], &x, &y);
            __threadfence_block();
            *reinterpret_cast<volatile unsigned *>(&R->seq[i]) = pos + kFwdCap;
            it.v = static_cast<uint32_t>(x) - 1;
            it.w = static_cast<uint32_t>(x >> 32) - 1;
            it.mask = y;
            have = true;
        }
    }
    return __ballot_sync(kFull, mine);
}

// Live in-neighbour row of (u, lane j of word t) in the materialised instances.
SKIM_DEV uint32_t live_row_len(const TravArgs &A, uint32_t u, uint32_t t, int j) {
    const uint64_t r = static_cast<uint64_t>(u) * A.l + A.lane_inst[static_cast<size_t>(t) * 64 + j];
    return (A.loff[r + 1] & kRowMask) - (A.loff[r] & kRowMask);
}

// A materialised reverse item names its row directly: v = first entry of the
// chunk, w = (instance << 25 | word << 6 | lane bit), mask = entries in the
// chunk (1..kChunk), so that the consumer needs no lookup before it reads the
// row.  Residual items carry word 0 and the instance as the lane bit.
SKIM_DEV uint32_t row_item_w(uint32_t t, int j, uint32_t inst) {
    return (inst << kInstShift) | (t << 6) | static_cast<uint32_t>(j);
}
SKIM_DEV void write_row_items(const TravArgs &A, unsigned long long s, uint64_t b0, uint64_t b1, uint32_t t, int j,
                              uint32_t inst) {
    for (uint64_t e = b0, q = 0; e < b1; e += kChunk, q++)
        write_item(A, s + q, static_cast<uint32_t>(e), row_item_w(t, j, inst),
                   b1 - e < kChunk ? b1 - e : static_cast<uint64_t>(kChunk));
}

// Warp-collective: queue the expansion of lane bits `nb` of entry (u, t)
// (table slot `slot`).  With materialised instances each lane gets items of
// its own (its row of live in-neighbours; none if the row is empty).
template <bool MAT>
SKIM_DEV void push_rev(const TravArgs &A, Acc &acc, uint32_t u, uint32_t t, uint64_t nb, uint64_t slot) {
    uint32_t ni = 0;
    if (MAT) {
        for (uint64_t m = nb; m; m &= m - 1) ni += n_chunks(live_row_len(A, u, t, __ffsll(m) - 1));
    } else if (nb) {
        ni = n_chunks(A.ptr[u + 1] - A.ptr[u], nb);
    }
    if (!__any_sync(kFull, ni != 0)) return;
    unsigned long long s = reserve_slots(A, acc, ni);
    if (ni && spill_if_full(A, s, ni)) {
        atomicOr(reinterpret_cast<unsigned long long *>(&A.pend[slot]), nb);
        return;
    }
    if (MAT) {
        uint32_t c = 0;
        for (uint64_t m = nb; m; m &= m - 1) {
            const int j = __ffsll(m) - 1;
            const uint32_t inst = A.lane_inst[static_cast<size_t>(t) * 64 + j];
            const uint64_t r = static_cast<uint64_t>(u) * A.l + inst;
            const uint64_t b0 = A.loff[r] & kRowMask, b1 = A.loff[r + 1] & kRowMask;
            write_row_items(A, s + c, b0, b1, t, j, inst);
            c += n_chunks(static_cast<uint32_t>(b1 - b0));
        }
    } else {
        for (uint32_t c = 0; c < ni; c++) write_item(A, s + c, u, (t << kChunkBits) | c, nb);
    }
}

// Warp-collective: lanes with `act` visit node u with lane bits `bits` in word t.
template <bool MAT>
SKIM_DEV void emit_rev(const TravArgs &A, Acc &acc, bool act, uint32_t u, uint32_t t, uint64_t bits) {
    if (!__any_sync(kFull, act && bits)) return;
    uint64_t nb = 0;
    bool first = false;
    uint64_t slot = 0;
    if (act && bits) {
        uint64_t old;
        uint64_t key = (static_cast<uint64_t>(u) << A.tbits) | t;
        if (hash_or(A.hkeys, A.hvals, A.hmask, A.tbits, A.hnode, key, bits, &old, &slot, &first)) {
            nb = bits & ~old;
        } else {
            atomicOr(&A.ctl->err, kErrHash);
        }
    }
    // record of the (node, word) entry, written once by its creator
    {
        unsigned ball = __ballot_sync(kFull, first);
        if (ball) {
            unsigned long long base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(&A.ctl->rec_count.v, static_cast<unsigned long long>(__popc(ball)));
            base = __shfl_sync(kFull, base, 0);
            if (first) {
                unsigned long long r = base + __popc(ball & lanemask_lt());
                if (r < A.rcap) {
                    A.rec_key[r] = (static_cast<uint64_t>(u) << A.tbits) | t;
                    A.rec_val[r] = static_cast<uint32_t>(slot);
                } else {
                    atomicOr(&A.ctl->err, kErrRecords);
                }
            }
        }
    }
    acc.visits += __popcll(nb);
    push_rev<MAT>(A, acc, u, t, nb, slot);
}

// Where a reverse search puts what it finds.  GlobalSink: visit records by
// one atomic per warp step, row items into the global queue.  RingSink (the
// per-warp-queue search below): records staged in shared memory, row items
// into the warp's own ring, the global queue only when the ring is full.
struct GlobalSink {
    // Warp-collective: lanes with `first` created table entry (key, slot).
    SKIM_DEV void record(const TravArgs &A, bool first, uint64_t key, uint64_t slot) {
        const unsigned ball = __ballot_sync(kFull, first);
        if (!ball) return;
        unsigned long long base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(&A.ctl->rec_count.v, static_cast<unsigned long long>(__popc(ball)));
        base = __shfl_sync(kFull, base, 0);
        if (first) {
            const unsigned long long r = base + __popc(ball & lanemask_lt());
            if (r < A.rcap) {
                A.rec_key[r] = key;
                A.rec_val[r] = static_cast<uint32_t>(slot);
            } else {
                atomicOr(&A.ctl->err, kErrRecords);
            }
        }
    }
    // Warp-collective: lanes with ni > 0 queue the ni chunks of row [b0, b1)
    // for lane j of word t (instance inst); a full queue parks the lane bit.
    SKIM_DEV void rows(const TravArgs &A, Acc &acc, uint32_t ni, uint64_t b0, uint64_t b1, uint32_t t, int j,
                       uint32_t inst, uint64_t slot) {
        if (!__any_sync(kFull, ni != 0)) return;
        const unsigned long long s = reserve_slots(A, acc, ni);
        if (ni && spill_if_full(A, s, ni)) {
            atomicOr(reinterpret_cast<unsigned long long *>(&A.pend[slot]), 1ull << j);
            return;
        }
        if (ni) write_row_items(A, s, b0, b1, t, j, inst);
    }
};

// Where a residual search puts its new items: the block's ring (null: none)
// while it has room, else the global queue.
struct FwdSink {
    FwdRing *ring;
};

// Warp-collective, materialised reverse searches: lanes with `act` reach node
// u for lane j of word t (instance inst).  The row bounds of (u, inst) and the
// pruning word are loaded together, before the visited-table update.
template <class SK>
SKIM_DEV void emit_rev_mat(const TravArgs &A, Acc &acc, SK &sk, bool act, uint32_t u, uint32_t t, int j,
                           uint32_t inst) {
    if (!__any_sync(kFull, act)) return;
    const uint64_t key = (static_cast<uint64_t>(u) << A.tbits) | t;
    uint64_t b0 = 0, b1 = 0, h0 = 0, k0 = 0, v0 = 0;
    if (act) {
        // the first visited-table slot, and the row of (u, inst) with
        // Algorithm 2's pruning flag: independent loads, in flight together
        h0 = table_slot(key, A.tbits, A.hnode, A.hmask);
        load_slot(A.hkeys, h0, &k0, &v0);
        const uint64_t r = static_cast<uint64_t>(u) * A.l + inst;
        const uint32_t w0 = A.loff[r], w1 = A.loff[r + 1];
        b0 = w0 & kRowMask;
        b1 = w1 & kRowMask;
        if (A.prune && (w0 & kRowFull)) act = false;  // Algorithm 2: local sketch full
    }
    const uint64_t bit = 1ull << j;
    bool fresh = false, first = false;
    uint64_t slot = 0;
    if (act) {
        uint64_t old;
        if (hash_or_from(A.hkeys, A.hvals, A.hmask, key, bit, h0, k0, v0, &old, &slot, &first))
            fresh = !(old & bit);
        else
            atomicOr(&A.ctl->err, kErrHash);
    }
    sk.record(A, first, key, slot);
    acc.visits += fresh ? 1 : 0;
    const uint32_t ni = fresh ? n_chunks(static_cast<uint32_t>(b1 - b0)) : 0;
    sk.rows(A, acc, ni, b0, b1, t, j, inst, slot);
}

// Row bounds, index length and index start of one pair (w, i), loaded ahead
// of time by a residual search whose item carries the single instance i.
struct PairPre {
    bool ok = false;
    uint64_t b0 = 0, b1 = 0, st = 0;
    uint32_t sl = 0;
};

// Warp-collective: queue the expansion of node w in instances `trav` and the
// erasure of the index entries of pairs (w, i), i in `erase`.  With
// materialised instances each instance gets row items of its own list of live
// out-neighbours (none if it is empty).  pre.ok: trav and erase hold at most
// the bit of pre's instance, whose values are taken from pre.  With a ring,
// the warp's new items go to the ring when they all fit.
template <bool MAT>
SKIM_DEV void push_fwd(const TravArgs &A, Acc &acc, uint32_t w, uint64_t trav, uint64_t erase, const PairPre &pre,
                       FwdRing *ring = nullptr) {
    uint32_t ni = 0;
    if (MAT) {
        for (uint64_t m = trav; m; m &= m - 1) {
            const uint64_t r = static_cast<uint64_t>(w) * A.l + (__ffsll(m) - 1);
            ni += n_chunks(static_cast<uint32_t>(pre.ok ? pre.b1 - pre.b0 : A.loff[r + 1] - A.loff[r]));
        }
    } else if (trav) {
        ni = n_chunks(A.ptr[w + 1] - A.ptr[w], trav);
    }
    for (uint64_t m = erase; m; m &= m - 1) {
        int i = __ffsll(m) - 1;
        ni += n_chunks(pre.ok ? pre.sl : A.seg_len[static_cast<uint64_t>(w) * A.l + i]);
    }
    if (!__any_sync(kFull, ni != 0)) return;
    unsigned long long s = 0;
    bool local = false;
    if (ring) {
        unsigned long long tot;
        const unsigned long long ex = warp_excl_scan(ni, &tot);
        unsigned base = 0;
        local = ring_reserve(A, ring, tot, &base);
        s = base + ex;
    }
    if (!local) {
        s = reserve_slots(A, acc, ni);
        if (ni && spill_if_full(A, s, ni)) {
            if (trav) atomicOr(reinterpret_cast<unsigned long long *>(&A.pend_trav[w]), trav);
            if (erase) atomicOr(reinterpret_cast<unsigned long long *>(&A.pend_erase[w]), erase);
            return;
        }
    }
    auto put = [&](unsigned long long q, uint32_t v, uint32_t iw, uint64_t m) {
        if (local)
            ring_put(A, ring, static_cast<unsigned>(q), v, iw, m);
        else
            write_item(A, q, v, iw, m);
    };
    uint32_t c = 0;
    if (MAT) {
        for (uint64_t m = trav; m; m &= m - 1) {
            const int i = __ffsll(m) - 1;
            const uint64_t r = static_cast<uint64_t>(w) * A.l + i;
            const uint64_t b0 = pre.ok ? pre.b0 : A.loff[r], b1 = pre.ok ? pre.b1 : A.loff[r + 1];
            for (uint64_t e = b0; e < b1; e += kChunk, c++)  // row items as write_row_items lays them out
                put(s + c, static_cast<uint32_t>(e), row_item_w(0, i, 0),
                    b1 - e < kChunk ? b1 - e : static_cast<uint64_t>(kChunk));
        }
    } else if (trav) {
        uint32_t nc = n_chunks(A.ptr[w + 1] - A.ptr[w], trav);
        for (; c < nc; c++) put(s + c, w, c, trav);
    }
    for (uint64_t m = erase; m; m &= m - 1) {
        int i = __ffsll(m) - 1;
        uint64_t pair = static_cast<uint64_t>(w) * A.l + i;
        uint32_t len = pre.ok ? pre.sl : A.seg_len[pair];
        if (!len) continue;
        A.seg_len[pair] = 0;  // erase index[w,i]
        uint64_t st = pre.ok ? pre.st : A.seg_start[pair];
        uint32_t ne = n_chunks(len);
        for (uint32_t e = 0; e < ne; e++, c++) put(s + c, len, kEraseTag | e, st + 1);
    }
}

// Warp-collective: lanes with `act` reach node w in the instances of `live`
// during a residual search.  A materialised item carries one instance: the
// pair's row bounds and index entries are requested together with the OR
// that covers it (an index is erased only by the lane whose OR newly covers
// its pair, so reading it first is safe).
template <bool MAT>
SKIM_DEV void emit_fwd(const TravArgs &A, Acc &acc, bool act, uint32_t w, uint64_t live, FwdRing *ring = nullptr) {
    if (!__any_sync(kFull, act && live)) return;
    uint64_t nb = 0;
    PairPre pre;
    if (act && live) {
        if (MAT && (live & (live - 1)) == 0) {
            const uint64_t r = static_cast<uint64_t>(w) * A.l + (__ffsll(live) - 1);
            pre.ok = true;
            pre.b0 = A.loff[r];
            pre.b1 = A.loff[r + 1];
            pre.sl = A.seg_len[r];
            pre.st = A.seg_start[r];
            const uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(&A.covered[w]), live);
            nb = live & ~old;
        } else {
            uint64_t cov = *reinterpret_cast<volatile uint64_t *>(&A.covered[w]);
            nb = live & ~cov;
            if (nb) {
                uint64_t old = atomicOr(reinterpret_cast<unsigned long long *>(&A.covered[w]), nb);
                nb &= ~old;
            }
        }
    }
    acc.cov += __popcll(nb);
    acc.visits += __popcll(nb);
    uint64_t erase = 0;
    for (uint64_t m = nb; m; m &= m - 1) {
        int i = __ffsll(m) - 1;
        if (pre.ok ? pre.sl : A.seg_len[static_cast<uint64_t>(w) * A.l + i]) erase |= 1ull << i;
    }
    push_fwd<MAT>(A, acc, w, nb, erase, pre, ring);
}

// Process the items held by the lanes with `have`, edges (or index entries)
// of all items flattened over the warp.
// Live lanes of an edge whose coin stream has state he: lane j is live iff
// fmix(he + g[j]) <= t1, g[j] = (instance of j + 1) * G.  Two coins per step
// so that the two hash chains overlap.
SKIM_DEV uint64_t live_lanes(uint64_t he, uint64_t m, uint64_t t1, const uint64_t *g) {
    uint64_t live = 0;
    while (m) {
        const int j1 = __ffsll(m) - 1;
        m &= m - 1;
        const uint64_t g1 = g[j1];
        if (m) {
            const int j2 = __ffsll(m) - 1;
            m &= m - 1;
            const uint64_t g2 = g[j2];
            const uint64_t c1 = fmix(he + g1), c2 = fmix(he + g2);
            live |= static_cast<uint64_t>(c1 <= t1) << j1;
            live |= static_cast<uint64_t>(c2 <= t1) << j2;
        } else {
            live |= static_cast<uint64_t>(fmix(he + g1) <= t1) << j1;
        }
    }
    return live;
}

// What one lane needs to expand its item.
struct Desc {
    uint32_t v, w, begin, cnt;
    uint64_t mask, tm1, g1;  // g1: stream offset when the item has a single lane
    bool erase, single;
    uint32_t inst;           // materialised reverse items: the lane's instance
};

template <bool FWD, bool MAT>
SKIM_DEV Desc describe(const TravArgs &A, bool have, const Item &it) {
    Desc d{};
    if (!have || it.w == kNopTag) return d;
    d.v = it.v;
    d.w = it.w;
    d.mask = it.mask;
    if (it.w & kEraseTag) {  // only residual searches create erase items
        d.erase = true;
        d.begin = (it.w & ~kEraseTag) * kChunk;
        d.cnt = min(kChunk, it.v - d.begin);
        return d;
    }
    const uint32_t chunk = it.w & ((1u << kChunkBits) - 1);
    if (MAT) {  // one lane (instance) and a chunk of its row (write_row_items)
        const uint32_t t = (it.w >> 6) & (kMaxWords - 1), j = it.w & 63u;
        d.begin = it.v;
        d.cnt = static_cast<uint32_t>(it.mask);
        d.mask = 1ull << j;
        d.w = t << kChunkBits;
        d.inst = FWD ? j : it.w >> kInstShift;
        return d;
    }
    const uint32_t e0 = A.ptr[it.v], e1 = A.ptr[it.v + 1];
    const uint32_t ce = chunk_edges(e1 - e0, it.mask);
    d.begin = e0 + chunk * ce;
    d.cnt = min(ce, e1 - d.begin);
    return d;
}

SKIM_DEV Desc shfl_desc(const Desc &d, int src) {
    Desc o;
    o.v = __shfl_sync(kFull, d.v, src);
    o.w = __shfl_sync(kFull, d.w, src);
    o.begin = __shfl_sync(kFull, d.begin, src);
    o.cnt = __shfl_sync(kFull, d.cnt, src);
    o.mask = __shfl_sync(kFull, d.mask, src);
    o.tm1 = __shfl_sync(kFull, d.tm1, src);
    o.g1 = __shfl_sync(kFull, d.g1, src);
    o.erase = __shfl_sync(kFull, d.erase, src);
    o.single = __shfl_sync(kFull, d.single, src);
    o.inst = __shfl_sync(kFull, d.inst, src);
    return o;
}

#ifndef SKIM_UNROLL
#define SKIM_UNROLL 1
#endif
#ifndef SKIM_TRAV_MIN_BLOCKS
#define SKIM_TRAV_MIN_BLOCKS 3
#endif
constexpr int kUnroll = SKIM_UNROLL;  // edges per lane per step: independent hash chains

// Coin test of CSR edge idx for item d: the lanes (reverse) or instances
// (forward) for which the edge is live; *tgt = the edge's other end.
#ifndef SKIM_HE_TABLE
#define SKIM_HE_TABLE 1
#endif
#ifndef SKIM_PREFETCH
#define SKIM_PREFETCH 1
#endif

// Per-edge value the live test needs: the coin-stream state of CSR edge idx
// (other end x), or with materialised instances its live mask (forward; the
// reverse live rows need nothing).
template <bool FWD, bool MAT>
SKIM_DEV uint64_t edge_key(const TravArgs &A, const Desc &d, uint32_t idx, uint32_t x) {
    if (MAT) return 0;  // materialised rows hold live edges only
#if SKIM_HE_TABLE
    return A.he[idx];
#else
    return FWD ? edge_state(A.cm.coin_key, d.v, x) : edge_state(A.cm.coin_key, x, d.v);
#endif
}

// Live lanes (reverse) or instances (forward) of an edge with other end x
// and coin-stream state he.
template <bool FWD, bool MAT>
SKIM_DEV uint64_t edge_live_xh(const TravArgs &A, const Desc &d, uint32_t idx, uint32_t x, uint64_t he,
                               const uint64_t *ginst) {
    if (MAT) return d.mask;
    if (FWD) return live_lanes(he, d.mask, edge_tm1_fwd(A, idx, d.v, x), ginst);
    const uint64_t t1 = edge_tm1_rev(A, idx, x, d.v, d.tm1);
    if (d.single) return fmix(he + d.g1) <= t1 ? d.mask : 0;
    return live_lanes(he, d.mask, t1, A.lane_g + static_cast<size_t>(d.w >> kChunkBits) * 64);
}

template <bool FWD, bool MAT>
SKIM_DEV uint64_t edge_live(const TravArgs &A, const Desc &d, uint32_t idx, uint32_t *tgt, const uint64_t *ginst) {
    const uint32_t x = A.col[idx];
    const uint64_t he = edge_key<FWD, MAT>(A, d, idx, x);
    *tgt = x;
    if (MAT) return d.mask;
    if (FWD) return live_lanes(he, d.mask, edge_tm1_fwd(A, idx, d.v, x), ginst);
    const uint64_t t1 = edge_tm1_rev(A, idx, x, d.v, d.tm1);
    if (d.single) return fmix(he + d.g1) <= t1 ? d.mask : 0;
    return live_lanes(he, d.mask, t1, A.lane_g + static_cast<size_t>(d.w >> kChunkBits) * 64);
}

// Algorithm 2: drop lanes whose instance-local sketch at u already holds k ranks.
SKIM_DEV uint64_t prune_full(const TravArgs &A, const Desc &d, uint32_t u, uint64_t live) {
    const uint64_t fu = A.full[u];
    if (!fu) return live;
    const uint8_t *li = A.lane_inst + static_cast<size_t>(d.w >> kChunkBits) * 64;
    for (uint64_t m = live; m; m &= m - 1) {
        const int j = __ffsll(m) - 1;
        if ((fu >> li[j]) & 1ull) live &= ~(1ull << j);
    }
    return live;
}

// Hand the live results of one step to the emitters (warp-collective).
template <bool FWD, bool MAT, class SK>
SKIM_DEV void emit_step(const TravArgs &A, Acc &acc, SK &sk, const Desc &d, const uint64_t *lv, const uint32_t *tg) {
#pragma unroll
    for (int q = 0; q < kUnroll; q++) {
        uint64_t live = lv[q];
        if constexpr (FWD) {
            emit_fwd<MAT>(A, acc, live != 0, tg[q], live, sk.ring);
        } else if constexpr (MAT) {
            emit_rev_mat(A, acc, sk, live != 0, tg[q], d.w >> kChunkBits, __ffsll(d.mask) - 1, d.inst);
        } else {
            if (live && A.prune) live = prune_full(A, d, tg[q], live);
            emit_rev<MAT>(A, acc, live != 0, tg[q], d.w >> kChunkBits, live);
        }
    }
}

// Expand entries [k0, k0 + kUnroll*stride) of item d, entry k at index
// begin + k for k < cnt (stride = 32 when the warp shares the item, 1 when
// the lane owns it).  Warp-collective.
template <bool FWD, bool MAT, class SK>
SKIM_DEV void expand_step(const TravArgs &A, Acc &acc, SK &sk, const Desc &d, uint32_t k0, uint32_t stride, bool own,
                          const uint64_t *ginst) {
    uint64_t lv[kUnroll];
    uint32_t tg[kUnroll];
#pragma unroll
    for (int q = 0; q < kUnroll; q++) {
        const uint32_t k = k0 + q * stride;
        lv[q] = 0;
        tg[q] = 0;
        if (own && k < d.cnt) {
            if (FWD && d.erase)
                atomicSub(&A.size[A.idx_nodes[(d.mask - 1) + d.begin + k]], 1u);
            else
                lv[q] = edge_live<FWD, MAT>(A, d, d.begin + k, &tg[q], ginst);
        }
    }
    uint64_t anyl = 0;
#pragma unroll
    for (int q = 0; q < kUnroll; q++) anyl |= lv[q];
    if (__any_sync(kFull, anyl != 0)) emit_step<FWD, MAT>(A, acc, sk, d, lv, tg);
}

// Expand the items held by the lanes with `have`: an item of 32 or more
// entries is swept by the whole warp (lane = entry), smaller items by their
// own lane.
template <bool FWD, bool MAT, class SK>
SKIM_DEV void process_items(const TravArgs &A, Acc &acc, SK &sk, bool have, const Item &it, const uint64_t *ginst) {
    const int lane = threadIdx.x & 31;
    Desc d = describe<FWD, MAT>(A, have, it);
    if (d.cnt && !d.erase) {
        acc.edges += d.cnt;
        if (!MAT) acc.coins += static_cast<unsigned long long>(d.cnt) * __popcll(d.mask);
        if (!FWD && !MAT) {
            d.tm1 = A.cm.model == 1 ? A.cm.thr_wc[d.v] : A.cm.tm1_uniform;
            d.single = (d.mask & (d.mask - 1)) == 0;
            if (d.single) d.g1 = A.lane_g[static_cast<size_t>(d.w >> kChunkBits) * 64 + (__ffsll(d.mask) - 1)];
        }
    }
    unsigned big = __ballot_sync(kFull, d.cnt >= 32);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const Desc b = shfl_desc(d, src);
#if SKIM_PREFETCH
        if (FWD && b.erase) {  // index-erase items
            for (uint32_t k0 = 0; k0 < b.cnt; k0 += 32 * kUnroll) expand_step<FWD, MAT>(A, acc, sk, b, k0 + lane, 32, true, ginst);
        } else {
            // one step ahead: the next edge's column and key are in flight
            // while the current coin is computed
            uint32_t x = 0;
            uint64_t h = 0;
            if (lane < b.cnt) {
                x = A.col[b.begin + lane];
                h = edge_key<FWD, MAT>(A, b, b.begin + lane, x);
            }
            for (uint32_t k0 = 0; k0 < b.cnt; k0 += 32) {
                const uint32_t k = k0 + lane;
                uint32_t xn = 0;
                uint64_t hn = 0;
                if (k + 32 < b.cnt) {
                    xn = A.col[b.begin + k + 32];
                    hn = edge_key<FWD, MAT>(A, b, b.begin + k + 32, xn);
                }
                uint64_t lv[kUnroll] = {0};
                uint32_t tg[kUnroll] = {0};
                if (k < b.cnt) {
                    lv[0] = edge_live_xh<FWD, MAT>(A, b, b.begin + k, x, h, ginst);
                    tg[0] = x;
                }
                if (__any_sync(kFull, lv[0] != 0)) emit_step<FWD, MAT>(A, acc, sk, b, lv, tg);
                x = xn;
                h = hn;
            }
        }
#else
        for (uint32_t k0 = 0; k0 < b.cnt; k0 += 32 * kUnroll) expand_step<FWD, MAT>(A, acc, sk, b, k0 + lane, 32, true, ginst);
#endif
    }
    const uint32_t mine = d.cnt < 32 ? d.cnt : 0;
    uint32_t steps = (mine + kUnroll - 1) / kUnroll;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) steps = max(steps, __shfl_xor_sync(kFull, steps, o));
    for (uint32_t st = 0; st < steps; st++) expand_step<FWD, MAT>(A, acc, sk, d, st * kUnroll, 1, mine != 0, ginst);
}

// ---- Reverse searches over materialised live rows, with per-warp queues ----
//
// The global queue (k_traverse, below) costs every item a 16-byte write and
// read in global memory and an atomic on a cursor that every warp shares.  Here each warp
// keeps the row items it creates in a ring of its own in shared memory and
// takes its next items from there, and stages its visit records in shared
// memory, writing them 32 or more at a time with one atomic.  The batch's
// first level (its source lanes) is claimed 32 lanes at a time by warps whose
// ring is empty.  A warp whose ring would overflow hands the step's items to
// the global queue instead; once the sources are used up a warp keeps at most
// kRingKeepTail items, so that idle warps share the last, long searches.  An
// idle warp claims global items only below the queue's reserved end (a slot
// there is written by a running warp right after its reservation), so no
// warp waits on a warp that is not running and the grid need not be resident
// all at once.  A warp leaves once no warp holds work (DevCtl::busy counts the
// warps that may) and neither the global queue nor the sources have any.
// Every wait is bounded as above; working warps advance DevCtl::beat now and
// then, so an idle warp counts a long search as progress.
#ifndef SKIM_RING_KEEP
#define SKIM_RING_KEEP 256
#endif
#ifndef SKIM_RING_KEEP_TAIL
#define SKIM_RING_KEEP_TAIL 64
#endif
#ifndef SKIM_RING_IDLE_NS
#define SKIM_RING_IDLE_NS 4096
#endif
constexpr uint32_t kRingCap = 256;                      // items per warp ring (a power of two)
constexpr uint32_t kRingKeep = SKIM_RING_KEEP;          // items a warp keeps while sources remain
constexpr uint32_t kRingKeepTail = SKIM_RING_KEEP_TAIL; // items a warp keeps once the sources are used up
constexpr uint32_t kRecStage = 64;                      // staged records per warp
constexpr int kRingThreads = 256;
constexpr unsigned kRingIdleMaxNs = SKIM_RING_IDLE_NS;  // longest sleep of an idle warp between polls
static_assert(kRingKeep <= kRingCap && kRingKeepTail <= kRingCap, "ring limits");

struct RingSink {
    Item *ring;
    uint64_t *rk;
    uint32_t *rs;
    uint32_t rh, rt, nrec, keep;  // warp-uniform: ring head and tail, staged records, ring limit

    // Warp-collective: write the staged records.
    SKIM_DEV void flush(const TravArgs &A) {
        __syncwarp();
        if (nrec == 0) return;
        const uint32_t lane = threadIdx.x & 31;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&A.ctl->rec_count.v, static_cast<unsigned long long>(nrec));
        base = __shfl_sync(kFull, base, 0);
        for (uint32_t q = lane; q < nrec; q += 32) {
            const unsigned long long r = base + q;
            if (r < A.rcap) {
                A.rec_key[r] = rk[q];
                A.rec_val[r] = rs[q];
            } else {
                atomicOr(&A.ctl->err, kErrRecords);
            }
        }
        __syncwarp();
        nrec = 0;
    }
    // Warp-collective; nrec < 32 on entry, so the stage (64) never overflows.
    SKIM_DEV void record(const TravArgs &A, bool first, uint64_t key, uint64_t slot) {
        const unsigned ball = __ballot_sync(kFull, first);
        if (!ball) return;
        if (first) {
            const uint32_t at = nrec + __popc(ball & lanemask_lt());
            rk[at] = key;
            rs[at] = static_cast<uint32_t>(slot);
        }
        nrec += __popc(ball);
        if (nrec >= 32) flush(A);
    }
    // Warp-collective: the lanes whose items fit below the ring limit (in lane
    // order) put them in the ring; the others hand theirs to the global queue.
    SKIM_DEV void rows(const TravArgs &A, Acc &acc, uint32_t ni, uint64_t b0, uint64_t b1, uint32_t t, int j,
                       uint32_t inst, uint64_t slot) {
        unsigned long long tot;
        const unsigned long long ex = warp_excl_scan(ni, &tot);
        if (tot == 0) return;
        const uint32_t used = rt - rh;
        const uint32_t room = keep > used ? keep - used : 0;
        const bool local = ni && ex + ni <= room;
        const unsigned lb = __ballot_sync(kFull, local);
        if (local) {
            const uint32_t w = row_item_w(t, j, inst);
            uint32_t at = rt + static_cast<uint32_t>(ex);
            for (uint64_t e = b0; e < b1; e += kChunk, at++) {
                Item it;
                it.v = static_cast<uint32_t>(e);
                it.w = w;
                it.mask = b1 - e < kChunk ? b1 - e : static_cast<uint64_t>(kChunk);
                ring[at & (kRingCap - 1)] = it;
            }
        }
        // the local lanes form a prefix in lane order: their items fill the
        // ring from rt on without gaps
        unsigned long long ltot = 0;
        if (lb) ltot = __shfl_sync(kFull, ex + ni, 31 - __clz(lb));
        rt += static_cast<uint32_t>(ltot);
        __syncwarp();
        if (ltot < tot) GlobalSink{}.rows(A, acc, local ? 0 : ni, b0, b1, t, j, inst, slot);
    }
};

// Warp-collective: expand the row items held by the lanes with `have`.  An
// item of 32 or more entries is swept by the whole warp (lane = entry, the
// next entry's id loaded while the current one is visited); the entries of
// the smaller items are spread over the lanes, 32 per round, so that a warp
// does not loop as long as its longest small row with most lanes idle.
SKIM_DEV void ring_expand(const TravArgs &A, Acc &acc, RingSink &sk, bool have, const Item &it) {
    const uint32_t lane = threadIdx.x & 31;
    const Desc d = describe<false, true>(A, have, it);
    acc.edges += d.cnt;
    const uint32_t dj = d.cnt ? static_cast<uint32_t>(__ffsll(d.mask) - 1) : 0;
    unsigned big = __ballot_sync(kFull, d.cnt >= 32);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t bb = __shfl_sync(kFull, d.begin, src), bc = __shfl_sync(kFull, d.cnt, src);
        const uint32_t bt = __shfl_sync(kFull, d.w, src) >> kChunkBits, bj = __shfl_sync(kFull, dj, src);
        const uint32_t bi = __shfl_sync(kFull, d.inst, src);
        uint32_t x = lane < bc ? A.col[bb + lane] : 0;
        for (uint32_t k0 = 0; k0 < bc; k0 += 32) {
            const uint32_t k = k0 + lane;
            const uint32_t xn = k + 32 < bc ? A.col[bb + k + 32] : 0;
            emit_rev_mat(A, acc, sk, k < bc, x, bt, static_cast<int>(bj), bi);
            x = xn;
        }
    }
    const uint32_t c = d.cnt < 32 ? d.cnt : 0;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= static_cast<uint32_t>(o)) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t g = 0; g < total; g += 32) {
        const uint32_t o = g + lane;
        // owner: the first lane whose inclusive count exceeds o
        uint32_t sl = 0;
#pragma unroll
        for (uint32_t step = 16; step > 0; step >>= 1) {
            const uint32_t v = __shfl_sync(kFull, incl, sl + step - 1);
            if (v <= o) sl += step;
        }
        const uint32_t sb = __shfl_sync(kFull, d.begin, sl), sp = __shfl_sync(kFull, incl - c, sl);
        const uint32_t st = __shfl_sync(kFull, d.w, sl) >> kChunkBits, sj = __shfl_sync(kFull, dj, sl);
        const uint32_t si = __shfl_sync(kFull, d.inst, sl);
        const bool has = o < total;
        const uint32_t x = has ? A.col[sb + (o - sp)] : 0;
        emit_rev_mat(A, acc, sk, has, x, st, static_cast<int>(sj), si);
    }
}

// Source lanes of a batch for the searches with per-warp queues.
struct RingSrc {
    const uint32_t *lane_pair;  // pair id v*l + i of every lane
    uint32_t B, l;
    const uint64_t *covered;    // SKIM: covered pairs are skipped (null: Algorithm 2)
    uint64_t *alive;            // SKIM: per word, the lanes whose source pair is uncovered
    int sources;                // 0: the sources were taken by an earlier launch
};

// Warp-collective: claim up to `want` global items (lanes first .. first +
// got - 1 receive them; `it`/`have` of the other lanes are left as they are).
// Returns the number claimed (0 if there were none or another warp won).
SKIM_DEV uint32_t ring_claim_global(const TravArgs &A, uint32_t first, uint32_t want, Item &it, bool &have) {
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long h = 0, got = 0;
    if (lane == 0) {
        h = ld_volatile(&A.ctl->q_head.v);
        const unsigned long long t = ld_volatile(&A.ctl->q_tail.v);
        const unsigned long long lim = t < A.qcap ? t : A.qcap;
        if (h < lim) {
            const unsigned long long n = lim - h < want ? lim - h : want;
            got = atomicCAS(&A.ctl->q_head.v, h, h + n) == h ? n : 0;
        }
    }
    h = __shfl_sync(kFull, h, 0);
    got = __shfl_sync(kFull, got, 0);
    if (!got) return 0;
    bool pending = lane >= first && lane < first + got;
    const unsigned long long slot = h + (lane - first);
    const uint64_t t0 = globaltimer();
    while (__any_sync(kFull, pending)) {
        if (pending && read_item(A, slot, &it)) {
            pending = false;
            have = true;
        }
        if (pending && globaltimer() - t0 > A.timeout_ns) {  // a reserved slot is written right away
            atomicOr(&A.ctl->err, kErrTimeout);
            pending = false;
        }
        if (__any_sync(kFull, pending)) __nanosleep(32);
    }
    return static_cast<uint32_t>(got);
}

// Warp-collective: claim up to 32 global items below lim (head h was read
// just before); false if another warp claimed them first.
SKIM_DEV bool ring_take_global(const TravArgs &A, Acc &acc, RingSink &sk, unsigned long long h,
                               unsigned long long lim) {
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long n = lim - h < 32 ? lim - h : 32;
    unsigned long long got = 0;
    if (lane == 0) got = atomicCAS(&A.ctl->q_head.v, h, h + n) == h ? n : 0;
    got = __shfl_sync(kFull, got, 0);
    if (!got) return false;
    Item it{0, 0, 0};
    bool pending = lane < got, have = false;
    const uint64_t t0 = globaltimer();
    while (__any_sync(kFull, pending)) {
        if (pending && read_item(A, h + lane, &it)) {
            pending = false;
            have = true;
        }
        if (pending && globaltimer() - t0 > A.timeout_ns) {  // a reserved slot is written right away
            atomicOr(&A.ctl->err, kErrTimeout);
            pending = false;
        }
        if (__any_sync(kFull, pending)) __nanosleep(32);
    }
    ring_expand(A, acc, sk, have, it);
    return true;
}

// Warp-collective: claim the next 32 source lanes of the batch and visit
// their nodes (Algorithm 2 prunes a full local sketch; SKIM skips a covered
// pair and marks the others alive).  False once the sources are used up.
SKIM_DEV bool ring_take_sources(const TravArgs &A, Acc &acc, RingSink &sk, const RingSrc &S) {
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long j0 = 0;
    if (lane == 0) j0 = atomicAdd(&A.ctl->src_next.v, 32ull);
    j0 = __shfl_sync(kFull, j0, 0);
    if (j0 >= S.B) return false;
    const uint32_t j = static_cast<uint32_t>(j0) + lane;
    bool act = j < S.B;
    uint32_t u = 0, i = 0;
    if (act) {
        const uint32_t pr = S.lane_pair[j];
        u = pr / S.l;
        i = pr % S.l;
        if (S.covered && ((S.covered[u] >> i) & 1ull)) act = false;
    }
    if (S.alive) {
        const unsigned b = __ballot_sync(kFull, act);
        if (lane == 0 && b)
            atomicOr(reinterpret_cast<unsigned long long *>(&S.alive[j0 >> 6]),
                     static_cast<unsigned long long>(b) << (((j0 >> 5) & 1) * 32));
    }
    emit_rev_mat(A, acc, sk, act, u, j >> 6, static_cast<int>(j & 63), i);
    return true;
}

#ifndef SKIM_RING_MIN_BLOCKS
#define SKIM_RING_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(kRingThreads, SKIM_RING_MIN_BLOCKS) k_rev_ring(TravArgs A, RingSrc S) {
    __shared__ Item s_ring[kRingThreads / 32][kRingCap];
    __shared__ uint64_t s_rk[kRingThreads / 32][kRecStage];
    __shared__ uint32_t s_rs[kRingThreads / 32][kRecStage];
    const uint32_t wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DevCtl *C = A.ctl;
    RingSink sk{s_ring[wib], s_rk[wib], s_rs[wib], 0, 0, 0, kRingKeep};
    Acc acc;
    bool src_done = !S.sources, busy = false;
    uint64_t t_progress = globaltimer();
    unsigned long long seen = 0;
    unsigned backoff = 32;
    uint32_t steps = 0;
    for (;;) {
        const uint32_t avail = sk.rt - sk.rh;
        // While sources remain, a ring that holds less than a full step takes
        // the next 32 source lanes first, so that steps run with full warps.
        if (avail < 32 && !src_done) {
            if (!busy) {
                if (lane == 0) {
                    atomicAdd(&C->busy.v, 1ull);
                    __threadfence();  // counted before the claim below
                }
                busy = true;
            }
            if (ring_take_sources(A, acc, sk, S)) continue;
            src_done = true;
        }
        if (avail) {
            const uint32_t nt = avail < 32 ? avail : 32;
            Item it{0, 0, 0};
            bool have = lane < nt;
            if (have) it = sk.ring[(sk.rh + lane) & (kRingCap - 1)];
            __syncwarp();
            sk.rh += nt;
            sk.keep = src_done ? kRingKeepTail : kRingKeep;
            // once the sources are used up, a partial step takes handed-over
            // items too
            if (src_done && nt < 32) ring_claim_global(A, nt, 32 - nt, it, have);
            ring_expand(A, acc, sk, have, it);
            if ((++steps & 15) == 0) {
                // a batch that overflowed its tables is re-run with fewer
                // lanes: stop working on it
                unsigned e = 0;
                if (lane == 0) {
                    if ((steps & 63) == 0) atomicAdd(&C->beat.v, 1ull);
                    e = *reinterpret_cast<volatile unsigned *>(&C->err);
                }
                if (__shfl_sync(kFull, e, 0) & (kErrRetryable | kErrTimeout)) {
                    sk.rh = sk.rt;
                    src_done = true;
                }
            }
            continue;
        }
        // the ring is empty and the sources are used up: items other warps
        // handed over
        unsigned long long h = 0, t = 0;
        if (lane == 0) {
            h = ld_volatile(&C->q_head.v);
            t = ld_volatile(&C->q_tail.v);
        }
        h = __shfl_sync(kFull, h, 0);
        t = __shfl_sync(kFull, t, 0);
        const unsigned long long lim = t < A.qcap ? t : A.qcap;
        if (h < lim) {
            if (!busy) {
                if (lane == 0) {
                    atomicAdd(&C->busy.v, 1ull);
                    __threadfence();
                }
                busy = true;
            }
            if (ring_take_global(A, acc, sk, h, lim)) {
                backoff = 32;
                continue;
            }
        }
        // nothing to do: records out, no longer counted as holding work
        sk.flush(A);
        if (busy) {
            if (lane == 0) {
                __threadfence();  // pushes of this warp are visible before the count drops
                atomicAdd(&C->busy.v, ~0ull);
            }
            busy = false;
        }
        int fin = 0;
        if (lane == 0) {
            __threadfence();
            const unsigned long long b = ld_volatile(&C->busy.v);
            __threadfence();
            const unsigned long long h2 = ld_volatile(&C->q_head.v), t2 = ld_volatile(&C->q_tail.v);
            const unsigned long long s2 = ld_volatile(&C->src_next.v);
            const bool no_src = !S.sources || s2 >= S.B;
            if (b == 0 && h2 >= (t2 < A.qcap ? t2 : A.qcap) && no_src) fin = 1;
            // progress anywhere: a claim, a push, a source, a working warp's beat
            const unsigned long long now = ld_volatile(&C->beat.v) + h2 * 3 + t2 * 5 + s2 * 7 + b * 11;
            if (now != seen) {
                seen = now;
                t_progress = globaltimer();
            }
            if (*reinterpret_cast<volatile unsigned *>(&C->err) & (kErrTimeout | kErrRetryable)) fin = 2;
            if (!fin && globaltimer() - t_progress > A.timeout_ns) {
                atomicOr(&C->err, kErrTimeout);
                fin = 2;
            }
        }
        fin = __shfl_sync(kFull, fin, 0);
        if (fin) break;
        // idle warps poll the shared cursors rarely, so that the working
        // warps' atomics on them are not held up
        __nanosleep(backoff);
        if (backoff < kRingIdleMaxNs) backoff <<= 1;
    }
    sk.flush(A);
    flush_acc(A, acc, false);
}

// ---- The global-queue search ----

// Items a warp finishes before it adds them to the shared done count with one
// atomic (the queue cursors are single words that every warp updates).
constexpr unsigned long long kDoneBatch = 64;

// Reverse searches over materialised rows (MAT) stage their visit records in
// shared memory and spread the entries of small row items over the warp's
// lanes, as the per-warp-queue search does (a RingSink whose ring limit is 0
// puts every row item into the global queue).  Residual searches over
// materialised rows keep items in the block's ring (FwdRing) while it has
// room; a warp takes ring items into its lanes that hold no queue item.
struct NoRing {};
template <bool FWD, bool MAT>
__global__ void __launch_bounds__(kTravThreads, FWD ? 1 : SKIM_TRAV_MIN_BLOCKS) k_traverse(TravArgs A) {
    constexpr bool kStaged = !FWD && MAT;
    constexpr bool kLocal = FWD && MAT && kFwdKeep > 0;
    __shared__ uint64_t ginst[64];  // (i + 1) * G for instance i (residual searches)
    __shared__ uint64_t s_rk[kStaged ? kTravThreads / 32 : 1][kStaged ? kRecStage : 1];
    __shared__ uint32_t s_rs[kStaged ? kTravThreads / 32 : 1][kStaged ? kRecStage : 1];
    __shared__ typename std::conditional<kLocal, FwdRing, NoRing>::type s_ring;
    FwdRing *ring = nullptr;
    if constexpr (kLocal) {
        ring = &s_ring;
        ring_init(ring);
    }
    if (threadIdx.x < 64) ginst[threadIdx.x] = kGolden * static_cast<uint64_t>(threadIdx.x + 1);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    DevCtl *C = A.ctl;
    Acc acc;
    GlobalSink gsink;
    FwdSink fsink{ring};
    const uint32_t wib = kStaged ? threadIdx.x >> 5 : 0;
    RingSink ssink{nullptr, s_rk[wib], s_rs[wib], 0, 0, 0, 0};
    uint64_t t_progress = globaltimer();
    unsigned long long seen_done = ld_volatile(&C->q_done.v);
    // items this warp has finished but not yet added to the done count: added
    // in batches, and always before the warp waits or leaves (a done count
    // that lags only delays the drain test)
    unsigned long long done_pend = 0;
    unsigned steps = 0;
    bool done = false;
    while (!done) {
        // Claims are interleaved across warps: claim c of a grid with W warps
        // takes, for lane l, queue slot (c / W) * 32W + l * W + (c mod W), so
        // consecutive items go to different warps.  (With contiguous claims
        // a narrow search - one seed - would run on a single warp.)
        unsigned long long claim = 0;
        if (lane == 0) claim = atomicAdd(&C->q_head.v, 1ull);
        claim = __shfl_sync(kFull, claim, 0);
        const unsigned long long W = static_cast<unsigned long long>(gridDim.x) * (blockDim.x / 32);
        const unsigned long long slot = (claim / W) * 32 * W + static_cast<unsigned long long>(lane) * W + claim % W;
        bool pending = slot < A.qcap;
        bool empty = !pending;  // resolved without an item
        unsigned backoff = 32, polls = 0;
        for (;;) {
            Item it{0, 0, 0};
            bool have = false;
            if (pending && read_item(A, slot, &it)) {
                have = true;
                pending = false;
            }
            const unsigned hb = __ballot_sync(kFull, have);
            unsigned lb = 0;  // lanes holding a ring item
            if constexpr (kLocal) {
                if (hb != kFull) lb = ring_take(A, ring, ~hb, have, it);
            }
            if (hb | lb) {
                if constexpr (kStaged)
                    ring_expand(A, acc, ssink, have, it);
                else if constexpr (FWD)
                    process_items<FWD, MAT>(A, acc, fsink, have, it, ginst);
                else
                    process_items<FWD, MAT>(A, acc, gsink, have, it, ginst);
                if constexpr (kLocal) {
                    // after the items' own pushes (their reservations are made)
                    __syncwarp();
                    if (lb && lane == 0) ring_finish(A, ring, __popc(lb));
                }
                // The drain test reads done, then tail, so the slots reserved
                // while processing must be counted in tail before these items
                // count as done.  No fence is needed: lane 0 made every
                // reservation of this warp with an atomic whose result it has
                // already used, so that atomic has been performed at the point
                // of coherence before this one is issued.  (Items themselves are
                // found by their non-zero fields, not by ordering.)
                acc.pushed = false;
                done_pend += __popc(hb);
                if (done_pend >= kDoneBatch) {
                    if (lane == 0) atomicAdd(&C->q_done.v, done_pend);
                    done_pend = 0;
                }
                t_progress = globaltimer();
                backoff = 32;
                polls = 0;
                // a batch that overflowed its tables is re-run smaller: stop
                // soon rather than finish a search whose result is dropped
                if ((++steps & 15) == 0) {
                    unsigned e = 0;
                    if (lane == 0) e = *reinterpret_cast<volatile unsigned *>(&C->err);
                    if (__shfl_sync(kFull, e, 0) & (kErrRetryable | kErrTimeout)) {
                        done = true;
                        break;
                    }
                }
            } else if (__any_sync(kFull, pending)) {
                if (done_pend) {
                    if (lane == 0) atomicAdd(&C->q_done.v, done_pend);
                    done_pend = 0;
                }
                // nothing ready: items are still being written, more may be
                // pushed, or the queue has drained.  The shared cursors are
                // read only every 8th poll of the warp's own slots.
                if ((++polls & 7) == 0) {
                    unsigned long long d = ld_volatile(&C->q_done.v);
                    __threadfence();
                    unsigned long long tl = ld_volatile(&C->q_tail.v);
                    if (d == tl && pending && slot >= tl) {
                        pending = false;
                        empty = true;
                    }
                    if (d != seen_done) {
                        seen_done = d;
                        t_progress = globaltimer();
                    }
                }
                // stop when another warp gave up or the batch overflowed
                const bool stopped = (polls & 7) == 0 && (*reinterpret_cast<volatile unsigned *>(&C->err) &
                                                          (kErrTimeout | kErrRetryable));
                const bool gave_up = globaltimer() - t_progress > A.timeout_ns;
                if (__any_sync(kFull, gave_up) && lane == 0) atomicOr(&C->err, kErrTimeout);
                if (__any_sync(kFull, gave_up || stopped)) {
                    done = true;
                    break;
                }
                if constexpr (kLocal) {
                    // a block whose ring has stayed empty frees its token
                    if (lane == 0 && globaltimer() - t_progress > kFwdParkNs) ring_release(A, ring);
                }
#ifndef SKIM_SPIN
#define SKIM_SPIN 0
#endif
#ifndef SKIM_FWD_SLEEP
#define SKIM_FWD_SLEEP 0
#endif
#if SKIM_SPIN == 0
                // a residual search's idle warps poll without pausing: it is
                // the only work on the device and its hops are latency-bound
                if (!FWD || SKIM_FWD_SLEEP) {
                    __nanosleep(backoff);
                    if (backoff < 512) backoff <<= 1;
                }
#elif SKIM_SPIN == 2
                {
                    const long long t0 = clock64();
                    while (clock64() - t0 < 256) {
                    }
                }
#endif
            }
            if (!__any_sync(kFull, pending)) break;
        }
        if (__any_sync(kFull, empty)) done = true;
    }
    if constexpr (kLocal) {
        // A warp leaves its block's ring empty (the queue ran out of slots,
        // or drained, in which case the ring is empty already): its items can
        // be taken by this block's warps only.  Warps still working take the
        // items they push themselves before they leave.
        uint64_t t_last = globaltimer();
        for (;;) {
            unsigned e = 0;
            if (lane == 0) e = *reinterpret_cast<volatile unsigned *>(&C->err);
            if (__shfl_sync(kFull, e, 0) & (kErrRetryable | kErrTimeout)) break;
            Item it{0, 0, 0};
            bool have = false;
            const unsigned lb = ring_take(A, ring, kFull, have, it);
            if (!lb) {
                int idle = 0;
                if (lane == 0) {
                    idle = ld_vol(&ring->tail) == ld_vol(&ring->head);
                    if (idle) ring_release(A, ring);
                }
                if (__shfl_sync(kFull, idle, 0)) break;
                if (globaltimer() - t_last > A.timeout_ns) {
                    if (lane == 0) atomicOr(&C->err, kErrTimeout);
                    break;
                }
                continue;
            }
            t_last = globaltimer();
            process_items<FWD, MAT>(A, acc, fsink, have, it, ginst);
            __syncwarp();
            if (lane == 0) ring_finish(A, ring, __popc(lb));
        }
    }
    if (done_pend && lane == 0) atomicAdd(&C->q_done.v, done_pend);
    if constexpr (kStaged) ssink.flush(A);
    flush_acc(A, acc, FWD);
}

}  // namespace

// Grid of the global-queue kernel k_traverse.  Its claims are interleaved
// over all warps of the grid (claim c of a warp covers a fixed set of slots),
// and a warp keeps its claim until the slot is written or the queue drains,
// so every block of the grid must be resident at once: a block that cannot
// start leaves slots below the tail unclaimed, and the resident warps then
// wait until the time limit and the call returns SKIM_ETIMEOUT (no hang).  So
// the grid is at most the blocks that fit on the device by the occupancy of
// every instantiation that may be launched with it, and another kernel that
// occupies SMs at the same time (another stream of this process, another
// context) can break it the same way.  The reverse searches over materialised
// rows (k_rev_ring) have no such requirement.
int traverse_grid(bool forward) {
    int dev = 0, sms = 0, per = 0, per2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // A residual search starts from one seed and stays narrow: one block per
    // SM keeps the idle warps (which poll) few.  Reverse searches of a batch
    // fill the machine: as many blocks as fit.
    if (forward) return sms;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_traverse<false, false>, kTravThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_traverse<false, true>, kTravThreads, 0);
    if (per2 < per) per = per2;
    if (per < 1) per = 1;
    return sms * per;
}

int rev_ring_grid() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rev_ring, kRingThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_rev_ring(const TravArgs &a, const uint32_t *lane_pair, uint32_t B, uint32_t l,
                            const uint64_t *covered, uint64_t *alive, bool sources, int grid, cudaStream_t s) {
    note_launch();
    const RingSrc src{lane_pair, B, l, covered, alive, sources ? 1 : 0};
    k_rev_ring<<<grid, kRingThreads, 0, s>>>(a, src);
    return cudaGetLastError();
}

cudaError_t launch_traverse(const TravArgs &a, bool forward, int grid, cudaStream_t s) {
    note_launch();
    if (forward) {
        if (a.mat)
            k_traverse<true, true><<<grid, kTravThreads, 0, s>>>(a);
        else
            k_traverse<true, false><<<grid, kTravThreads, 0, s>>>(a);
    } else {
        if (a.mat)
            k_traverse<false, true><<<grid, kTravThreads, 0, s>>>(a);
        else
            k_traverse<false, false><<<grid, kTravThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

namespace {

// Sources of a batch: lane j starts at the node of its pair.  Algorithm 2
// prunes a source whose local sketch in its instance is full; SKIM skips a
// covered source pair (its rank is consumed without a search).
__global__ void k_rev_sources(TravArgs A, const uint32_t *lane_pair, uint32_t B, uint32_t l, const uint64_t *covered,
                              uint64_t *alive) {
    const int lane = threadIdx.x & 31;
    Acc acc;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w * 32 < B; w += warps) {
        const uint32_t j = w * 32 + lane;
        bool act = j < B;
        uint32_t u = 0, i = 0;
        if (act) {
            uint32_t pr = lane_pair[j];
            u = pr / l;
            i = pr % l;
            if (A.prune && ((A.full[u] >> i) & 1ull)) act = false;
            if (covered && ((covered[u] >> i) & 1ull)) act = false;
        }
        if (alive) {
            unsigned b = __ballot_sync(kFull, act);
            if (lane == 0 && b) {
                uint64_t bits = static_cast<uint64_t>(b) << ((w & 1) * 32);
                atomicOr(reinterpret_cast<unsigned long long *>(&alive[w >> 1]), bits);
            }
        }
        GlobalSink gsink;
        if (A.mat)
            emit_rev_mat(A, acc, gsink, act, u, j >> 6, static_cast<int>(j & 63), i);
        else
            emit_rev<false>(A, acc, act, u, j >> 6, 1ull << (j & 63));
    }
    flush_acc(A, acc, false);
}

__global__ void k_respill_rev(TravArgs A, uint64_t R) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
    const uint64_t tmask = (1ull << A.tbits) - 1;
    for (uint64_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w * 32 < R; w += warps) {
        const uint64_t r = w * 32 + lane;
        uint64_t p = 0, slot = 0, key = 0;
        if (r < R) {
            slot = A.rec_val[r];
            key = A.rec_key[r];
            p = atomicExch(reinterpret_cast<unsigned long long *>(&A.pend[slot]), 0ull);
        }
        Acc acc;
        if (A.mat)
            push_rev<true>(A, acc, static_cast<uint32_t>(key >> A.tbits), static_cast<uint32_t>(key & tmask), p, slot);
        else
            push_rev<false>(A, acc, static_cast<uint32_t>(key >> A.tbits), static_cast<uint32_t>(key & tmask), p, slot);
    }
}

__global__ void k_respill_fwd(TravArgs A, uint32_t n) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w * 32 < n; w += warps) {
        const uint32_t v = w * 32 + lane;
        uint64_t pt = 0, pe = 0;
        if (v < n) {
            pt = atomicExch(reinterpret_cast<unsigned long long *>(&A.pend_trav[v]), 0ull);
            pe = atomicExch(reinterpret_cast<unsigned long long *>(&A.pend_erase[v]), 0ull);
        }
        Acc acc;
        if (A.mat)
            push_fwd<true>(A, acc, v < n ? v : 0, pt, pe, PairPre{});
        else
            push_fwd<false>(A, acc, v < n ? v : 0, pt, pe, PairPre{});
    }
}

// The seed x covers its pairs in every instance: with materialised instances
// lane j takes instances j and j + 32, otherwise lane 0 takes them all.
__global__ void k_fwd_source(TravArgs A, uint32_t x) {
    const uint64_t lmask = A.l == 64 ? ~0ull : ((1ull << A.l) - 1);
    Acc acc;
    if (A.mat) {
        for (uint32_t i0 = 0; i0 < A.l; i0 += 32) {
            const uint32_t i = i0 + threadIdx.x;
            emit_fwd<true>(A, acc, i < A.l, x, i < A.l ? 1ull << i : 0);
        }
    } else {
        emit_fwd<false>(A, acc, threadIdx.x == 0, x, lmask);
    }
    flush_acc(A, acc, true);
}

}  // namespace

cudaError_t launch_rev_sources(const TravArgs &a, const uint32_t *lane_pair, uint32_t B, uint32_t l,
                               const uint64_t *covered, uint64_t *alive, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    unsigned warps = (B + 31) / 32;
    unsigned blocks = (warps + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    note_launch();
    k_rev_sources<<<blocks, 256, 0, s>>>(a, lane_pair, B, l, covered, alive);
    return cudaGetLastError();
}

cudaError_t launch_respill_rev(const TravArgs &a, uint64_t R, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    uint64_t warps = (R + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    note_launch();
    k_respill_rev<<<static_cast<unsigned>(blocks), 256, 0, s>>>(a, R);
    return cudaGetLastError();
}

cudaError_t launch_respill_fwd(const TravArgs &a, uint32_t n, cudaStream_t s) {
    uint64_t warps = (n + 31) / 32;
    uint64_t blocks = (warps + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    note_launch();
    k_respill_fwd<<<static_cast<unsigned>(blocks), 256, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_fwd_source(const TravArgs &a, uint32_t x, cudaStream_t s) {
    note_launch();
    k_fwd_source<<<1, 32, 0, s>>>(a, x);
    return cudaGetLastError();
}

}  // namespace skim

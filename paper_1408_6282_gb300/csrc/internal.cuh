// internal.cuh -- launchers and argument blocks shared by the libskim
// translation units (host-visible declarations; kernels live in the .cu files).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

struct skim_ctx;  // the C ABI's opaque context (capi.cu)

namespace skim {

// Live-edge threshold model (Section 6: uniform p, weighted cascade 1/indeg,
// trivalency classes).
struct CoinModel {
    int model;            // 0 uniform, 1 weighted cascade, 2 trivalency, 3 per-edge thresholds (many graphs)
    uint64_t tm1_uniform;  // floor(p * 2^64) - 1
    uint64_t tm1_class[3];
    const uint64_t *thr_wc;  // per node: floor((2^64-1) / indeg(node))
    uint64_t coin_key;
    uint64_t prob_key;
};

// Arguments of the asynchronous traversal kernels.
struct TravArgs {
    const uint32_t *ptr;  // CSR row pointers in the search direction
    const uint32_t *col;
    CoinModel cm;
    Item *q;
    uint64_t qcap;
    DevCtl *ctl;
    uint64_t timeout_ns;
    // reverse searches (lanes = ranks of a batch)
    uint64_t *hkeys;
    uint64_t *hvals;
    uint64_t hmask;             // the batch's table prefix (slots - 1), cleared before the batch
    uint64_t *rec_key;
    uint32_t *rec_val;
    uint64_t rcap;
    uint32_t tbits;             // record key = (node << tbits) | word
    uint32_t hnode;             // visited-table slots grouped by node (batches of few words)
    const uint8_t *lane_inst;   // instance of every lane of the batch
    const uint64_t *lane_g;     // per lane: (instance + 1) * G, the lane's coin-stream offset
    const uint64_t *he;         // per CSR edge: state of its coin stream, fmix(coin_key ^ (u << 32 | v))
    const uint64_t *tm1e;       // per CSR edge: live threshold (model 3)
    const uint64_t *full;       // Algorithm 2 pruning: instances whose local sketch holds k ranks
    int prune;
    uint64_t *pend;             // per table slot: lane bits whose expansion was spilled
    // residual (forward) searches (lanes = instances)
    uint64_t *covered;
    const uint64_t *seg_start;
    uint32_t *seg_len;
    uint32_t *size;
    const uint32_t *idx_nodes;
    uint32_t l;
    uint64_t *pend_trav;        // per node: instances whose expansion was spilled
    uint64_t *pend_erase;       // per node: instances whose index erasure was spilled
    // materialised instances (mat != 0): reverse searches walk the live
    // in-neighbours of (node v, instance i), col[loff[v*l+i] .. loff[v*l+i+1])
    // (offsets masked by kRowMask; kRowFull on a row start marks a full local
    // sketch), forward searches the live out-neighbours the same way
    int mat;
    const uint32_t *loff;
    const uint64_t *lmask;
};

// graph.cu
cudaError_t launch_check_edges(const uint32_t *src, const uint32_t *dst, uint64_t m, uint32_t n, unsigned *bad,
                               cudaStream_t s);
// ptr[v] = first index with row[index] >= v, for v = 0..n (row sorted)
cudaError_t launch_row_ptr(const uint32_t *row, uint64_t m, uint32_t n, uint32_t *ptr, cudaStream_t s);
// rhe[e] = fhe[rev2fwd[e]] = edge_state(coin_key, rcol[e], rrow[e]) over the reverse CSR
cudaError_t launch_edge_states_both(const uint32_t *rcol, const uint32_t *rrow, const uint32_t *rev2fwd, uint64_t m,
                                    uint64_t coin_key, uint64_t *rhe, uint64_t *fhe, cudaStream_t s);
cudaError_t launch_make_rev_keys(const uint32_t *src, const uint32_t *dst, uint64_t m, uint64_t *key, uint32_t *val,
                                 cudaStream_t s);
cudaError_t launch_split_rev(const uint64_t *key, const uint32_t *val, uint64_t m, uint32_t *rcol, uint32_t *rrow,
                             uint32_t *rev2fwd, cudaStream_t s);
cudaError_t launch_wc_thresholds(const uint32_t *rptr, uint32_t n, uint64_t *thr, cudaStream_t s);
// Per-edge coin-stream states of a CSR: he[e] for edge (row node, col[e]);
// reverse = 1 when rows are heads (edge col[e] -> row).
// Materialised instances (Section 2: the l live-edge graphs): live masks of
// every CSR edge (bit i = coin of instance i), and the node-major lists of live
// in-neighbours: counts per (v, i) into off[v*l + i], then (after an exclusive
// scan of off) the sources themselves.
cudaError_t launch_live_masks(const uint32_t *rrow, const uint32_t *rcol, const uint64_t *rhe, const uint64_t *rtm1,
                              const uint32_t *rev2fwd, const CoinModel &cm, uint64_t m, uint32_t l, uint64_t *rmask,
                              uint64_t *fmask, cudaStream_t s);
// Rows of more than 2048 edges are counted and filled in pieces, using a
// workspace of live_pieces_bytes(m); the count pass of a CSR direction must
// precede its fill pass with the same workspace.
size_t live_pieces_bytes(uint64_t m);
cudaError_t launch_live_count(const uint32_t *ptr, const uint64_t *mask, uint32_t n, uint64_t m, uint32_t l,
                              uint64_t *off, void *pieces_ws, cudaStream_t s);
cudaError_t launch_live_fill(const uint32_t *ptr, const uint32_t *col, const uint64_t *mask, uint32_t n, uint64_t m,
                             uint32_t l, const uint64_t *off, uint32_t *live, void *pieces_ws, cudaStream_t s);
// off32[r] = off[r] for r <= count (offsets below 2^31; no row flagged full)
cudaError_t launch_offsets_u32(const uint64_t *off, uint64_t count, uint32_t *off32, cudaStream_t s);
// clear the full flags (kRowFull) of rows 0 .. count - 1
cudaError_t launch_clear_row_flags(uint32_t *off32, uint64_t count, cudaStream_t s);

// Rank order of all pairs: bucket by the top bits, then sort each bucket.
// rank of pair x = v*l+i is fmix(rank_key + G*x), or fmix(rbase[v] + G*i)
// when a per-node base is given (graphs of a batch, each with its own key).
size_t rank_sort_workspace_bytes(uint64_t nl);
// Structured permutation (Section 3.1; ic = false: pairs (v, sigma_v(c))) or
// IC-model positions (Section 3.2; ic = true: nodes) for the first `chunks`
// chunks of n positions: sorted_rank[t] = t, sorted_pair[t] = pair or node.
uint64_t perm_key(uint64_t rank_key);
size_t perm_sort_workspace_bytes(uint32_t n, uint32_t l, uint32_t chunks, bool ic);
cudaError_t perm_sort(uint64_t rank_key, uint32_t n, uint32_t l, uint32_t chunks, bool ic, uint64_t *sorted_rank,
                      uint32_t *sorted_pair, void *ws, cudaStream_t s);
cudaError_t rank_sort(uint64_t rank_key, const uint64_t *rbase, uint32_t l, uint64_t nl, uint64_t *sorted_rank,
                      uint32_t *sorted_pair, void *ws, cudaStream_t s);

// Graphs of a batch (a disjoint union): per-graph keys and models, node ->
// graph, and the per-node / per-edge tables derived from them.
struct BatchDesc {
    uint32_t count;
    const uint32_t *node_graph;  // per node
    const uint32_t *node_off;    // per graph: first node
    const uint64_t *coin_key, *rank_key, *prob_key, *tm1_uniform;  // per graph
    const int *model;            // per graph: 0 uniform, 1 wc, 2 trivalency
    uint64_t tm1_class[3];       // trivalency thresholds for p = 0.1, 0.01, 0.001
};
cudaError_t launch_node_graph(const uint32_t *node_off, uint32_t count, uint32_t *node_graph, cudaStream_t s);
cudaError_t launch_edge_states_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, const BatchDesc &b,
                                     int reverse, uint64_t *he, cudaStream_t s);
cudaError_t launch_edge_tm1_batch(const uint32_t *ptr, const uint32_t *col, uint32_t n, const BatchDesc &b,
                                  const uint64_t *thr_wc, int reverse, uint64_t *tm1, cudaStream_t s);
cudaError_t launch_rank_bases(const BatchDesc &b, uint32_t n, uint32_t l, uint64_t *rbase, cudaStream_t s);

// traverse.cu
cudaError_t launch_rev_sources(const TravArgs &a, const uint32_t *lane_pair, uint32_t B, uint32_t l,
                               const uint64_t *covered, uint64_t *alive, cudaStream_t s);
cudaError_t launch_fwd_source(const TravArgs &a, uint32_t x, cudaStream_t s);
cudaError_t launch_traverse(const TravArgs &a, bool forward, int grid, cudaStream_t s);
// Re-queue spilled work (after a drained traversal that set DevCtl::spill).
cudaError_t launch_respill_rev(const TravArgs &a, uint64_t R, cudaStream_t s);
cudaError_t launch_respill_fwd(const TravArgs &a, uint32_t n, cudaStream_t s);
int traverse_grid(bool forward);  // resident blocks for the persistent traversal
// Reverse searches over materialised live rows with per-warp queues in shared
// memory (Algorithms 1 and 2): the batch's source lanes are taken by the
// kernel itself (sources = false: an earlier launch took them; covered/alive
// as for launch_rev_sources).  The source cursor DevCtl::src_next must be zero
// before the first launch of a batch.
int rev_ring_grid();
cudaError_t launch_rev_ring(const TravArgs &a, const uint32_t *lane_pair, uint32_t B, uint32_t l,
                            const uint64_t *covered, uint64_t *alive, bool sources, int grid, cudaStream_t s);

// batch.cu
cudaError_t launch_lane_inst(const uint32_t *lane_pair, const uint64_t *lane_rank, uint32_t B, uint32_t l,
                             uint8_t *lane_inst, uint64_t *lane_g, cudaStream_t s);
// Algorithm 2 acceptance of a batch's sorted records.  flag: R + 1 uint64 and
// starts: R + 1 uint32 of scratch; scan_ws: scan workspace for R + 1 entries.
// Algorithm 2's acceptance of a batch's sorted records; record r's lane bits
// are hvals[2 * rec_val[r]].
// row_flag (may be null): live-row offsets whose kRowFull bit is set with the
// full bit of (v, i).
cudaError_t launch_accept(const uint64_t *rec_key, const uint32_t *rec_val, const uint64_t *hvals, uint64_t R,
                          uint32_t tbits, const uint8_t *lane_inst, const uint64_t *lane_rank, uint32_t l, uint32_t k,
                          uint8_t *lcnt, uint64_t *full, uint32_t *row_flag, uint64_t *X, uint32_t *xlen, DevCtl *ctl,
                          cudaStream_t s);

// recsort.cu: order a batch's R records by key, node by node.  cnt: n + 1
// counters, all zero on entry and on return; off: n + 1 node offsets (out);
// tmp: R scratch words; list: n scratch entries; nlist: 2 scratch counters.
cudaError_t launch_node_sort(uint64_t *rec_key, uint32_t *rec_val, uint64_t R, uint32_t tbits, uint32_t n,
                             uint64_t *cnt, uint64_t *off, uint64_t *tmp, uint32_t *list, unsigned *nlist,
                             void *scan_ws, cudaStream_t s);
// SKIM batch: the records' lane bits gathered from the visited table into
// rbits (R words), read by the three kernels below.
cudaError_t launch_gather_bits(const uint32_t *rec_val, const uint64_t *hvals, uint64_t R, uint64_t *rbits,
                               cudaStream_t s);
cudaError_t launch_candidates(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                              const uint64_t *alive, uint32_t lo, const uint32_t *size, uint32_t k, DevCtl *ctl,
                              cudaStream_t s);
cudaError_t launch_commit_count(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                                const uint64_t *alive, uint32_t lo, uint32_t hi, uint32_t *size, uint64_t *lane_cnt,
                                DevCtl *ctl, cudaStream_t s);
cudaError_t launch_commit_scatter(const uint64_t *rec_key, const uint64_t *rbits, uint64_t R, uint32_t tbits,
                                  const uint64_t *alive, uint32_t lo, uint32_t hi, const uint64_t *lane_off,
                                  uint32_t *lane_fill, const uint64_t *idx_ctr, uint32_t *idx_nodes, cudaStream_t s);
cudaError_t launch_commit_segments(const uint32_t *lane_pair, uint32_t lo, uint32_t hi, const uint64_t *lane_cnt,
                                   const uint64_t *lane_off, const uint64_t *idx_ctr, uint64_t *seg_start,
                                   uint32_t *seg_len, cudaStream_t s);
// idx_ctr[1] = idx_ctr[0]; idx_ctr[0] += *total (the index entries a commit added)
cudaError_t launch_idx_advance(uint64_t *idx_ctr, const unsigned long long *total, cudaStream_t s);
cudaError_t launch_refilter(const uint32_t *lane_pair, uint32_t lo, uint32_t B, uint32_t l, const uint64_t *covered,
                            uint64_t *alive, cudaStream_t s);
cudaError_t launch_argmax_size(const uint32_t *size, uint32_t n, DevCtl *ctl, cudaStream_t s);
cudaError_t launch_min_unchosen(const uint8_t *chosen, uint32_t n, DevCtl *ctl, cudaStream_t s);
// Section 4.3.2: k' = max size over v != x with the stop lane p taken out
// (sizes are restored); atomicMax into *out, which the caller zeroes.
cudaError_t launch_second_size(const uint32_t *idx_nodes, const uint64_t *idx_base, const uint64_t *lane_off,
                               const uint64_t *lane_cnt, uint32_t p, uint32_t *size, uint32_t n, uint32_t x,
                               uint32_t *out, cudaStream_t s);

// query.cu
// Scratch of the multi-block query path: hash tables (total_slots keys and
// values), per-query top-rank slots, per-chunk partial sums, an error flag.
struct QueryScratch {
    uint64_t *hkeys;
    uint64_t *hvals;
    uint64_t *top_tau;
    unsigned *top_used;
    void *partial;
    unsigned *err;
};
uint32_t query_chunks(uint64_t table_slots);  // chunks of one query's table
size_t query_partial_bytes();                  // bytes per chunk partial
// How a threshold becomes a term of Eq. unionest, and the final divisor:
//  mode 0 (uniform 64-bit ranks): 1 / (h * 2^-64), divided by l;
//  mode 1 (structured permutation, Section 3.1): num / h with num = n*l - 1,
//          1 for a sketch that is not full, divided by l;
//  mode 2 (IC model, Section 3.2): num / h with num = n, 0 for a sketch that
//          is not full, divided by 1.
struct QueryTerms {
    int mode;
    double num;
    double div;
};
QueryTerms query_terms_of(const skim_ctx *c);
cudaError_t launch_node_estimates(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, uint32_t l,
                                  int mode, double *out, cudaStream_t s);
cudaError_t launch_query_multi(const uint64_t *X, const uint32_t *xlen, uint32_t n, uint32_t k, const QueryTerms &terms,
                               const uint32_t *seeds, const uint64_t *offsets, const uint64_t *table_off,
                               const uint64_t *chunk_off, uint32_t q, uint64_t total_slots, uint64_t total_seeds,
                               uint32_t total_chunks, const QueryScratch &qs, double *out, cudaStream_t s);

}  // namespace skim

/*
 * skim.h -- C ABI of libskim: combined bottom-k reachability sketches, SKIM
 * greedy seed selection and the sketch-based influence oracle on one GB300
 * GPU (sm_103a).
 *
 * Method: Cohen, Delling, Pajor, Werneck, "Sketch-based Influence
 * Maximization and Computation: Scaling up with Guarantees" (arXiv 1408.6282).
 *
 * Conventions for every call:
 *   - Return value: SKIM_OK (0) on success, a negative SKIM_E* code otherwise;
 *     skim_strerror() names it.  After SKIM_ECUDA or SKIM_ETIMEOUT the
 *     context is unusable and must be destroyed.
 *   - Ownership: inputs are borrowed for the duration of the call and copied;
 *     outputs are written to caller-owned buffers.  All device memory used by
 *     a context is allocated by the library, on the context's stream, from a
 *     pool per device, and skim_destroy() returns it to that pool (see
 *     skim_release_memory()).
 *   - Pointers marked (host) must be host memory; pointers marked
 *     (host|device) may be either, as stated by the accompanying flag.
 *   - Calls on one context are not thread-safe; use one context per thread.
 *   - All work runs on the stream given at creation (NULL: the legacy default
 *     stream); calls that return results on the host synchronise that stream.
 */
#ifndef SKIM_H
#define SKIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKIM_OK 0
#define SKIM_EINVAL -1    /* bad argument: null pointer, node id >= n, k < 2, l == 0 or l > 64, ... */
#define SKIM_ENOMEM -2    /* device or host allocation failed */
#define SKIM_ENOTBUILT -3 /* query before skim_build_sketches() */
#define SKIM_ETIMEOUT -4  /* a device-side wait hit its iteration cap; context unusable */
#define SKIM_ECUDA -5     /* a CUDA runtime call failed; context unusable */
#define SKIM_EGRAPH -6    /* edge list not canonical (unsorted, duplicate or self-loop) */
#define SKIM_ERANGE -7    /* a size exceeds a stated limit */

/* Probability models of the binary IC model (Section 6, "uniform" and
 * "weighted cascade"; trivalency assigns p in {0.1, 0.01, 0.001} per edge). */
#define SKIM_PROB_UNIFORM 0
#define SKIM_PROB_WC 1
#define SKIM_PROB_TRIVALENCY 2

/* Directed graph as a canonical edge list: m pairs (src[e], dst[e]) sorted by
 * (src, dst), no duplicates, no self-loops, ids < n.  An edge (u,v) means u
 * can infect v (Section 2).  on_device = 0: src/dst are host pointers;
 * 1: device pointers on the current device. */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint32_t *src;
    const uint32_t *dst;
    int on_device;
} skim_graph;

/* Parameters (Sections 3-4):
 *   l          number of IC instances, 1..64 (one 64-bit word per node holds a
 *              node's instances);
 *   k          sketch size, 2..255;
 *   prob_model SKIM_PROB_*; p is the uniform edge probability, 0 < p <= 1;
 *   coin_key   key of the live-edge coins: edge (u,v) is live in instance i
 *              iff fmix(fmix(coin_key ^ (u<<32|v)) + (i+1)*G) <= floor(p*2^64)-1,
 *              fmix the SplitMix64 output function, G = 0x9E3779B97F4A7C15;
 *              for weighted cascade the bound is floor((2^64-1)/indeg(v));
 *   rank_key   rank of pair (v,i) is fmix(rank_key + (v*l+i)*G), read as
 *              a real in [0,1) after scaling by 2^-64 (ranks never tie);
 *   prob_key   trivalency class of edge (u,v): fmix(prob_key ^ (u<<32|v)) % 3;
 *   batch_lanes  ranks per batched search, 0 = automatic (2M; 4M on graphs of
 *              2^23 nodes or more);
 *   rank_mode  SKIM_RANKS_*: how the pairs are ordered and what a sketch holds.
 *     SKIM_RANKS_UNIFORM (0): the uniform 64-bit ranks above.
 *     SKIM_RANKS_PERMUTATION (1): structured permutation ranks (Section 3.1).
 *       Positions 0..n*l-1 (the paper's T is the position plus one) come in
 *       l chunks of n; chunk c lists every node once, ordered by
 *       w(v,c) = fmix(K_w + (c*n+v)*G), K_w = fmix(rank_key ^ 0x7065726d75746531),
 *       and pairs node v with its (c+1)-th instance in the order of the ranks
 *       r(v,i) above.  Sketches hold positions; Algorithm 2 processes only the
 *       first min(k,l)*n positions (no later one can enter a sketch).
 *     SKIM_RANKS_IC_MODEL (2): IC-model sketches (Section 3.2), the limit of
 *       infinitely many instances: requires l = 1; position t < k*n (same
 *       chunk order, k chunks) has a fresh instance of its own whose coins use
 *       t in place of i; searches are not pruned.  SKIM is not available.
 *   Queries read a position threshold q as the uniform rank q/(n*l-1)
 *   (mode 1) or estimate n/q per rank (mode 2); see skim_oracle_query. */
typedef struct {
    uint32_t l;
    uint32_t k;
    int prob_model;
    double p;
    uint64_t coin_key;
    uint64_t rank_key;
    uint64_t prob_key;
    uint32_t batch_lanes;
    uint32_t rank_mode;
} skim_params;

#define SKIM_RANKS_UNIFORM 0
#define SKIM_RANKS_PERMUTATION 1
#define SKIM_RANKS_IC_MODEL 2

typedef struct skim_ctx skim_ctx;

/* Create a context on the current CUDA device: copies the graph, builds both
 * CSR directions in device memory and the rank order of all n*l pairs
 * (Section 3; "shuffle the nl node-instance pairs" of Algorithms 1 and 2 is
 * read as increasing rank order).  stream: a cudaStream_t, or NULL.
 * Errors: SKIM_EINVAL, SKIM_EGRAPH, SKIM_ENOMEM, SKIM_ECUDA. */
int skim_create(const skim_graph *g, const skim_params *prm, void *stream, skim_ctx **out);

/* Many independent graphs in one context (the batched form): graph g's node
 * v becomes node off_g + v, off_g = n_0 + ... + n_{g-1}, of a disjoint union
 * whose sketches are built in one pass of rank-batched searches
 * (skim_build_sketches; each graph's ranks stay in increasing order inside
 * the merged order, so Algorithm 2 stays exact per graph).  Every graph keeps
 * its own keys and probability model (params[g]); l and k must be equal.
 * graphs[g] are host edge lists.  Queries take union node ids; skim_greedy is
 * not defined on a batch (SKIM_EINVAL).  Errors as skim_create. */
int skim_create_batch(const skim_graph *graphs, const skim_params *params, uint32_t count, void *stream,
                      skim_ctx **out);

/* Autotuner of the rank-batch size: builds the sketches once per candidate
 * lane count, keeps the fastest for later builds.  best (host) receives it;
 * seconds (host, optional) the time of each candidate. */
int skim_autotune_batch_lanes(skim_ctx *ctx, const uint32_t *candidates, uint32_t count, uint32_t *best,
                              double *seconds);

/* Switches of the rank-batched searches (Algorithms 1 and 2 run a batch of
 * consecutive ranks as one search; none of these changes a result):
 *   batch_lanes            ranks per batch, 0 = automatic (2M, 4M on graphs
 *                          of 2^23 nodes or more, or fewer when the previous
 *                          batch's records per lane say so);
 *   ring_records_per_lane  a batch whose searches are expected to leave at
 *                          most this many visit records per lane (from the
 *                          previous batch) runs with per-warp work queues in
 *                          shared memory; larger searches share one global
 *                          queue over the whole GPU (default 8; 0 = always
 *                          the global queue);
 *   node_sort_density      a batch's visit records are placed by node
 *                          buckets (a counting pass over buckets of 2^s
 *                          consecutive nodes, s chosen for about one bucket
 *                          per record) when the buckets number at most
 *                          node_sort_density * records, else radix sorted
 *                          (default 4; 0 = always radix sorted). */
typedef struct {
    uint32_t batch_lanes;
    double ring_records_per_lane;
    uint32_t node_sort_density;
} skim_tuning;
int skim_get_tuning(skim_ctx *ctx, skim_tuning *out);
int skim_set_tuning(skim_ctx *ctx, const skim_tuning *t);

/* Autotuner over whole settings: builds the sketches once per candidate
 * (host array of count settings), keeps the fastest for later builds and
 * writes its index to *best (count if every build failed; the settings are
 * then left as they were).  seconds (host, optional): each candidate's build
 * time.  Errors: SKIM_EINVAL for a candidate with a negative records
 * threshold; a failing build's code. */
int skim_autotune(skim_ctx *ctx, const skim_tuning *candidates, uint32_t count, uint32_t *best, double *seconds);

/* Recompute the rank order of the n*l pairs (done by skim_create; exposed so
 * that a caller can time it).  Restarts SKIM (as skim_greedy_reset); the
 * sketches are unaffected (the ranks themselves do not change). */
int skim_rank_order(skim_ctx *ctx);

/* Generate the l live-edge instances (Section 2; Algorithms 1 and 2 take a set
 * of instances): every edge's coin in every instance is drawn once (the coin
 * above), giving a 64-bit live mask per edge in both CSR orders and, per
 * (node v, instance i), the list of v's live in-neighbours.  Searches then
 * walk live edges only.  Done by skim_create; exposed so that a caller can
 * time it.  Restarts SKIM (as skim_greedy_reset); sketches are unaffected (the
 * coins do not change).  The IC model (SKIM_RANKS_IC_MODEL) has an instance
 * per rank position and draws coins during the searches instead, as does a
 * context with 2^31 or more live (edge, instance) pairs. */
int skim_instances(skim_ctx *ctx);

/* Choose how searches draw the live edges (Section 2).  on = 1 (the default):
 * walk the materialised live rows of skim_instances where they exist.
 * on = 0: evaluate every edge's coin for the lanes that reach it during the
 * search (the hash above; no instance is stored), as the IC model and contexts
 * with 2^31 or more live pairs always do.  Both give bit-identical sketches,
 * seeds and coverages.  Takes effect at the next build or SKIM call and
 * restarts SKIM (as skim_greedy_reset). */
int skim_set_live_rows(skim_ctx *ctx, int on);

/* live_pairs: live (edge, instance) pairs of the last skim_instances;
 * materialised: 1 if searches use the materialised instances (host outputs). */
int skim_instance_stats(skim_ctx *ctx, uint64_t *live_pairs, int *materialised);

/* Algorithm 2 (Section 5.2): combined bottom-k reachability sketches X_v of
 * all nodes (Eq. combinedrs), computed by rank-batched pruned reverse
 * searches; the result equals the definition exactly.  Sketches stay in
 * device memory.  May be called again (recomputes). */
int skim_build_sketches(skim_ctx *ctx);

/* Copy sketches out: x_out[v*k + j] = j-th smallest rank of X_v (row-major,
 * n*k uint64), len_out[v] = |X_v| (n uint32).  out_on_device selects the
 * memory kind of both outputs.  SKIM_ENOTBUILT before skim_build_sketches(). */
int skim_get_sketches(skim_ctx *ctx, uint64_t *x_out, uint32_t *len_out, int out_on_device);

/* One node's sketch (Eq. combinedrs): out_k[j] = j-th smallest rank of X_v for
 * j < *out_len (out_k (host) must hold k entries; entries past *out_len are
 * left untouched), *out_len = |X_v| <= k (host).
 * Errors: SKIM_EINVAL (null pointer, v >= n), SKIM_ENOTBUILT. */
int skim_get_sketch(skim_ctx *ctx, uint32_t v, uint64_t *out_k, uint32_t *out_len);

/* Device pointers to the resident sketches (valid until the next build or
 * destroy), for callers that keep them on the GPU. */
int skim_sketch_pointers(skim_ctx *ctx, const uint64_t **x_dev, const uint32_t **len_dev);

/* SKIM, Algorithm 1 (Section 4): select n_seeds more seeds.  Continues the
 * sequence on repeated calls (resume after tau_v, Section 4).  Outputs (host):
 * seeds_out[j] the j-th new seed, cov_out[j] its marginal coverage in
 * node-instance pairs, i.e. l * I_j (integer).  Tie rules: the seed is the
 * smallest node id among nodes whose partial sketch reaches k on the same
 * rank; when ranks run out, argmax size with ties to the smallest id, and the
 * smallest unchosen id once everything is covered.
 * Errors: SKIM_EINVAL if the total would exceed n. */
int skim_greedy(skim_ctx *ctx, uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out);

/* skim_greedy plus what each selection saw, for adaptive error estimation
 * (Section 4.3.2).  For the j-th new seed, tau_out[j] is the threshold rank:
 * the 64-bit rank whose reverse search made the seed's partial sketch reach k
 * (read as tau * 2^-64), and kprime_out[j] is k', the largest partial sketch
 * size among all other nodes once that rank is taken out (k' <= k - 1).  When
 * the ranks have run out the seed comes from exact residual counts: then
 * tau_out[j] = 0 and kprime_out[j] = -1.  Either output may be NULL; with both
 * NULL this is skim_greedy.  Recording costs three small kernels per seed and
 * device arrays of 12 * n_seeds bytes for the call.  Errors as skim_greedy. */
int skim_greedy_ex(skim_ctx *ctx, uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out, uint64_t *tau_out,
                   int32_t *kprime_out);

/* Confidence bound on the sum of discrepancies of a SKIM run (Section 4.3.2,
 * Eq. chernoff); host-only FP64, no context, no GPU.  The discrepancy of
 * iteration j is the gap, in node-instance pairs, between the largest
 * marginal coverage in that residual problem and delta[j], the coverage of
 * the seed selected.  With mu = tau_j (delta_j + d) (tau_j = tau[j] * 2^-64)
 * and nu = 1 - k'_j / mu, P[D_j > d] <= B_j(d) = (e^-nu / (1-nu)^(1-nu))^mu,
 * or 1 where mu <= k'_j; kprime[j] = -1 is a point mass at 0.  Each D_j is
 * rounded up to the grid {0, step, 2 step, ...} of `bins` cells, with the mass
 * past the last cell held in an overflow cell that counts as unbounded; the
 * sum's bound is the convolution over j.
 * Inputs (host): delta, tau, kprime as written by skim_greedy_ex (s entries);
 * step > 0 in pairs; bins >= 1; conf[c] in (0, 1).
 * Outputs (host): bound_out[c] = the smallest grid value b with
 * P[sum > b] <= 1 - conf[c] (pairs; +inf if only the overflow cell would do);
 * ccdf_out (may be NULL, bins + 1 entries): ccdf_out[i] bounds P[sum > i step]
 * for i < bins, ccdf_out[bins] is the overflow mass.
 * Errors: SKIM_EINVAL for a null array that is needed, step <= 0 or not
 * finite, bins = 0, a confidence outside (0, 1), or kprime[j] < -1. */
int skim_discrepancy_bound(uint32_t s, const uint64_t *delta, const uint64_t *tau, const int32_t *kprime,
                           double step, uint32_t bins, uint32_t n_conf, const double *conf, double *bound_out,
                           double *ccdf_out);

/* Restart SKIM from the empty seed set (drops covered pairs and the index). */
int skim_greedy_reset(skim_ctx *ctx);

/* Influence oracle query (Section 5.1, Eq. unionest, Cohen-Kaplan union
 * estimator): estimate of Inf(S) = |union of R_u, u in S| / l from the
 * sketches of S.  seeds (host), n_seeds >= 0; duplicates allowed; the empty
 * set gives 0.  The sum is formed exactly in fixed point and rounded once, so
 * the result does not depend on summation order.  est_out (host).
 * With SKIM_RANKS_PERMUTATION a threshold position q (k-th smallest of a full
 * sketch) reads as the uniform rank q/(n*l-1), so each rank charged to it adds
 * (n*l-1)/q (Section 5.1's permutation version); with SKIM_RANKS_IC_MODEL the
 * estimate is the l -> infinity limit: n/q per rank, nothing for a rank whose
 * largest threshold belongs to a sketch that is not full, no division by l. */
int skim_oracle_query(skim_ctx *ctx, const uint32_t *seeds, uint32_t n_seeds, double *est_out);

/* Influence estimate of every single node from its own sketch (out[v], n
 * doubles; host memory, or device memory if out_on_device):
 *   SKIM_RANKS_UNIFORM: (k-1)/tau_v / l, tau_v = h * 2^-64 (Section 3);
 *   SKIM_RANKS_PERMUTATION: (1 + (k-1)(n*l-1)/q) / l, the estimator of
 *     Section 3.1 with T - 1 = q the k-th smallest position;
 *   SKIM_RANKS_IC_MODEL: n (k-1) / q (Section 3.2);
 * and |X_v| / l (0 in the IC model) when the sketch is not full.
 * Errors: SKIM_EINVAL, SKIM_ENOTBUILT. */
int skim_node_estimates(skim_ctx *ctx, double *out, int out_on_device);

/* Batched form of skim_oracle_query: q queries given in CSR form.
 * offsets[q+1] (host), seeds[offsets[q]] (host|device per on_device),
 * est_out[q] (host|device per on_device).  Each result is bitwise identical
 * to the single-query call. */
int skim_oracle_query_batch(skim_ctx *ctx, const uint64_t *offsets, uint32_t q,
                            const uint32_t *seeds, double *est_out, int on_device);

/* Counters of the last build / greedy call (see SKIM_STAT_* indices). */
#define SKIM_STAT_REV_VISITS 0      /* (node, rank) visits of reverse searches */
#define SKIM_STAT_REV_COINS 1       /* coins evaluated by reverse searches */
#define SKIM_STAT_INSERTIONS 2      /* sketch insertions (build) or commits (greedy) */
#define SKIM_STAT_FWD_VISITS 3      /* (node, instance) pairs covered by residual searches */
#define SKIM_STAT_FWD_COINS 4       /* coins evaluated by residual searches */
#define SKIM_STAT_BATCHES 5         /* rank batches */
#define SKIM_STAT_RANKS 6           /* ranks consumed */
#define SKIM_STAT_RETRIES 7         /* batches re-run with fewer lanes after a table overflow */
#define SKIM_STAT_REV_EDGES 8       /* edges scanned by reverse searches (all lanes of an item share one scan) */
#define SKIM_STAT_FWD_EDGES 9       /* edges scanned by residual searches */
#define SKIM_STAT_REQUEUES 10       /* searches resumed after a full work queue parked work */
#define SKIM_STAT_COUNT 11
int skim_get_stats(skim_ctx *ctx, uint64_t *out, uint32_t count);

/* Kernel timing with CUDA events on the context's stream (off by default).
 * When on, the device time of each launch group below is accumulated until
 * the next call with reset != 0.  Kinds (index into ms_out / launches_out):
 *   SKIM_K_REV   reverse searches (Algorithms 1 and 2, the batched BFS)
 *   SKIM_K_FWD   residual forward searches (Algorithm 1)
 *   SKIM_K_ACCEPT Algorithm 2 acceptance into the sketches
 *   SKIM_K_SORT  grouping of visit records by node (radix sort), emptying their table slots
 *   SKIM_K_STEP  SKIM per-node steps (first-to-k candidates, commits)
 *   SKIM_K_RANKS rank order of the n*l pairs
 *   SKIM_K_QUERY union-estimator queries
 *   SKIM_K_SETUP CSR construction and validation
 *   SKIM_K_INSTANCES generation of the live-edge instances (skim_instances)
 *   SKIM_K_SOURCES the sources of each batch of reverse searches (their first level)
 * Turning timing on creates a pool of 2048 CUDA events at once (so that no
 * event is created inside a timed bracket).  A bracket that holds a host
 * synchronisation (SKIM_K_STEP) also counts the host's share of that wait. */
#define SKIM_K_REV 0
#define SKIM_K_FWD 1
#define SKIM_K_ACCEPT 2
#define SKIM_K_SORT 3
#define SKIM_K_STEP 4
#define SKIM_K_RANKS 5
#define SKIM_K_QUERY 6
#define SKIM_K_SETUP 7
#define SKIM_K_INSTANCES 8
#define SKIM_K_SOURCES 9
#define SKIM_K_COUNT 10
int skim_set_timing(skim_ctx *ctx, int on);

/* Number of kernels this library has launched in the calling process since it
 * was loaded (all contexts).  out (host). */
int skim_kernel_launches(uint64_t *out);
int skim_kernel_times(skim_ctx *ctx, double *ms_out, uint64_t *launches_out, uint32_t count, int reset);

/* Bound of every device-side wait of this context's searches: a warp that
 * sees no progress for `ns` nanoseconds (default 2e9) gives up, every warp of
 * the search then returns, and the call reports SKIM_ETIMEOUT (the context
 * is then unusable; destroy it).  A short limit makes the waits give up on
 * purpose, which is how failure handling is tested.  Errors: SKIM_EINVAL
 * (null context, ns = 0). */
int skim_set_wait_limit_ns(skim_ctx *ctx, uint64_t ns);

/* Shape of a context: nodes n, sketch size k, instances l (host outputs). */
int skim_context_shape(skim_ctx *ctx, uint32_t *n, uint32_t *k, uint32_t *l);

/* ---- Serving: the influence oracle as a continuous-batching request loop ----
 * (queries of Section 5.1, Eq. unionest, over sketches resident on the GPU).
 * A server thread admits submitted seed sets into launch groups while
 * in-flight slots (max_inflight queries) and scratch memory (scratch_slots
 * hash-table slots of 16 bytes, split over `streams` streams; a query of |S|
 * seeds needs the next power of two >= 2|S|(k-1)+2) allow, and launches each
 * group on a free stream.  Groups on different streams run concurrently; a
 * request that arrives while others are on the GPU joins the next group as
 * soon as slots and memory free up.  Each result is bitwise identical to
 * skim_oracle_query on the same seeds.  The context's sketches must stay
 * built, and the context must not be used by other calls, until
 * skim_server_stop() returns.  Submit, poll and wait may be called from any
 * host thread.  Errors: SKIM_EINVAL, SKIM_ENOTBUILT, SKIM_ENOMEM; submit
 * returns SKIM_ERANGE for a query larger than one stream's scratch. */
typedef struct skim_server skim_server;
int skim_server_start(skim_ctx *ctx, uint32_t max_inflight, uint64_t scratch_slots, uint32_t streams,
                      skim_server **out);
/* Queue one query (seeds (host) are copied); *ticket identifies it. */
int skim_server_submit(skim_server *srv, const uint32_t *seeds, uint32_t n_seeds, uint64_t *ticket);
/* Non-blocking: *done = 1 and *est set once the result is ready (each
 * result is returned once). */
int skim_server_poll(skim_server *srv, uint64_t ticket, int *done, double *est);
/* Blocking with a timeout: SKIM_ETIMEOUT if the result is not ready in time. */
int skim_server_wait(skim_server *srv, uint64_t ticket, double *est, uint32_t timeout_ms);
/* Load generator: submit query j (seeds[offsets[j] .. offsets[j+1]), host) at
 * arrival_s[j] seconds after the call starts, from the calling thread, then
 * wait for all; latency_s[j] = completion time - submit time, est_out[j] the
 * estimate. */
int skim_server_replay(skim_server *srv, const double *arrival_s, const uint64_t *offsets, const uint32_t *seeds,
                       uint32_t q, double *latency_s, double *est_out);
/* Launch groups so far and the queries they held. */
int skim_server_stats(skim_server *srv, uint64_t *groups, uint64_t *queries);
/* Finish the queued work, stop the thread and free the server. */
int skim_server_stop(skim_server *srv);

/* Allocation-free influence query, for callers that cannot allocate device
 * memory (code that runs inside another framework's memory pool or under a
 * fixed memory budget, where a cudaMalloc is not allowed).  The paper has no
 * counterpart: it computes the same estimate as skim_oracle_query (Eq.
 * unionest, summed exactly and rounded once), but its scratch hash table is a
 * fixed 4 MiB array of static device memory that every GPU loading the
 * library holds until the process exits.  Nothing is allocated and nothing
 * is synchronised: the call is asynchronous on `stream` (a cudaStream_t, or
 * NULL).
 *   x_dev, len_dev  sketches in device memory, as skim_get_sketches lays them
 *                   out (n*k ranks row-major, n lengths), e.g. from
 *                   skim_sketch_pointers();
 *   rank_mode       SKIM_RANKS_* of the context the sketches came from: a
 *                   threshold h reads as in skim_oracle_query (uniform: 2^64/h
 *                   per rank, divided by l; permutation: (n*l-1)/h, divided
 *                   by l; IC model: n/h, nothing for a sketch that is not
 *                   full, l must be 1);
 *   seeds_dev       n_seeds node ids in device memory (duplicates allowed);
 *   est_dev         one double in device memory; receives the estimate, or a
 *                   quiet NaN if a seed id is >= n.
 * Limit: 2*n_seeds*(k-1)+2 <= 2^18 (n_seeds <= 2080 for k = 64); larger
 * queries return SKIM_ERANGE.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not use this entry after cudaDeviceReset() on that
 * device (the kept address would be stale).  All calls on a device share the
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  A CUDA error already
 * pending on the calling thread is left in place and reported as SKIM_ECUDA
 * without a launch.
 * Errors: SKIM_EINVAL (null pointer, k, l or rank_mode out of range),
 * SKIM_ERANGE, SKIM_ECUDA. */
int skim_union_estimate_static(const uint64_t *x_dev, const uint32_t *len_dev, uint32_t n, uint32_t k, uint32_t l,
                               uint32_t rank_mode, const uint32_t *seeds_dev, uint32_t n_seeds, double *est_dev,
                               void *stream);

int skim_destroy(skim_ctx *ctx);

/* The library keeps one stream-ordered device memory pool per device: blocks
 * that skim_destroy() frees stay reserved for the next context on that
 * device, so a context per graph or per request does not pay for cudaMalloc
 * and cudaFree of its scratch (several GB at R-MAT scale 20) each time.
 * skim_release_memory() hands every block that no live context holds back to
 * the device, on every device the library has used; live contexts are not
 * affected.  Thread-safe.
 * Errors: SKIM_ECUDA. */
int skim_release_memory(void);

const char *skim_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SKIM_H */

/*
 * skim_oracle.c -- plain, slow, single-threaded CPU oracle for SKIM
 * (Cohen, Delling, Pajor, Werneck, "Sketch-based Influence Maximization and
 * Computation: Scaling up with Guarantees", arXiv 1408.6282).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or table with the CUDA library: the hash, coin and rank definitions below
 * are written out here independently from their published definitions.
 *
 * What it computes (each function names the passage it follows):
 *   - ranks r(v,i) and live-edge coins of the binary IC model (Sections 2-3),
 *   - combined reachability sketches by the definition (Eq. combinedrs) and
 *     by Algorithm 2 (per-instance pruned searches, merged and trimmed),
 *   - SKIM, Algorithm 1, step by step, with the tie rules stated at skim(),
 *   - the Cohen-Kaplan union estimator (Eq. unionest) and the bottom-k
 *     estimator of the union (Section 5.1),
 *   - exact influence by forward BFS (Eq. InfbinaryIC),
 *   - structured permutation ranks (Section 3.1) for the sketches and SKIM,
 *     IC-model sketches (Section 3.2), and their estimators.
 *
 * Parity status: every function is pinned by tests against brute force on
 * tiny graphs, closed forms or invariants; none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* ------------------------------------------------------------------------ */
/* Hashes.  SplitMix64 (Steele, Lea, Flood 2014): output function fmix and   */
/* the stream x_t = fmix(s + t*GOLDEN).                                      */
/* ------------------------------------------------------------------------ */
static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

static uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Rank of node-instance pair (v,i): an independent uniform value per pair
 * (Section 3), here a 64-bit integer read as r / 2^64.  The map from pair
 * index v*l+i to rank is a bijection, so ranks never tie. */
uint64_t or_rank(uint64_t rank_key, uint32_t l, uint32_t v, uint32_t i) {
    return fmix(rank_key + GOLDEN * ((uint64_t)v * l + i));
}

/* Probability models (Section 6): 0 uniform p, 1 weighted cascade 1/indeg(head),
 * 2 trivalency (p in {0.1, 0.01, 0.001} by an edge hash).  An edge is live in
 * instance i iff its coin c <= tm1, where tm1 = floor(p * 2^64) - 1. */
static uint64_t uniform_tm1(double p) {
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)ldexp(p, 64) - 1u;
}

typedef struct {
    uint32_t n;
    uint64_t m;
    uint32_t l, k;
    int model;
    double p;
    uint64_t coin_key, rank_key, prob_key;
    uint64_t *fptr; uint32_t *fcol;   /* forward CSR: out-neighbours of u */
    uint64_t *rptr; uint32_t *rcol;   /* reverse CSR: in-neighbours of v  */
    uint64_t tm1_uniform;
    uint64_t tm1_class[3];
} graph_t;

static uint64_t edge_tm1(const graph_t *g, uint32_t u, uint32_t v) {
    if (g->model == 0) return g->tm1_uniform;
    if (g->model == 1) return UINT64_MAX / (g->rptr[v + 1] - g->rptr[v]);
    uint64_t cls = fmix(g->prob_key ^ (((uint64_t)u << 32) | v)) % 3u;
    return g->tm1_class[cls];
}

/* Live-edge coin for directed edge (u,v) in instance i: the (i+1)-th output of
 * the SplitMix64 stream whose state is fmix(coin_key ^ edge_id). */
static int live(const graph_t *g, uint32_t u, uint32_t v, uint64_t i) {
    uint64_t he = fmix(g->coin_key ^ (((uint64_t)u << 32) | v));
    uint64_t c = fmix(he + GOLDEN * (i + 1));
    return c <= edge_tm1(g, u, v);
}

int or_live(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
            int model, double p, uint64_t coin_key, uint64_t prob_key,
            uint32_t u, uint32_t v, uint32_t i);

static void graph_free(graph_t *g) {
    free(g->fptr); free(g->fcol); free(g->rptr); free(g->rcol);
    memset(g, 0, sizeof(*g));
}

/* Build both CSR directions from a canonical edge list (sorted by (src,dst),
 * no duplicates, no self-loops).  Rows of both directions end up sorted. */
static int graph_init(graph_t *g, uint32_t n, uint64_t m, const uint32_t *src,
                      const uint32_t *dst, uint32_t l, uint32_t k, int model,
                      double p, uint64_t coin_key, uint64_t rank_key, uint64_t prob_key) {
    memset(g, 0, sizeof(*g));
    if (n == 0 || l == 0 || k < 2 || model < 0 || model > 2) return OR_EINVAL;
    if (model == 0 && !(p > 0.0 && p <= 1.0)) return OR_EINVAL;
    g->n = n; g->m = m; g->l = l; g->k = k; g->model = model; g->p = p;
    g->coin_key = coin_key; g->rank_key = rank_key; g->prob_key = prob_key;
    g->tm1_uniform = model == 0 ? uniform_tm1(p) : 0;
    g->tm1_class[0] = uniform_tm1(0.1);
    g->tm1_class[1] = uniform_tm1(0.01);
    g->tm1_class[2] = uniform_tm1(0.001);
    g->fptr = calloc((size_t)n + 1, sizeof(uint64_t));
    g->rptr = calloc((size_t)n + 1, sizeof(uint64_t));
    g->fcol = malloc((m ? m : 1) * sizeof(uint32_t));
    g->rcol = malloc((m ? m : 1) * sizeof(uint32_t));
    if (!g->fptr || !g->rptr || !g->fcol || !g->rcol) { graph_free(g); return OR_ENOMEM; }
    for (uint64_t e = 0; e < m; e++) {
        if (src[e] >= n || dst[e] >= n || src[e] == dst[e]) { graph_free(g); return OR_EINVAL; }
        g->fptr[src[e] + 1]++;
        g->rptr[dst[e] + 1]++;
    }
    for (uint32_t v = 0; v < n; v++) { g->fptr[v + 1] += g->fptr[v]; g->rptr[v + 1] += g->rptr[v]; }
    uint64_t *fpos = malloc((size_t)n * sizeof(uint64_t));
    uint64_t *rpos = malloc((size_t)n * sizeof(uint64_t));
    if (!fpos || !rpos) { free(fpos); free(rpos); graph_free(g); return OR_ENOMEM; }
    memcpy(fpos, g->fptr, (size_t)n * sizeof(uint64_t));
    memcpy(rpos, g->rptr, (size_t)n * sizeof(uint64_t));
    /* edges arrive sorted by (src, dst): forward rows sorted by dst, and
     * reverse rows filled in increasing src order */
    for (uint64_t e = 0; e < m; e++) {
        g->fcol[fpos[src[e]]++] = dst[e];
        g->rcol[rpos[dst[e]]++] = src[e];
    }
    free(fpos); free(rpos);
    return OR_OK;
}

int or_live(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
            int model, double p, uint64_t coin_key, uint64_t prob_key,
            uint32_t u, uint32_t v, uint32_t i) {
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, 1, 2, model, p, coin_key, 0, prob_key);
    if (rc) return rc;
    int r = (model == 1 && g.rptr[v + 1] == g.rptr[v]) ? 0 : live(&g, u, v, i);
    graph_free(&g);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Small helpers                                                             */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

typedef struct { uint64_t key; uint32_t val; uint32_t pad; } kv_t;
static int cmp_kv(const void *a, const void *b) {
    uint64_t x = ((const kv_t *)a)->key, y = ((const kv_t *)b)->key;
    return x < y ? -1 : x > y;
}

/* Counters reported to callers (layout shared with the Python wrapper):
 *  [0] reverse expansions: node-instance pairs scanned and not pruned
 *  [1] reverse edge scans: sum of in-degrees over those expansions
 *  [2] sketch insertions
 *  [3] forward (residual) expansions
 *  [4] forward edge scans
 *  [5] ranks processed (BFS sources not skipped)
 *  [6] ranks consumed (rank cursor advance, skipped ones included)
 *  [7] index entries erased
 *  [8] live reverse edges: over the reverse expansions, the in-edges that are
 *      live in the expansion's instance (whether or not their tail is new)
 *  [9] live forward edges: the same over the forward expansions */
#define OR_NCOUNT 10

/* ------------------------------------------------------------------------ */
/* Eq. combinedrs by definition: X_u = bottom-k of the ranks of R_u, R_u    */
/* found by a forward BFS from u in every instance (Section 3).              */
/* ------------------------------------------------------------------------ */
int or_sketch_of_node(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                      uint32_t l, uint32_t k, int model, double p,
                      uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
                      uint32_t u, uint64_t *x_out, uint32_t *len_out, uint64_t *reach_out) {
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, l, k, model, p, coin_key, rank_key, prob_key);
    if (rc) return rc;
    if (u >= n) { graph_free(&g); return OR_EINVAL; }
    uint32_t *queue = malloc((size_t)n * sizeof(uint32_t));
    uint8_t *seen = malloc(n);
    uint64_t cap = 1024, cnt = 0;
    uint64_t *ranks = malloc(cap * sizeof(uint64_t));
    if (!queue || !seen || !ranks) { rc = OR_ENOMEM; goto done; }
    for (uint32_t i = 0; i < l; i++) {
        memset(seen, 0, n);
        uint32_t head = 0, tail = 0;
        queue[tail++] = u; seen[u] = 1;
        while (head < tail) {
            uint32_t v = queue[head++];
            if (cnt == cap) {
                cap *= 2;
                uint64_t *r2 = realloc(ranks, cap * sizeof(uint64_t));
                if (!r2) { rc = OR_ENOMEM; goto done; }
                ranks = r2;
            }
            ranks[cnt++] = or_rank(rank_key, l, v, i);
            for (uint64_t e = g.fptr[v]; e < g.fptr[v + 1]; e++) {
                uint32_t w = g.fcol[e];
                if (!seen[w] && live(&g, v, w, i)) { seen[w] = 1; queue[tail++] = w; }
            }
        }
    }
    qsort(ranks, cnt, sizeof(uint64_t), cmp_u64);
    *len_out = (uint32_t)(cnt < k ? cnt : k);
    for (uint32_t j = 0; j < *len_out; j++) x_out[j] = ranks[j];
    if (reach_out) *reach_out = cnt;
done:
    free(queue); free(seen); free(ranks);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Structured permutation ranks (Section 3.1).  Positions are 0-based (the    */
/* paper's permutation rank T is the position plus one).  Chunk c holds        */
/* positions c*n .. c*n + n - 1 and every node exactly once, ordered by the    */
/* key w(v,c) = fmix(K_w + GOLDEN*(c*n + v)), K_w = fmix(rank_key ^ PERM_SALT).*/
/* In the instance model the node's pair in chunk c is (v, sigma_v(c)), where  */
/* sigma_v lists node v's instances by increasing r(v,i): each chunk draws an  */
/* instance uniformly among those v has not used yet.  In the IC model         */
/* (Section 3.2) position t has a fresh instance of its own, numbered t.       */
/* ------------------------------------------------------------------------ */
static const uint64_t PERM_SALT = 0x7065726d75746531ULL;

static uint64_t perm_key(uint64_t rank_key) { return fmix(rank_key ^ PERM_SALT); }

/* nodes of chunk c in position order */
static void chunk_nodes(uint32_t n, uint64_t c, uint64_t kw, kv_t *buf, uint32_t *out) {
    for (uint32_t v = 0; v < n; v++) {
        buf[v].key = fmix(kw + GOLDEN * (c * n + v));
        buf[v].val = v;
    }
    qsort(buf, n, sizeof(kv_t), cmp_kv);
    for (uint32_t j = 0; j < n; j++) out[j] = buf[j].val;
}

/* pos_out[v*l + i] = position of pair (v,i) among all n*l */
int or_perm_positions(uint32_t n, uint32_t l, uint64_t rank_key, uint64_t *pos_out) {
    if (n == 0 || l == 0 || l > 255) return OR_EINVAL;
    kv_t *buf = malloc((size_t)(n > l ? n : l) * sizeof(kv_t));
    uint8_t *sigma = malloc((size_t)n * l);
    uint32_t *nodes = malloc((size_t)n * sizeof(uint32_t));
    if (!buf || !sigma || !nodes) { free(buf); free(sigma); free(nodes); return OR_ENOMEM; }
    for (uint32_t v = 0; v < n; v++) {
        for (uint32_t i = 0; i < l; i++) { buf[i].key = or_rank(rank_key, l, v, i); buf[i].val = i; }
        qsort(buf, l, sizeof(kv_t), cmp_kv);
        for (uint32_t c = 0; c < l; c++) sigma[(size_t)v * l + c] = (uint8_t)buf[c].val;
    }
    const uint64_t kw = perm_key(rank_key);
    for (uint32_t c = 0; c < l; c++) {
        chunk_nodes(n, c, kw, buf, nodes);
        for (uint32_t j = 0; j < n; j++) {
            uint32_t v = nodes[j];
            pos_out[(size_t)v * l + sigma[(size_t)v * l + c]] = (uint64_t)c * n + j;
        }
    }
    free(buf); free(sigma); free(nodes);
    return OR_OK;
}

/* node_out[t] = node at IC-model position t, for t < chunks * n */
int or_ic_nodes(uint32_t n, uint32_t chunks, uint64_t rank_key, uint32_t *node_out) {
    if (n == 0) return OR_EINVAL;
    kv_t *buf = malloc((size_t)n * sizeof(kv_t));
    if (!buf) return OR_ENOMEM;
    const uint64_t kw = perm_key(rank_key);
    for (uint32_t c = 0; c < chunks; c++) chunk_nodes(n, c, kw, buf, node_out + (size_t)c * n);
    free(buf);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: for each instance i, process the pairs (u,i) by increasing    */
/* rank; reverse BFS from u in G(i); a scanned node whose local sketch holds  */
/* k ranks is pruned, otherwise the rank joins its local sketch.  After the   */
/* instance, every local sketch is merged into the global one and trimmed to  */
/* k, then cleared (Section 5.2).                                             */
/* ------------------------------------------------------------------------ */
/* rank_mode 0: uniform 64-bit ranks r(v,i); 1: structured permutation
 * positions (every pair is processed; positions past min(k,l)*n simply never
 * survive the merge). */
int or_build_sketches_mode(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                           uint32_t l, uint32_t k, int model, double p,
                           uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
                           uint64_t *x_out, uint32_t *len_out, uint64_t *counters, int rank_mode) {
    if (rank_mode != 0 && rank_mode != 1) return OR_EINVAL;
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, l, k, model, p, coin_key, rank_key, prob_key);
    if (rc) return rc;
    uint64_t *pos = NULL;
    if (rank_mode == 1) {
        pos = malloc((size_t)n * l * sizeof(uint64_t));
        if (!pos) { graph_free(&g); return OR_ENOMEM; }
        rc = or_perm_positions(n, l, rank_key, pos);
        if (rc) { free(pos); graph_free(&g); return rc; }
    }
    uint64_t cnt[OR_NCOUNT] = {0};
    kv_t *order = malloc((size_t)n * sizeof(kv_t));
    uint64_t *local = malloc((size_t)n * k * sizeof(uint64_t));
    uint32_t *llen = calloc(n, sizeof(uint32_t));
    uint32_t *stamp = calloc(n, sizeof(uint32_t));
    uint32_t *queue = malloc((size_t)n * sizeof(uint32_t));
    uint64_t *merged = malloc((size_t)2 * k * sizeof(uint64_t));
    if (!order || !local || !llen || !stamp || !queue || !merged) { rc = OR_ENOMEM; goto done; }
    for (uint32_t v = 0; v < n; v++) len_out[v] = 0;
    uint32_t bfs_id = 0;
    for (uint32_t i = 0; i < l; i++) {
        /* pairs of instance i by increasing rank */
        for (uint32_t u = 0; u < n; u++) {
            order[u].key = pos ? pos[(size_t)u * l + i] : or_rank(rank_key, l, u, i);
            order[u].val = u;
        }
        qsort(order, n, sizeof(kv_t), cmp_kv);
        for (uint32_t t = 0; t < n; t++) {
            uint32_t u = order[t].val;
            uint64_t r = order[t].key;
            cnt[6]++;
            bfs_id++;
            if (bfs_id == 0) { memset(stamp, 0, (size_t)n * sizeof(uint32_t)); bfs_id = 1; }
            uint32_t head = 0, tail = 0;
            queue[tail++] = u; stamp[u] = bfs_id;
            int any = 0;
            while (head < tail) {
                uint32_t v = queue[head++];
                if (llen[v] == k) continue;                 /* prune */
                local[(size_t)v * k + llen[v]++] = r;       /* ranks arrive increasing */
                any = 1;
                cnt[0]++; cnt[2]++;
                cnt[1] += g.rptr[v + 1] - g.rptr[v];
                for (uint64_t e = g.rptr[v]; e < g.rptr[v + 1]; e++) {
                    uint32_t w = g.rcol[e];                 /* in-edge w -> v */
                    if (!live(&g, w, v, i)) continue;
                    cnt[8]++;
                    if (stamp[w] != bfs_id) { stamp[w] = bfs_id; queue[tail++] = w; }
                }
            }
            if (any) cnt[5]++;
        }
        /* merge the local sketches of instance i into the global ones */
        for (uint32_t v = 0; v < n; v++) {
            uint32_t a = 0, b = 0, o = 0, la = len_out[v], lb = llen[v];
            uint64_t *xa = x_out + (size_t)v * k, *xb = local + (size_t)v * k;
            while (o < k && (a < la || b < lb)) {
                if (b >= lb || (a < la && xa[a] < xb[b])) merged[o++] = xa[a++];
                else merged[o++] = xb[b++];
            }
            memcpy(xa, merged, o * sizeof(uint64_t));
            len_out[v] = o;
            llen[v] = 0;
        }
    }
    if (counters) memcpy(counters, cnt, sizeof(cnt));
done:
    free(order); free(local); free(llen); free(stamp); free(queue); free(merged); free(pos);
    graph_free(&g);
    return rc;
}

int or_build_sketches(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                      uint32_t l, uint32_t k, int model, double p,
                      uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
                      uint64_t *x_out, uint32_t *len_out, uint64_t *counters) {
    return or_build_sketches_mode(n, m, src, dst, l, k, model, p, coin_key, rank_key, prob_key,
                                  x_out, len_out, counters, 0);
}

/* ------------------------------------------------------------------------ */
/* IC-model sketches (Section 3.2): the limit of infinitely many instances.   */
/* Position t (t < k*n; every node reaches itself, so after k chunks each     */
/* sketch is full) has its own instance G_t; its rank t joins the sketch of    */
/* every node that reaches node(t) in G_t, while that sketch has fewer than k  */
/* entries.  Positions arrive in increasing order, so sketches stay sorted.   */
/* No search is pruned: a node that is full in G_t says nothing about its     */
/* in-neighbours in G_t.                                                      */
/* ------------------------------------------------------------------------ */
int or_build_ic_sketches(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                         uint32_t k, int model, double p,
                         uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
                         uint64_t *x_out, uint32_t *len_out, uint64_t *counters) {
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, 1, k, model, p, coin_key, rank_key, prob_key);
    if (rc) return rc;
    uint64_t cnt[OR_NCOUNT] = {0};
    const uint64_t npos = (uint64_t)k * n;
    uint32_t *node = malloc(npos * sizeof(uint32_t));
    uint32_t *stamp = calloc(n, sizeof(uint32_t));
    uint32_t *queue = malloc((size_t)n * sizeof(uint32_t));
    if (!node || !stamp || !queue) { rc = OR_ENOMEM; goto done; }
    rc = or_ic_nodes(n, k, rank_key, node);
    if (rc) goto done;
    for (uint32_t v = 0; v < n; v++) len_out[v] = 0;
    uint32_t bfs_id = 0;
    for (uint64_t t = 0; t < npos; t++) {
        cnt[5]++; cnt[6]++;
        bfs_id++;
        if (bfs_id == 0) { memset(stamp, 0, (size_t)n * sizeof(uint32_t)); bfs_id = 1; }
        uint32_t head = 0, tail = 0;
        queue[tail++] = node[t]; stamp[node[t]] = bfs_id;
        while (head < tail) {
            uint32_t v = queue[head++];
            if (len_out[v] < k) { x_out[(size_t)v * k + len_out[v]++] = t; cnt[2]++; }
            cnt[0]++;
            cnt[1] += g.rptr[v + 1] - g.rptr[v];
            for (uint64_t e = g.rptr[v]; e < g.rptr[v + 1]; e++) {
                uint32_t w = g.rcol[e];
                if (!live(&g, w, v, t)) continue;
                cnt[8]++;
                if (stamp[w] != bfs_id) { stamp[w] = bfs_id; queue[tail++] = w; }
            }
        }
    }
    if (counters) memcpy(counters, cnt, sizeof(cnt));
done:
    free(node); free(stamp); free(queue);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exact influence (Eq. InfbinaryIC): sum over instances of the number of     */
/* nodes reachable from S, i.e. |union of R_u, u in S| as an integer.         */
/* ------------------------------------------------------------------------ */
int or_exact_coverage(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                      uint32_t l, int model, double p, uint64_t coin_key, uint64_t prob_key,
                      const uint32_t *seeds, uint32_t s, uint64_t *prefix_out) {
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, l, 2, model, p, coin_key, 0, prob_key);
    if (rc) return rc;
    uint8_t *cov = calloc((size_t)n * l, 1);
    uint32_t *queue = malloc((size_t)n * sizeof(uint32_t));
    if (!cov || !queue) { rc = OR_ENOMEM; goto done; }
    uint64_t total = 0;
    /* prefix_out[j] = coverage of seeds[0..j] */
    for (uint32_t j = 0; j < s; j++) {
        uint32_t x = seeds[j];
        if (x >= n) { rc = OR_EINVAL; goto done; }
        for (uint32_t i = 0; i < l; i++) {
            uint8_t *c = cov + (size_t)i * n;
            if (c[x]) continue;
            uint32_t head = 0, tail = 0;
            queue[tail++] = x; c[x] = 1; total++;
            while (head < tail) {
                uint32_t v = queue[head++];
                for (uint64_t e = g.fptr[v]; e < g.fptr[v + 1]; e++) {
                    uint32_t w = g.fcol[e];
                    if (!c[w] && live(&g, v, w, i)) { c[w] = 1; total++; queue[tail++] = w; }
                }
            }
        }
        if (prefix_out) prefix_out[j] = total;
    }
done:
    free(cov); free(queue);
    graph_free(&g);
    return rc;
}

/* Sort records of all n*l pairs by rank: 12 bytes each (packed) so that the
 * largest runs fit in host memory. */
typedef struct __attribute__((packed)) { uint64_t key; uint32_t val; } kv12_t;
static int cmp_kv12(const void *a, const void *b) {
    uint64_t x = ((const kv12_t *)a)->key, y = ((const kv12_t *)b)->key;
    return x < y ? -1 : x > y;
}

/* ------------------------------------------------------------------------ */
/* SKIM, Algorithm 1 (Section 4), sequential.  Readings where the paper is    */
/* silent or garbled:                                                         */
/*  - the skip test before a search is on the source pair: covered[u,i]       */
/*    (the text prints covered[v,i] with v unbound; Section 4 says covered    */
/*    pairs are skipped);                                                     */
/*  - the search of the rank that first fills a sketch is completed and the   */
/*    seed is the smallest node id among nodes whose size reached k in it     */
/*    (all share the same estimate; the residual erases that rank anyway);    */
/*  - when the ranks run out: argmax size, ties to the smallest id; if every  */
/*    size is 0 (everything covered) the smallest id not yet chosen;          */
/*  - the rank cursor resumes after the rank that produced the seed.          */
/* Outputs seeds[j] and the integer marginal coverage cov[j] = l * I_j.       */
/* ------------------------------------------------------------------------ */
int or_skim_mode(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                 uint32_t l, uint32_t k, int model, double p,
                 uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
                 uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out,
                 uint32_t *size_out, uint64_t *counters,
                 uint64_t *tau_out, int32_t *kprime_out, int rank_mode) {
    if (rank_mode != 0 && rank_mode != 1) return OR_EINVAL;
    graph_t g;
    int rc = graph_init(&g, n, m, src, dst, l, k, model, p, coin_key, rank_key, prob_key);
    if (rc) return rc;
    if (n_seeds > n) { graph_free(&g); return OR_EINVAL; }
    uint64_t nl = (uint64_t)n * l;
    uint64_t cnt[OR_NCOUNT] = {0};
    kv12_t *order = malloc(nl * sizeof(kv12_t));
    uint8_t *covered = calloc(nl, 1);           /* covered[u*l + i] */
    uint32_t *size = calloc(n, sizeof(uint32_t));
    uint32_t *stamp = calloc(n, sizeof(uint32_t));
    uint32_t *queue = malloc((size_t)n * sizeof(uint32_t));
    uint8_t *chosen = calloc(n, 1);
    /* index: map from a processed pair to the list of nodes whose partial
     * sketch holds its rank.  Keys are pair ids < n*l, so the map is
     * addressed directly: list of pair p = nodes[ix_start[p] .. + ix_len[p]),
     * ix_len[p] = 0 for a pair with no entry (never processed, or erased). */
    uint64_t *ix_start = malloc(nl * sizeof(uint64_t));
    uint32_t *ix_len = calloc(nl, sizeof(uint32_t));
    uint64_t ncap = 1 << 20, nused = 0;
    uint32_t *nodes = malloc(ncap * sizeof(uint32_t));
    if (!order || !covered || !size || !stamp || !queue || !chosen || !ix_start || !ix_len || !nodes) {
        rc = OR_ENOMEM;
        goto done;
    }

    /* "shuffle the nl pairs": increasing rank order (uniform ranks, or the
     * structured permutation's positions, Section 3.1) */
    if (rank_mode == 1) {
        uint64_t *pos = malloc(nl * sizeof(uint64_t));
        if (!pos) { rc = OR_ENOMEM; goto done; }
        rc = or_perm_positions(n, l, rank_key, pos);
        for (uint64_t x = 0; x < nl && !rc; x++) { order[x].key = pos[x]; order[x].val = (uint32_t)x; }
        free(pos);
        if (rc) goto done;
    } else {
        for (uint64_t x = 0; x < nl; x++) {
            order[x].key = or_rank(rank_key, l, (uint32_t)(x / l), (uint32_t)(x % l));
            order[x].val = (uint32_t)x;
        }
    }
    qsort(order, nl, sizeof(kv12_t), cmp_kv12);

    uint64_t rank = 0;
    uint32_t bfs_id = 0;
    for (uint32_t sidx = 0; sidx < n_seeds; sidx++) {
        int64_t x = -1;
        /* build sketches until a size reaches k */
        while (rank < nl && x < 0) {
            uint64_t pair = order[rank].val;
            rank++;
            cnt[6]++;
            uint32_t u = (uint32_t)(pair / l), i = (uint32_t)(pair % l);
            if (covered[pair]) continue;
            cnt[5]++;
            ix_start[pair] = nused;
            ix_len[pair] = 0;
            bfs_id++;
            if (bfs_id == 0) { memset(stamp, 0, (size_t)n * sizeof(uint32_t)); bfs_id = 1; }
            uint32_t head = 0, tail = 0;
            queue[tail++] = u; stamp[u] = bfs_id;
            while (head < tail) {
                uint32_t v = queue[head++];
                size[v]++;
                if (nused == ncap) {
                    ncap += ncap / 2;
                    uint32_t *n2 = realloc(nodes, ncap * sizeof(uint32_t));
                    if (!n2) { rc = OR_ENOMEM; goto done; }
                    nodes = n2;
                }
                nodes[nused++] = v; ix_len[pair]++;
                cnt[0]++; cnt[2]++;
                if (size[v] == k && (x < 0 || v < (uint32_t)x)) x = v;
                cnt[1] += g.rptr[v + 1] - g.rptr[v];
                for (uint64_t e = g.rptr[v]; e < g.rptr[v + 1]; e++) {
                    uint32_t w = g.rcol[e];
                    if (!live(&g, w, v, i)) continue;
                    cnt[8]++;
                    if (stamp[w] != bfs_id) { stamp[w] = bfs_id; queue[tail++] = w; }
                }
            }
        }
        if (x >= 0) {
            /* Section 4.3.2 (adaptive error estimation): the threshold rank of
             * this iteration is the rank whose search stopped, and k' is the
             * largest sketch size among the other nodes once that rank is
             * taken out again (it is not part of any sketch for this count):
             * size[v] minus one for every v its search visited (stamp). */
            if (tau_out) tau_out[sidx] = order[rank - 1].key;
            if (kprime_out) {
                int32_t kp = 0;
                for (uint32_t v = 0; v < n; v++) {
                    if (v == (uint32_t)x) continue;
                    int32_t sz = (int32_t)size[v] - (stamp[v] == bfs_id ? 1 : 0);
                    if (sz > kp) kp = sz;
                }
                kprime_out[sidx] = kp;
            }
        }
        if (x < 0) {
            /* selection from exact residual counts: no estimation error */
            if (tau_out) tau_out[sidx] = 0;
            if (kprime_out) kprime_out[sidx] = -1;
            /* ranks exhausted: node with the largest partial sketch */
            uint32_t best = 0;
            for (uint32_t v = 1; v < n; v++) if (size[v] > size[best]) best = v;
            if (size[best] == 0) {
                best = 0;
                while (best < n && chosen[best]) best++;
            }
            x = best;
        }
        /* residual problem: forward BFS from x in every instance */
        uint64_t ix_cov = 0;
        for (uint32_t i = 0; i < l; i++) {
            if (covered[(uint64_t)x * l + i]) continue;
            uint32_t head = 0, tail = 0;
            queue[tail++] = (uint32_t)x; covered[(uint64_t)x * l + i] = 1;
            while (head < tail) {
                uint32_t v = queue[head++];
                ix_cov++;
                cnt[3]++;
                uint64_t pair = (uint64_t)v * l + i;
                if (ix_len[pair]) {
                    for (uint32_t t = 0; t < ix_len[pair]; t++) size[nodes[ix_start[pair] + t]]--;
                    cnt[7] += ix_len[pair];
                    ix_len[pair] = 0;                   /* erase */
                }
                cnt[4] += g.fptr[v + 1] - g.fptr[v];
                for (uint64_t e = g.fptr[v]; e < g.fptr[v + 1]; e++) {
                    uint32_t w = g.fcol[e];
                    uint64_t pw = (uint64_t)w * l + i;
                    if (!live(&g, v, w, i)) continue;
                    cnt[9]++;
                    if (!covered[pw]) { covered[pw] = 1; queue[tail++] = w; }
                }
            }
        }
        chosen[x] = 1;
        seeds_out[sidx] = (uint32_t)x;
        cov_out[sidx] = ix_cov;
    }
    if (size_out) memcpy(size_out, size, (size_t)n * sizeof(uint32_t));
    if (counters) memcpy(counters, cnt, sizeof(cnt));
done:
    free(order); free(covered); free(size); free(stamp); free(queue); free(chosen);
    free(ix_start); free(ix_len); free(nodes);
    graph_free(&g);
    return rc;
}

int or_skim(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
            uint32_t l, uint32_t k, int model, double p,
            uint64_t coin_key, uint64_t rank_key, uint64_t prob_key,
            uint32_t n_seeds, uint32_t *seeds_out, uint64_t *cov_out,
            uint32_t *size_out, uint64_t *counters,
            uint64_t *tau_out, int32_t *kprime_out) {
    return or_skim_mode(n, m, src, dst, l, k, model, p, coin_key, rank_key, prob_key, n_seeds, seeds_out,
                        cov_out, size_out, counters, tau_out, kprime_out, 0);
}

/* ------------------------------------------------------------------------ */
/* Influence estimation from sketches (Section 5.1).                          */
/* Sketches are given as rows of k slots with lengths; a rank h reads as the */
/* real h * 2^-64 (rounded to nearest double).  tau_u = k-th smallest if the  */
/* sketch is full, else 1.                                                    */
/* ------------------------------------------------------------------------ */
static double tau_of(const uint64_t *x, uint32_t len, uint32_t k) {
    return len == k ? ldexp((double)x[k - 1], -64) : 1.0;
}

typedef struct { double tau; uint32_t node; uint32_t pos; } tsort_t;
static int cmp_tau_desc(const void *a, const void *b) {
    double x = ((const tsort_t *)a)->tau, y = ((const tsort_t *)b)->tau;
    if (x != y) return x > y ? -1 : 1;
    uint32_t p = ((const tsort_t *)a)->pos, q = ((const tsort_t *)b)->pos;
    return p < q ? -1 : p > q;
}

/* Eq. unionest (Cohen-Kaplan): sum over distinct ranks z in the union of
 * X_v minus {tau_v} of 1 / max{tau_u : z in X_u minus {tau_u}}; computed as
 * the paper describes: sort the sketches by decreasing threshold and charge
 * each distinct rank to the first sketch that holds it.  Returns the
 * influence estimate, i.e. the union estimate divided by l. */
int or_union_estimate(const uint64_t *x, const uint32_t *len, uint32_t n, uint32_t k,
                      uint32_t l, const uint32_t *seeds, uint32_t s, double *est_out) {
    if (s == 0) { *est_out = 0.0; return OR_OK; }
    tsort_t *ts = malloc((size_t)s * sizeof(tsort_t));
    uint64_t cap = 1; while (cap < 2ull * s * k + 2) cap <<= 1;
    uint64_t *seen = calloc(cap, sizeof(uint64_t));   /* z+1, 0 empty */
    if (!ts || !seen) { free(ts); free(seen); return OR_ENOMEM; }
    for (uint32_t j = 0; j < s; j++) {
        if (seeds[j] >= n) { free(ts); free(seen); return OR_EINVAL; }
        ts[j].node = seeds[j]; ts[j].pos = j;
        ts[j].tau = tau_of(x + (size_t)seeds[j] * k, len[seeds[j]], k);
    }
    qsort(ts, s, sizeof(tsort_t), cmp_tau_desc);
    double sum = 0.0;
    for (uint32_t j = 0; j < s; j++) {
        uint32_t u = ts[j].node, lu = len[u];
        const uint64_t *xu = x + (size_t)u * k;
        uint32_t cnt = lu == k ? k - 1 : lu;           /* X_u minus {tau_u} */
        for (uint32_t t = 0; t < cnt; t++) {
            uint64_t z = xu[t];
            uint64_t h = fmix(z) & (cap - 1);
            int fresh = 1;
            while (seen[h]) {
                if (seen[h] == z + 1) { fresh = 0; break; }
                h = (h + 1) & (cap - 1);
            }
            if (fresh) { seen[h] = z + 1; sum += 1.0 / ts[j].tau; }
        }
    }
    *est_out = sum / (double)l;
    free(ts); free(seen);
    return OR_OK;
}

/* Bottom-k sketch of the union (Section 5.1): tau = k-th smallest of the union
 * of the sketches; estimate (k-1)/tau, or the exact count |union| when it has
 * fewer than k elements; divided by l. */
int or_bottomk_union_estimate(const uint64_t *x, const uint32_t *len, uint32_t n, uint32_t k,
                              uint32_t l, const uint32_t *seeds, uint32_t s, double *est_out) {
    uint64_t tot = 0;
    for (uint32_t j = 0; j < s; j++) { if (seeds[j] >= n) return OR_EINVAL; tot += len[seeds[j]]; }
    uint64_t *all = malloc((tot ? tot : 1) * sizeof(uint64_t));
    if (!all) return OR_ENOMEM;
    uint64_t c = 0;
    for (uint32_t j = 0; j < s; j++)
        for (uint32_t t = 0; t < len[seeds[j]]; t++) all[c++] = x[(size_t)seeds[j] * k + t];
    qsort(all, c, sizeof(uint64_t), cmp_u64);
    uint64_t d = 0;
    for (uint64_t t = 0; t < c; t++) if (t == 0 || all[t] != all[t - 1]) all[d++] = all[t];
    double est;
    if (d < k) est = (double)d;
    else est = (double)(k - 1) / ldexp((double)all[k - 1], -64);
    free(all);
    *est_out = est / (double)l;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Estimators for permutation ranks (Sections 3.1, 3.2 and 5.1).             */
/* A sketch holds positions; a full sketch's threshold is its k-th smallest   */
/* position, T - 1 in the paper's 1-based numbering.                          */
/*  rank_mode 1 (D = n*l pairs): the union estimator of Eq. unionest reads    */
/*    the threshold position q as the uniform rank q / (D - 1), so a rank      */
/*    charged to it adds (D - 1) / q; a sketch that is not full has           */
/*    threshold 1 and adds 1 per rank; the sum is divided by l.              */
/*  rank_mode 2 (IC model): the limit l -> infinity of the same: a rank       */
/*    charged to threshold q adds n / q, and one charged to a sketch that is  */
/*    not full adds nothing.                                                  */
/* Thresholds are compared as integers (not full = larger than any).          */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t thr; uint32_t node; uint32_t pos; } qsort_t;
static int cmp_thr_desc(const void *a, const void *b) {
    uint64_t x = ((const qsort_t *)a)->thr, y = ((const qsort_t *)b)->thr;
    if (x != y) return x > y ? -1 : 1;
    uint32_t p = ((const qsort_t *)a)->pos, q = ((const qsort_t *)b)->pos;
    return p < q ? -1 : p > q;
}

static double perm_term(uint64_t thr, int rank_mode, uint32_t n, uint32_t l) {
    if (thr == UINT64_MAX) return rank_mode == 2 ? 0.0 : 1.0;
    if (rank_mode == 2) return (double)n / (double)thr;
    return (double)((uint64_t)n * l - 1) / (double)thr;
}

int or_union_estimate_mode(const uint64_t *x, const uint32_t *len, uint32_t n, uint32_t k,
                           uint32_t l, const uint32_t *seeds, uint32_t s, int rank_mode, double *est_out) {
    if (rank_mode == 0) return or_union_estimate(x, len, n, k, l, seeds, s, est_out);
    if (rank_mode != 1 && rank_mode != 2) return OR_EINVAL;
    if (s == 0) { *est_out = 0.0; return OR_OK; }
    qsort_t *ts = malloc((size_t)s * sizeof(qsort_t));
    uint64_t cap = 1; while (cap < 2ull * s * k + 2) cap <<= 1;
    uint64_t *seen = calloc(cap, sizeof(uint64_t));   /* z+1, 0 empty */
    if (!ts || !seen) { free(ts); free(seen); return OR_ENOMEM; }
    for (uint32_t j = 0; j < s; j++) {
        if (seeds[j] >= n) { free(ts); free(seen); return OR_EINVAL; }
        ts[j].node = seeds[j]; ts[j].pos = j;
        ts[j].thr = len[seeds[j]] == k ? x[(size_t)seeds[j] * k + k - 1] : UINT64_MAX;
    }
    qsort(ts, s, sizeof(qsort_t), cmp_thr_desc);
    double sum = 0.0;
    for (uint32_t j = 0; j < s; j++) {
        uint32_t u = ts[j].node, lu = len[u];
        const uint64_t *xu = x + (size_t)u * k;
        uint32_t cnt = lu == k ? k - 1 : lu;
        const double term = perm_term(ts[j].thr, rank_mode, n, l);
        for (uint32_t t = 0; t < cnt; t++) {
            uint64_t z = xu[t];
            uint64_t h = fmix(z) & (cap - 1);
            int fresh = 1;
            while (seen[h]) {
                if (seen[h] == z + 1) { fresh = 0; break; }
                h = (h + 1) & (cap - 1);
            }
            if (fresh) { seen[h] = z + 1; sum += term; }
        }
    }
    *est_out = rank_mode == 2 ? sum : sum / (double)l;
    free(ts); free(seen);
    return OR_OK;
}

/* Influence estimate of every single node from its own sketch:
 *  rank_mode 0: (k - 1) / tau_u with tau_u = h * 2^-64 (Section 3), or |X_u|
 *    when the sketch is not full; divided by l.
 *  rank_mode 1: the unbiased permutation estimator 1 + (k-1)(D-1)/(T-1)
 *    (Section 3.1), T - 1 = the k-th smallest position, or |X_u| when not
 *    full; divided by l.
 *  rank_mode 2: n (k - 1) / (T - 1) (Section 3.2); 0 when not full. */
int or_node_estimates(const uint64_t *x, const uint32_t *len, uint32_t n, uint32_t k,
                      uint32_t l, int rank_mode, double *out) {
    if (rank_mode < 0 || rank_mode > 2) return OR_EINVAL;
    for (uint32_t u = 0; u < n; u++) {
        const uint32_t lu = len[u];
        double e;
        if (lu < k) {
            e = rank_mode == 2 ? 0.0 : (double)lu / (double)l;
        } else {
            const uint64_t q = x[(size_t)u * k + k - 1];
            if (rank_mode == 0) e = (double)(k - 1) / ldexp((double)q, -64) / (double)l;
            else if (rank_mode == 1)
                e = (1.0 + (double)(k - 1) * (double)((uint64_t)n * l - 1) / (double)q) / (double)l;
            else e = (double)n * (double)(k - 1) / (double)q;
        }
        out[u] = e;
    }
    return OR_OK;
}

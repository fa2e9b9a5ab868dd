/*
 * Betweenness-centrality ORACLE — test infrastructure only.
 *
 * Plain, sequential, obviously-correct CPU code that the CUDA path is checked against.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
 * load it; the product library never links, loads or calls it, and the two share no
 * source, header, table or helper.
 *
 * What it computes (Vella, Carbone, Bernaschi, "Algorithms and Heuristics for Scalable
 * Betweenness Centrality Computation on Multi-GPU Systems"):
 *   - Brandes' algorithm, Alg. 1 (Sec. 2): per source s a FIFO BFS that counts shortest
 *     paths sigma, pushing every dequeued vertex on a stack S; then S is popped and each
 *     popped w pushes sigma[v]/sigma[w] * (1 + delta[w]) to every predecessor v
 *     (Eq. 2), and BC[w] += delta[w] for w != s (Eq. 3).  Predecessors are not stored:
 *     v is a predecessor of w iff (v, w) is an edge and d[v] = d[w] - 1 (the
 *     predecessor-free formulation of Sec. 3.2).  Alg. 1 pops "v" but then loops over
 *     Pred[w]; the popped vertex is read as w.
 *   - the 1-degree variant, Eq. 3 / Eq. 4 (Sec. 2.1) and Alg. 6 (Sec. 3.4.1): a leaf u
 *     (deg(u) = 1) whose neighbour v has deg(v) >= 2 is removed, omega[v] counts the
 *     removed leaves of v; on the residual graph delta uses (1 + delta[w] + omega[w]),
 *     every contribution of source s is weighted by (omega[s] + 1), and s receives the
 *     deferred leaf term omega[s] * (2 n_s - omega[s] - 3), n_s = sum over the vertices
 *     reached from s of (1 + omega[v]) (Sec. 3.4.1).  Eq. 3 writes the term with the
 *     incremented omega; the pre-increment reading above is the one that gives (n-1)(n-2)
 *     on a star.  Only one removal round is made (Sec. 3.4.1 footnote 1).
 *
 * Ordered-pair convention: every source is a BFS root, so each unordered pair is counted
 * from both ends (the factor 2 of Eq. 3); results are twice the unordered values.
 *
 * Number formats.  sigma64 is the exact path count modulo 2^64 with a sticky per-vertex
 * overflow flag (set by a carry out of any addition, or inherited from a predecessor).
 * sigmaL, delta and BC are long double: the grid workload reaches sigma ~ 2^1730, past
 * the fp64 range, and long double has a 15-bit exponent on both x86-64 (80-bit) and
 * AArch64 (binary128).  BC is returned as double.
 */
#include <float.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

_Static_assert(LDBL_MAX_EXP >= 16384, "oracle needs a long double with a 15-bit exponent");

typedef struct {
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col_idx;
} ograph;

typedef struct {
    int32_t *depth;
    uint64_t *sigma;
    uint8_t *ovf;
    long double *sigmaL;
    long double *delta;
    int32_t *queue; /* BFS queue; also the stack S of Alg. 1 (read backwards) */
} owork;

static int owork_alloc(owork *w, int32_t n) {
    size_t N = (size_t)(n > 0 ? n : 1);
    w->depth = (int32_t *)malloc(N * sizeof(int32_t));
    w->sigma = (uint64_t *)malloc(N * sizeof(uint64_t));
    w->ovf = (uint8_t *)malloc(N);
    w->sigmaL = (long double *)malloc(N * sizeof(long double));
    w->delta = (long double *)malloc(N * sizeof(long double));
    w->queue = (int32_t *)malloc(N * sizeof(int32_t));
    if (!w->depth || !w->sigma || !w->ovf || !w->sigmaL || !w->delta || !w->queue) return -1;
    for (int32_t v = 0; v < n; v++) {
        w->depth[v] = -1;
        w->sigma[v] = 0;
        w->ovf[v] = 0;
        w->sigmaL[v] = 0.0L;
        w->delta[v] = 0.0L;
    }
    return 0;
}

static void owork_free(owork *w) {
    free(w->depth); free(w->sigma); free(w->ovf);
    free(w->sigmaL); free(w->delta); free(w->queue);
}

/* Shortest-path counting from s (Alg. 1, BFS part).  Returns the number of reached
 * vertices; w->queue[0..count) holds them in BFS (non-decreasing depth) order. */
static int32_t o_bfs(const ograph *g, owork *w, int32_t s) {
    int32_t head = 0, tail = 0;
    w->depth[s] = 0;
    w->sigma[s] = 1;
    w->sigmaL[s] = 1.0L;
    w->queue[tail++] = s;
    while (head < tail) {
        int32_t v = w->queue[head++];
        int32_t dv = w->depth[v];
        for (int32_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
            int32_t x = g->col_idx[e];
            if (w->depth[x] < 0) {            /* first discovery: enqueue */
                w->depth[x] = dv + 1;
                w->queue[tail++] = x;
            }
            if (w->depth[x] == dv + 1) {      /* v is a predecessor of x */
                uint64_t before = w->sigma[x];
                w->sigma[x] = before + w->sigma[v];
                if (w->sigma[x] < before) w->ovf[x] = 1;
                w->ovf[x] |= w->ovf[v];
                w->sigmaL[x] += w->sigmaL[v];
            }
        }
    }
    return tail;
}

static void o_reset(owork *w, int32_t count) {
    for (int32_t i = 0; i < count; i++) {
        int32_t v = w->queue[i];
        w->depth[v] = -1;
        w->sigma[v] = 0;
        w->ovf[v] = 0;
        w->sigmaL[v] = 0.0L;
        w->delta[v] = 0.0L;
    }
}

/* Dependency accumulation (Alg. 1, stack part, with Eq. 4's omega terms). */
static void o_accumulate(const ograph *g, owork *w, int32_t s, int32_t count,
                         const int32_t *omega, long double *bc) {
    long double ws = omega ? (long double)omega[s] + 1.0L : 1.0L;
    for (int32_t i = count - 1; i >= 0; i--) {
        int32_t x = w->queue[i];             /* pop x from S */
        int32_t dx = w->depth[x];
        long double coef = (1.0L + w->delta[x] + (omega ? (long double)omega[x] : 0.0L)) / w->sigmaL[x];
        for (int32_t e = g->row_ptr[x]; e < g->row_ptr[x + 1]; e++) {
            int32_t v = g->col_idx[e];
            if (w->depth[v] == dx - 1)       /* v in Pred[x] */
                w->delta[v] += w->sigmaL[v] * coef;
        }
        if (x != s) bc[x] += ws * w->delta[x];
    }
    if (omega && omega[s] > 0) {
        long double ns = 0.0L;               /* component size incl. removed leaves */
        for (int32_t i = 0; i < count; i++) ns += 1.0L + (long double)omega[w->queue[i]];
        long double om = (long double)omega[s];
        bc[s] += om * (2.0L * ns - om - 3.0L);
    }
}

/* ---------------------------------------------------------------- public entry points */

/* Single-source shortest-path counts: depth (-1 = unreached), sigma mod 2^64, overflow
 * flag, and optionally the long-double sigma.  Returns the number of reached vertices. */
int32_t oracle_sssp(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t s,
                    int32_t *depth, uint64_t *sigma, uint8_t *ovf, long double *sigmaL) {
    ograph g = {n, row_ptr, col_idx};
    owork w;
    if (s < 0 || s >= n) return -1;
    if (owork_alloc(&w, n)) { owork_free(&w); return -2; }
    int32_t count = o_bfs(&g, &w, s);
    for (int32_t v = 0; v < n; v++) {
        depth[v] = w.depth[v];
        sigma[v] = w.sigma[v];
        ovf[v] = w.ovf[v];
        if (sigmaL) sigmaL[v] = w.sigmaL[v];
    }
    owork_free(&w);
    return count;
}

typedef struct {
    const ograph *g;
    const int32_t *src;
    int64_t lo, hi;
    const int32_t *omega;
    long double *bc;
    int status;
} ojob;

static void *o_worker(void *arg) {
    ojob *j = (ojob *)arg;
    owork w;
    if (owork_alloc(&w, j->g->n)) { owork_free(&w); j->status = -2; return NULL; }
    for (int64_t i = j->lo; i < j->hi; i++) {
        int32_t s = j->src[i];
        int32_t count = o_bfs(j->g, &w, s);
        o_accumulate(j->g, &w, s, count, j->omega, j->bc);
        o_reset(&w, count);
    }
    owork_free(&w);
    j->status = 0;
    return NULL;
}

/* BC contributions of a multiset of sources (each occurrence counted).  omega == NULL:
 * plain Brandes (Eq. 2, 3).  omega != NULL: the graph is the residual graph and Eq. 4 /
 * the leaf term are applied.  nthreads workers take contiguous source ranges, each with
 * its own long-double BC; the partial vectors are summed in worker order. */
int oracle_bc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
              const int32_t *src, int64_t k, const int32_t *omega, double *bc, int nthreads) {
    ograph g = {n, row_ptr, col_idx};
    for (int64_t i = 0; i < k; i++)
        if (src[i] < 0 || src[i] >= n) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > k && k > 0) nthreads = (int)k;
    ojob *jobs = (ojob *)calloc((size_t)nthreads, sizeof(ojob));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return -2; }
    int rc = 0;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].g = &g;
        jobs[t].src = src;
        jobs[t].lo = k * t / nthreads;
        jobs[t].hi = k * (t + 1) / nthreads;
        jobs[t].omega = omega;
        jobs[t].bc = (long double *)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
        jobs[t].status = -3;
        if (!jobs[t].bc) rc = -2;
    }
    if (rc == 0) {
        if (nthreads == 1) {
            o_worker(&jobs[0]);
        } else {
            for (int t = 0; t < nthreads; t++) pthread_create(&tid[t], NULL, o_worker, &jobs[t]);
            for (int t = 0; t < nthreads; t++) pthread_join(tid[t], NULL);
        }
        for (int t = 0; t < nthreads; t++) if (jobs[t].status) rc = jobs[t].status;
    }
    if (rc == 0) {
        for (int32_t v = 0; v < n; v++) {
            long double acc = 0.0L;
            for (int t = 0; t < nthreads; t++) acc += jobs[t].bc[v];
            bc[v] = (double)acc;
        }
    }
    for (int t = 0; t < nthreads; t++) free(jobs[t].bc);
    free(jobs);
    free(tid);
    return rc;
}

/* 1-degree preprocessing (Alg. 6 on one processor; Eq. 3's omega update).  A vertex u
 * with deg(u) = 1 whose only neighbour v has deg(v) >= 2 is removed: omega[v] += 1 and
 * both arcs (u,v), (v,u) leave the graph.  A K2 component (both ends of degree 1) is
 * kept.  Vertex ids are unchanged; removed vertices get residual degree 0 and
 * removed[u] = 1.  res_col_idx must hold nnz entries; *res_nnz receives the count. */
int oracle_prune_deg1(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      int32_t *omega, uint8_t *removed, int32_t *res_row_ptr,
                      int32_t *res_col_idx, int64_t *res_nnz) {
    for (int32_t v = 0; v < n; v++) { omega[v] = 0; removed[v] = 0; }
    for (int32_t u = 0; u < n; u++) {
        if (row_ptr[u + 1] - row_ptr[u] != 1) continue;
        int32_t v = col_idx[row_ptr[u]];
        if (row_ptr[v + 1] - row_ptr[v] >= 2) {
            removed[u] = 1;
            omega[v] += 1;
        }
    }
    int64_t out = 0;
    res_row_ptr[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        if (!removed[u]) {
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                int32_t v = col_idx[e];
                if (!removed[v]) res_col_idx[out++] = v;
            }
        }
        res_row_ptr[u + 1] = (int32_t)out;
    }
    *res_nnz = out;
    return 0;
}

/* sizeof(long double) as compiled, for the Python side's sanity check. */
int oracle_long_double_size(void) { return (int)sizeof(long double); }

/*
 * bc.h — C ABI of the GB300 exact betweenness-centrality library (libbc.so).
 *
 * Method: Vella, Carbone, Bernaschi, "Algorithms and Heuristics for Scalable
 * Betweenness Centrality Computation on Multi-GPU Systems" (arXiv 1602.00963).
 *   BC(v)      = sum_{s != v != t} sigma_st(v) / sigma_st                      (Eq. 1)
 *   delta_s(v) = sum_{w : v in pred(w)} sigma_sv / sigma_sw * (1 + delta_s(w)) (Eq. 2)
 *   BC(v)      = sum_{s != v} delta_s(v)                                       (Eq. 3)
 * computed per source by a level-synchronous BFS that counts sigma (Alg. 2, 3) and a
 * backward sweep over the same levels (Alg. 4, 5); optionally with the 1-degree
 * reduction of Eq. 3 / Eq. 4 and Alg. 6 (Sec. 3.4.1).
 *
 * Conventions (all entry points):
 *   - Graphs are undirected and unweighted, given as a symmetric CSR with int32 indices:
 *     row_ptr[n+1], col_idx[nnz], each unordered edge present in both rows, rows sorted,
 *     no self-loops and no duplicates (checked when BC_VALIDATE is given).  m = nnz / 2.
 *   - BC values follow the ordered-pair convention of Alg. 1 (every vertex is a source,
 *     so an undirected pair is counted from both ends): twice the unordered values.
 *   - Every function returns a bc_status.  Out-parameters are written only on BC_OK.
 *     bc_last_error() returns this thread's text for the last failure.  No C++
 *     exception crosses the ABI.
 *   - Input buffers are caller-owned and only read during the call; the library copies
 *     what it keeps.  Output buffers are caller-owned.  With BC_DEVICE_PTRS the
 *     array arguments are device pointers on the context's device (e.g. a torch
 *     tensor's data_ptr()); otherwise they are host pointers.
 *   - cuda_stream (nullable; a cudaStream_t) orders the call after prior work on that
 *     stream; the call returns once its results are complete.
 *   - Handles are opaque and owned by the library until bc_destroy().
 */
#ifndef BC_H_
#define BC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bc_status;
enum {
  BC_OK = 0,
  BC_EINVAL = 1,     /* bad argument, malformed CSR, unsupported flag combination */
  BC_ENOMEM = 2,     /* device or host allocation failed (or exceeds the HBM budget) */
  BC_EAGAIN = 3,     /* request still running / handle busy */
  BC_ETIMEDOUT = 4,  /* a bounded device wait gave up, or a poll timed out */
  BC_ECUDA = 5,      /* CUDA runtime error */
  BC_ENOTFOUND = 6,  /* unknown request id */
  BC_ECANCELED = 7   /* request was cancelled */
};

/* ---- flags ------------------------------------------------------------------------ */
#define BC_DEVICE_PTRS    (1u << 0)  /* array arguments are device pointers            */
#define BC_VALIDATE       (1u << 1)  /* bc_graph_create: check the CSR invariants       */
#define BC_PRUNE_DEG1     (1u << 2)  /* bc_exact: 1-degree reduction (Eq. 3/4, Alg. 6)  */
#define BC_PATH_PLAIN     (1u << 3)  /* force the per-source path (one BFS per source)  */
#define BC_PATH_TILED     (1u << 4)  /* force the multi-source tile path                */
#define BC_LOOP_LAUNCH    (1u << 5)  /* tile path: one kernel launch per level phase    */
#define BC_LOOP_GRAPH     (1u << 6)  /* tile path: level loop replayed as a CUDA graph  */
#define BC_PLAIN_GRID     (1u << 7)  /* per-source path: always the grid-wide kernel     */
#define BC_PLAIN_CTA      (1u << 13) /* per-source path: one source per CTA at any size  */
/* (by default the per-source path runs graphs of up to 65,536 vertices one source per CTA,
 *  all SMs on different sources; larger graphs use the grid-wide kernel, one source at a
 *  time over the whole GPU, unless BC_PLAIN_CTA or the autotuner picks the per-CTA kernel,
 *  which suits sparse high-diameter graphs; it holds 48 bytes per vertex per CTA, two CTAs
 *  per SM, for graphs of up to 2^24 vertices) */
/* bc_exact: 2-degree heuristic (Sec. 3.4.2).  A set of degree-2 vertices c, no two sharing
 * a neighbour or being one, is run without a traversal of its own: the shortest-path DAG of c
 * is derived from those of its two neighbours a, b (run from the same CTA) and c's
 * dependencies are accumulated on it (dynamic merging of frontiers, Alg. 8 / Alg. 9).  The
 * result equals the plain run.  With BC_PRUNE_DEG1 both heuristics apply (the paper's H3):
 * the triples are chosen on the residual graph and every run carries the leaf weights.
 * Per-source path on graphs of up to 65,536 vertices only; not with BC_PATH_TILED or
 * BC_PLAIN_GRID (BC_EINVAL). */
#define BC_DEG2           (1u << 12)
/* bc_exact / bc_sources, grid-wide per-source kernel only (needs BC_PATH_PLAIN |
 * BC_PLAIN_GRID, else BC_EINVAL): the backward sweep scans each level's degree prefix CD
 * again instead of reusing the one the forward sweep stored (Sec. 3.1's reuse switched off,
 * for measuring it).  The prefix values are the same, so the result differs only by the
 * order of the kernel's floating-point atomic additions. */
#define BC_NO_CD_REUSE    (1u << 14)
/* bc_exact / bc_sources: the result depends only on the graph, the sources, the flags and
 * the GPU model (reading R9 of Eq. 2's sums: a fixed summation order, so repeated runs agree
 * bit for bit).  Every path sums in a fixed order whether or not the flag is given: the tile
 * path adds each source's terms in the order of an entry's edges, the per-CTA kernel chooses
 * a vertex's thread or warp path by degree alone, and the grid-wide kernel adds dependency
 * terms as 128-bit fixed-point integers.  What the flag adds: the configuration that
 * bc_autotune cached on the graph (a choice made by timing, so it can differ from one process
 * to the next) is not used; without a path flag the default per-source path runs. */
#define BC_DETERMINISTIC  (1u << 15)
/* bc_exact / bc_sources, tile path: run the sources in the given order.  By default a call
 * of at least four tiles groups its sources by locality first (each source's distances to
 * 32 seeded landmark vertices, found once per graph, sorted lexicographically): sources
 * close in the graph share most levels, so a tile's masks are denser and it walks fewer
 * entries.  The sum over the sources is the same; only its rounding order differs. */
#define BC_KEEP_ORDER     (1u << 16)
/* bits 8..11: tile width selector for BC_PATH_TILED: 0 = autotuned, else 32 << (k-1) */
#define BC_TILE_SHIFT     8
#define BC_TILE_MASK      (0xFu << BC_TILE_SHIFT)
#define BC_TILE(T)        ((uint32_t)((T) == 32 ? 1 : (T) == 64 ? 2 : (T) == 128 ? 3 : (T) == 256 ? 4 : 0) << BC_TILE_SHIFT)

typedef struct bc_ctx bc_ctx;
typedef struct bc_graph bc_graph;

/* Per-call statistics (all fields written on BC_OK when the pointer is non-null). */
typedef struct {
  double seconds;                 /* device time of the traversal (CUDA events)           */
  int64_t sources;                /* BFS roots processed (multiset count)                 */
  int64_t teps_sources;           /* sources counted for TEPS (Sec. 4.1, Eq. 5)           */
  int64_t edges;                  /* m = undirected edges of the input graph              */
  double gteps;                   /* teps_sources * m / seconds / 1e9                     */
  int32_t max_depth;              /* deepest BFS level seen                               */
  int32_t tile_width;             /* sources per launch: 1 = per-source path              */
  int64_t sigma_overflow_sources; /* sources whose path count passed 2^64 somewhere       */
  int64_t levels;                 /* BFS levels executed, summed over launches            */
  int64_t kernel_launches;        /* library kernels launched by the call                 */
  int64_t reached_vertices;       /* sum over sources of reached vertices                 */
  int64_t reached_arcs;           /* sum over sources of adjacency entries of reached v.  */
} bc_stats;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the library's own
 * device allocations (0 = no cap).  flags: reserved, pass 0. */
bc_status bc_ctx_create(int device, size_t hbm_budget_bytes, uint32_t flags, bc_ctx **out);

/* Upload a graph (Sec. 2 graph model) and keep it resident.  nnz < 2^31.  With
 * BC_VALIDATE the CSR is checked (monotone row_ptr, ids in range, no self-loop,
 * strictly increasing rows, symmetric) and BC_EINVAL is returned on a violation. */
bc_status bc_graph_create(bc_ctx *ctx, int32_t n, const int32_t *row_ptr,
                          const int32_t *col_idx, int64_t nnz, uint32_t flags,
                          bc_graph **out);

/* Exact BC over every source (Alg. 1 outer loop).  bc_out[n] receives the result.
 * BC_PRUNE_DEG1 applies the 1-degree reduction (Eq. 3, Eq. 4, Alg. 6; one removal
 * round, Sec. 3.4.1 footnote 1): the BFS runs on the residual graph from the
 * non-removed vertices only, with exactly the same result. */
bc_status bc_exact(bc_graph *g, uint32_t flags, double *bc_out, void *cuda_stream,
                   bc_stats *stats);

/* Sum over a multiset of sources src[k] (each occurrence counted) of delta_s (Eq. 3
 * restricted to the given roots).  BC_PRUNE_DEG1 is rejected (BC_EINVAL): Eq. 4 is
 * stated for the full source set only. */
bc_status bc_sources(bc_graph *g, const int32_t *src, int32_t k, uint32_t flags,
                     double *bc_out, void *cuda_stream, bc_stats *stats);

/* Single-source shortest-path counting (Alg. 2 / Alg. 3) on the per-source path (one CTA
 * for graphs of up to 65,536 vertices, the grid-wide kernel above that or with
 * BC_PLAIN_GRID): depth[n] (-1 = unreached), sigma[n] = number of shortest paths modulo
 * 2^64, and sigma_ovf[n] = 1 where the true count is >= 2^64.  Host buffers unless
 * BC_DEVICE_PTRS. */
bc_status bc_sssp(bc_graph *g, int32_t s, uint32_t flags, int32_t *depth, uint64_t *sigma,
                  uint8_t *sigma_ovf);

/* The same quantities for k <= 256 sources computed together by the tile path:
 * arrays are [k][n] (source-major).  Parity hook for the batched kernels. */
bc_status bc_tile_sssp(bc_graph *g, const int32_t *src, int32_t k, uint32_t flags,
                       int32_t *depth, uint64_t *sigma, uint8_t *sigma_ovf);

/* Device-side 1-degree preprocessing (Alg. 6, Eq. 3's omega): omega[n], removed[n]
 * (1 = leaf taken out), and the residual CSR: res_row_ptr[n+1], res_col_idx (capacity
 * nnz), *res_nnz.  Vertex ids are kept; removed vertices get residual degree 0. */
bc_status bc_prune(bc_graph *g, uint32_t flags, int32_t *omega, uint8_t *removed,
                   int32_t *res_row_ptr, int32_t *res_col_idx, int64_t *res_nnz);

/* ---- autotuner ----------------------------------------------------------------------- */
typedef struct {
  int32_t tile_width;     /* 32, 64, 128 or 256 (0 = per-source path is faster)      */
  float alpha;            /* top-down -> bottom-up when frontier arcs > alpha * unvisited
                             arcs (tile path: > alpha * all arcs)                     */
  float beta;             /* bottom-up -> top-down: per-source path when frontier vertices
                             < n / beta; tile path when the frontier's arcs fall below
                             nnz / beta (0: the alpha test decides every level)       */
  int32_t loop_mode;      /* 0 persistent kernel, 1 per-level launches, 2 CUDA graph  */
  int32_t plain_cta;      /* tile_width 0: 1 = the per-source path runs one source per
                             CTA at any size (as BC_PLAIN_CTA)                        */
  double probe_seconds;   /* time the tuner spent                                      */
  int32_t hub_degree;     /* tile path, forward: candidates of this degree or more have
                             their parents summed in warp work items of hub_chunk edges
                             (load balance)                                           */
  int32_t hub_chunk;      /* tile path, backward: entries of this degree or more are split
                             into warp work items of this many edges                  */
} bc_tune_result;

/* Time the candidate configurations on a small seeded probe of sources and cache the
 * winner on the graph (later bc_exact / bc_sources calls without an explicit tile
 * selector use it).  probe_sources = 0 picks a default. */
bc_status bc_autotune(bc_graph *g, int32_t probe_sources, uint64_t seed, bc_tune_result *out);

/* ---- serving: continuous batching of BC requests ------------------------------------- */
enum { BC_REQ_EXACT_LIST = 0, BC_REQ_SAMPLED = 1 };

typedef struct {
  bc_graph *graph;        /* a graph created on the same context                      */
  int32_t mode;           /* BC_REQ_EXACT_LIST: src[k]; BC_REQ_SAMPLED: k sources drawn */
  int32_t k;              /* number of sources                                        */
  const int32_t *src;     /* host array, copied at submit (EXACT_LIST)                */
  uint64_t seed;          /* SAMPLED: seed of the draw                                */
  double *bc_out;         /* host buffer [n], written before the request completes    */
} bc_request;

typedef struct {
  bc_status status;       /* BC_OK, or the failure                                    */
  double queue_seconds;   /* submit -> first tile started                             */
  double latency_seconds; /* submit -> completion                                     */
  double scale;           /* SAMPLED: n_nonisolated / k (estimator scale); else 1.0   */
  int64_t sources;        /* sources processed                                        */
} bc_result;

/* Enqueue a request; returns at once with *request_id.  The scheduler admits it when
 * its device footprint fits the context budget, merges its sources with those of
 * other requests on the same graph into shared tiles and overlaps work on several
 * streams.  SAMPLED draws k distinct non-isolated sources from `seed` (SplitMix64
 * stream); bc_out holds the raw sum of delta_s over the drawn sources. */
bc_status bc_stream_submit(bc_ctx *ctx, const bc_request *req, uint64_t *request_id);

/* The k distinct non-isolated sources that a BC_REQ_SAMPLED request with this seed
 * uses (SplitMix64 stream, Floyd's sampling over the non-isolated vertices in increasing
 * id order), written to the host array src_out[k] in increasing order. */
bc_status bc_sample_sources(bc_graph *g, int32_t k, uint64_t seed, int32_t *src_out);

/* Wait up to timeout_us (0 = do not wait, <0 = forever) for a request.  Returns
 * BC_EAGAIN while it runs; BC_OK once finished (res filled, id released). */
bc_status bc_stream_poll(bc_ctx *ctx, uint64_t request_id, int32_t timeout_us, bc_result *res);

/* Cancel a queued request (a running one finishes its current tile first). */
bc_status bc_stream_cancel(bc_ctx *ctx, uint64_t request_id);

/* Destroy a graph or a context.  A graph with requests in flight returns BC_EAGAIN;
 * destroying a context destroys its graphs and stops its scheduler. */
bc_status bc_destroy(void *handle);

/* Copy this thread's last error text into buf (always NUL-terminated). */
void bc_last_error(char *buf, size_t len);

/* Library version string. */
const char *bc_version(void);

/* ---- allocation-free entry point ------------------------------------------------------
 * No counterpart in the paper: an interface addition for callers that must not allocate
 * device memory — code running inside memory owned by another allocator (a framework's
 * caching allocator, a fixed pool that must not fragment), latency-critical loops where
 * cudaMalloc's implicit device synchronisation is not acceptable, or processes under a
 * hard device-memory quota.
 * Computes the same as bc_sources(..., BC_PATH_PLAIN | BC_DEVICE_PTRS, ...): the sum
 * over the multiset src[k] of delta_s, on the graph given by row_ptr[n+1] / col_idx[nnz]
 * (a symmetric CSR as for bc_graph_create; its structure is not validated here).  Every
 * pointer is a device pointer owned by the caller; bc_out[n] is overwritten (zeros for
 *  k = 0).  Working storage is one static device array of about 4.2 MB, sized for
 * BC_NOALLOC_MAX_N vertices, that every GPU loading the library holds until the process
 * exits; the CUDA runtime places it on a device when it loads the library's device code
 * there (with lazy module loading: at the latest during the first call on that device),
 * and no call allocates anything.  The call clears that array at its start, checks every
 * source id on the device, and synchronises cuda_stream twice (after the check and after
 * the traversal): it returns when the result is complete.  Calls in one process share the
 * array and are serialised (one runs at a time, to completion); each process has its own
 * copy of it, so calls in different processes never share it.  The first call on a device
 * looks up the array's device address with that device current: make it before any stream
 * capture.  BC_EINVAL: n outside [1, BC_NOALLOC_MAX_N], nnz odd or outside [0, 2^31), k < 0,
 * a NULL pointer, or a source id outside [0, n). */
#define BC_NOALLOC_MAX_N 65536
bc_status bc_sources_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             int64_t nnz, const int32_t *src, int32_t k, double *bc_out,
                             void *cuda_stream);

/* Testing hook: device-wait limit in milliseconds for bounded spins (grid barriers);
 * 0 makes every wait give up at once so the BC_ETIMEDOUT path can be exercised. */
bc_status bc_set_wait_limit_ms(bc_ctx *ctx, int64_t ms);

#ifdef __cplusplus
}
#endif
#endif /* BC_H_ */

// C ABI of libbc.so: contexts, resident graphs, dispatch and error reporting.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "bc_internal.h"
#include "bc_scan.cuh"

namespace bcl {

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }
bc_status fail(bc_status st, const std::string &msg) {
  t_err = msg;
  return st;
}
bc_status cuda_fail(cudaError_t e, const char *what) {
  t_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BC_ENOMEM : BC_ECUDA;
}

// Allocation failure injection for tests: BC_FAULT_ALLOC=k makes the k-th accounted
// device allocation of the process fail with BC_ENOMEM.
static std::atomic<long> g_alloc_count{0};
static long fault_alloc_at() {
  static long at = [] {
    const char *e = getenv("BC_FAULT_ALLOC");
    return e ? atol(e) : 0L;
  }();
  return at;
}

bc_status DevMem::alloc(void **p, size_t bytes) {
  long k = ++g_alloc_count;
  if (fault_alloc_at() > 0 && k == fault_alloc_at())
    return fail(BC_ENOMEM, "injected allocation failure (BC_FAULT_ALLOC)");
  size_t prev = used.fetch_add(bytes);
  if (budget && prev + bytes > budget) {
    used.fetch_sub(bytes);
    return fail(BC_ENOMEM, "device allocation of " + std::to_string(bytes) +
                               " bytes exceeds the context HBM budget");
  }
  if (p) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      used.fetch_sub(bytes);
      *p = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
  }
  return BC_OK;
}

void DevMem::release(void *p, size_t bytes) {
  if (p) cudaFree(p);
  used.fetch_sub(bytes);
}

namespace {

// ---------------------------------------------------------------- small kernels
__global__ void k_validate(int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                           int *err) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
    int32_t a = rp[v], b = rp[v + 1];
    if (v == 0 && a != 0) atomicMax(err, 1);
    if (v == n - 1 && (int64_t)b != nnz) atomicMax(err, 1);
    if (b < a) { atomicMax(err, 2); continue; }
    int32_t prev = -1;
    for (int32_t e = a; e < b; e++) {
      int32_t w = ci[e];
      if (w < 0 || w >= n) { atomicMax(err, 3); break; }
      if (w == v) { atomicMax(err, 4); break; }
      if (w <= prev) { atomicMax(err, 5); break; }
      prev = w;
      // symmetry: v must appear in w's sorted row
      int32_t lo = rp[w], hi = rp[w + 1];
      bool found = false;
      while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        int32_t x = ci[mid];
        if (x == v) { found = true; break; }
        if (x < v) lo = mid + 1; else hi = mid;
      }
      if (!found) { atomicMax(err, 6); break; }
    }
  }
}

__global__ void k_degree_stats(int32_t n, const int32_t *rp, unsigned long long *nonisolated,
                               int *maxdeg) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long cnt = 0;
  int mx = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
    int d = rp[v + 1] - rp[v];
    cnt += d > 0;
    mx = max(mx, d);
  }
  for (int o = 16; o; o >>= 1) {
    cnt += __shfl_down_sync(BC_FULL, cnt, o);
    mx = max(mx, __shfl_down_sync(BC_FULL, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(nonisolated, cnt);
    atomicMax(maxdeg, mx);
  }
}

// Sources of a full run: every vertex with at least one edge (an isolated source
// reaches nothing and contributes nothing).
// flag[v] = 1 for a vertex with an edge (v < n), flag[n] = 0
__global__ void k_nonisolated_flags(int32_t n, const int32_t *rp, int32_t *flag) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = (v < n && rp[v + 1] > rp[v]) ? 1 : 0;
}

// out[pos[v]] = v for every vertex with an edge: the list in increasing vertex order
__global__ void k_nonisolated_scatter(int32_t n, const int32_t *rp, const int32_t *pos, int32_t *out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (rp[v + 1] > rp[v]) out[pos[v]] = (int32_t)v;
}

__global__ void k_check_sources(int32_t n, const int32_t *src, int32_t k, int *err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    if (src[i] < 0 || src[i] >= n) atomicMax(err, 1);
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

int grid_for(int64_t work, int num_sms) {
  int64_t b = (work + 255) / 256;
  int64_t cap = (int64_t)num_sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

Ctx *as_ctx(void *h) {
  Ctx *c = (Ctx *)h;
  return (c && c->magic == kCtxMagic) ? c : nullptr;
}
Graph *as_graph(void *h) {
  Graph *g = (Graph *)h;
  return (g && g->magic == kGraphMagic) ? g : nullptr;
}

struct DevBuf {
  Ctx *ctx = nullptr;
  void *p = nullptr;
  size_t bytes = 0;
  bc_status get(Ctx *c, size_t b) {
    ctx = c;
    bytes = b;
    return c->mem.alloc(&p, b);
  }
  ~DevBuf() {
    if (p) ctx->mem.release(p, bytes);
  }
};

}  // namespace

// Dispatch a multiset of device-resident sources to the per-source or the tile path.
bc_status run_sources(Graph *g, const int32_t *d_src, int32_t k, uint32_t flags,
                      const int32_t *omega, bool leaf_term, double *d_bc, cudaStream_t st,
                      bc_stats *stats, const DeviceGraph *dg) {
  Ctx *ctx = g->ctx;
  if ((flags & BC_NO_CD_REUSE) && (flags & (BC_PATH_PLAIN | BC_PLAIN_GRID)) != (BC_PATH_PLAIN | BC_PLAIN_GRID))
    return fail(BC_EINVAL, "BC_NO_CD_REUSE applies to the grid-wide per-source kernel only "
                           "(BC_PATH_PLAIN | BC_PLAIN_GRID)");
  if (k <= 0) return BC_OK;
  bool tiled = (flags & BC_PATH_TILED) != 0;
  bool plain = (flags & BC_PATH_PLAIN) != 0;
  int T = 0;
  uint32_t tsel = (flags & BC_TILE_MASK) >> BC_TILE_SHIFT;
  if (tsel >= 1 && tsel <= 4) T = 32 << (tsel - 1);
  float alpha = 0.5f, beta = 24.f, tile_beta = 0.f;
  int hub = 0, hub_chunk = 0;
  int loop_mode = (flags & BC_LOOP_LAUNCH) ? 1 : (flags & BC_LOOP_GRAPH) ? 2 : 0;
  // BC_DETERMINISTIC: the autotuner's cached choice (made by timing) is not used
  const bool tuned = g->tune.ready && !(flags & BC_DETERMINISTIC);
  if (tuned) {
    alpha = g->tune.res.alpha;
    if (g->tune.res.tile_width > 0) {  // the tuned thresholds of the tile path
      tile_beta = g->tune.res.beta;
      hub = g->tune.res.hub_degree;
      hub_chunk = g->tune.res.hub_chunk;
    } else if (g->tune.res.beta > 0.f) {
      beta = g->tune.res.beta;
    }
    if (!tiled && !plain) {
      if (g->tune.res.tile_width > 0) {
        tiled = true;
        if (!T) T = g->tune.res.tile_width;
        if (!(flags & (BC_LOOP_LAUNCH | BC_LOOP_GRAPH))) loop_mode = g->tune.res.loop_mode;
      } else {
        plain = true;
      }
    }
  }
  if (!tiled && !plain) tiled = T > 0;
  if (tiled && !plain) {
    if (!T) T = 64;
    // sources grouped by locality (at least four tiles; BC_KEEP_ORDER: as given)
    int32_t *osrc = nullptr;
    size_t obytes = 0;
    if (!(flags & BC_KEEP_ORDER) && (int64_t)k >= 4ll * T) {
      bc_status s = order_sources(g, dg, d_src, k, T, st, &osrc, &obytes);
      if (s) return s;
    }
    TileArgs ta{};
    ta.g = dg;
    ta.omega = omega;
    ta.src = osrc ? osrc : d_src;
    ta.nsrc = k;
    ta.bc = d_bc;
    ta.T = T;
    ta.loop_mode = loop_mode;
    ta.alpha = alpha;
    ta.beta = tile_beta;
    ta.hub = hub;
    ta.hub_chunk = hub_chunk;
    bc_status s = tile_run(ctx, g, &g->tile, ta, st, stats);
    if (osrc) {
      cudaStreamSynchronize(st);  // the tile has finished with the ordered list
      ctx->mem.release(osrc, obytes);
    }
    if (s) return s;
    (void)leaf_term;
    return BC_OK;
  }
  PlainArgs pa{};
  pa.g = dg;
  pa.omega = omega;
  pa.src = d_src;
  pa.nsrc = k;
  pa.bc = d_bc;
  pa.leaf_term = leaf_term;
  pa.max_degree = g->max_degree;
  pa.alpha = alpha;
  pa.beta = beta;
  pa.no_cd_reuse = (flags & BC_NO_CD_REUSE) != 0;
  const bool want_cta = (flags & BC_PLAIN_CTA) || (!(flags & (BC_PATH_PLAIN | BC_DETERMINISTIC)) &&
                                                    g->tune.ready && g->tune.res.plain_cta);
  if (!(flags & BC_PLAIN_GRID) && (cta_fits(dg->n) || (want_cta && dg->n <= kCtaForcedMaxN)))
    return cta_run(ctx, g, &g->cta, pa, st, stats);
  bc_status s = plain_ensure(ctx, &g->plain, dg->n);
  if (s) return s;
  return plain_run(ctx, &g->plain, pa, st, stats);
}

}  // namespace bcl

using namespace bcl;

// ================================================================== C ABI
extern "C" {

const char *bc_version(void) { return "gb300-bc 0.1 (sm_103a)"; }

void bc_last_error(char *buf, size_t len) {
  if (!buf || !len) return;
  size_t k = t_err.size() < len - 1 ? t_err.size() : len - 1;
  memcpy(buf, t_err.data(), k);
  buf[k] = 0;
}

bc_status bc_ctx_create(int device, size_t hbm_budget_bytes, uint32_t flags, bc_ctx **out) {
  if (!out) return fail(BC_EINVAL, "bc_ctx_create: out is NULL");
  if (flags != 0) return fail(BC_EINVAL, "bc_ctx_create: flags must be 0");
  int ndev = 0;
  BC_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(BC_EINVAL, "bc_ctx_create: no such device");
  BC_CUDA_TRY(cudaSetDevice(device));
  int coop = 0;
  BC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  if (!coop) return fail(BC_EINVAL, "device does not support cooperative launches");
  Ctx *c = new (std::nothrow) Ctx();
  if (!c) return fail(BC_ENOMEM, "bc_ctx_create: host allocation failed");
  c->device = device;
  c->mem.budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (const char *e = getenv("BC_WAIT_LIMIT_MS")) c->wait_limit_ns = (uint64_t)atoll(e) * 1000000ull;
  cudaError_t e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaStreamCreate");
  }
  *out = (bc_ctx *)c;
  return BC_OK;
}

bc_status bc_set_wait_limit_ms(bc_ctx *ctx, int64_t ms) {
  Ctx *c = as_ctx(ctx);
  if (!c || ms < 0) return fail(BC_EINVAL, "bc_set_wait_limit_ms: bad argument");
  c->wait_limit_ns = (uint64_t)ms * 1000000ull;
  return BC_OK;
}

bc_status bc_graph_create(bc_ctx *ctx, int32_t n, const int32_t *row_ptr,
                          const int32_t *col_idx, int64_t nnz, uint32_t flags,
                          bc_graph **out) {
  Ctx *c = as_ctx(ctx);
  if (!c || !out || !row_ptr || (nnz > 0 && !col_idx))
    return fail(BC_EINVAL, "bc_graph_create: NULL argument");
  if (n <= 0) return fail(BC_EINVAL, "bc_graph_create: n must be positive");
  if (nnz < 0 || nnz >= (int64_t)1 << 31)
    return fail(BC_EINVAL, "bc_graph_create: nnz must be in [0, 2^31) (int32 CSR)");
  if (nnz % 2) return fail(BC_EINVAL, "bc_graph_create: a symmetric CSR has an even nnz");
  if (flags & ~(BC_DEVICE_PTRS | BC_VALIDATE)) return fail(BC_EINVAL, "bc_graph_create: bad flags");
  BC_CUDA_TRY(cudaSetDevice(c->device));
  Graph *g = new (std::nothrow) Graph();
  if (!g) return fail(BC_ENOMEM, "bc_graph_create: host allocation failed");
  g->ctx = c;
  g->g.n = n;
  g->g.nnz = nnz;
  size_t rb = ((size_t)n + 1) * 4, cb = (size_t)nnz * 4;
  bc_status s = c->mem.alloc((void **)&g->g.rp, rb);
  if (!s) s = c->mem.alloc((void **)&g->g.ci, cb);
  if (s) {
    if (g->g.rp) c->mem.release(g->g.rp, rb);
    delete g;
    return s;
  }
  cudaStream_t st = c->own_stream;
  cudaMemcpyKind kind = (flags & BC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(g->g.rp, row_ptr, rb, kind, st);
  if (e == cudaSuccess && cb) e = cudaMemcpyAsync(g->g.ci, col_idx, cb, kind, st);
  int *d_scr = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_scr, 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_scr, 0, 16, st);
  int hs[4] = {0, 0, 0, 0};
  if (e == cudaSuccess && (flags & BC_VALIDATE)) {
    k_validate<<<grid_for(n, c->num_sms), 256, 0, st>>>(n, nnz, g->g.rp, g->g.ci, d_scr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_degree_stats<<<grid_for(n, c->num_sms), 256, 0, st>>>(
        n, g->g.rp, (unsigned long long *)(d_scr + 2), d_scr + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, d_scr, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (d_scr) cudaFree(d_scr);
    c->mem.release(g->g.rp, rb);
    c->mem.release(g->g.ci, cb);
    delete g;
    return cuda_fail(e, "bc_graph_create: upload");
  }
  if (hs[0]) {
    cudaFree(d_scr);
    c->mem.release(g->g.rp, rb);
    c->mem.release(g->g.ci, cb);
    delete g;
    static const char *why[] = {"", "row_ptr[0] != 0 or row_ptr[n] != nnz", "row_ptr decreases",
                                "column index out of range", "self-loop", "row not strictly increasing (duplicate edge or unsorted)",
                                "CSR is not symmetric"};
    return fail(BC_EINVAL, std::string("bc_graph_create: invalid CSR: ") + why[hs[0] < 7 ? hs[0] : 0]);
  }
  g->max_degree = hs[1];
  g->n_nonisolated = (int64_t)(*(unsigned long long *)(hs + 2));
  g->d_chk = d_scr;  // kept for the source checks of later calls
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->graphs.push_back(g);
  }
  *out = (bc_graph *)g;
  return BC_OK;
}

// All non-isolated vertices of dg, in increasing order, as a device source list built
// into `buf` (an ordered compaction: flags, exclusive scan, scatter), so every call gives
// the same sources to the same tiles and CTAs.
static bc_status full_source_list(Graph *g, const DeviceGraph *dg, int32_t **list, int32_t *count,
                                  DevBuf &buf, cudaStream_t st) {
  Ctx *c = g->ctx;
  const int64_t n1 = (int64_t)dg->n + 1;
  bc_status s = buf.get(c, (size_t)n1 * 4);
  if (s) return s;
  int32_t *flag = nullptr, *pos = nullptr;
  void *scratch = nullptr;
  cudaError_t e = cudaMalloc(&flag, (size_t)n1 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&pos, (size_t)n1 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&scratch, scan_scratch_bytes(n1));
  const int nb = grid_for(dg->n, c->num_sms);
  if (e == cudaSuccess) {
    k_nonisolated_flags<<<nb, 256, 0, st>>>(dg->n, dg->rp, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_exclusive_i32(flag, pos, n1, scratch, st);
  if (e == cudaSuccess) {
    k_nonisolated_scatter<<<nb, 256, 0, st>>>(dg->n, dg->rp, pos, (int32_t *)buf.p);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, pos + dg->n, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (flag) cudaFree(flag);
  if (pos) cudaFree(pos);
  if (scratch) cudaFree(scratch);
  if (e != cudaSuccess) return cuda_fail(e, "source list");
  *list = (int32_t *)buf.p;
  *count = h;
  return BC_OK;
}

// 2-degree heuristic (Sec. 3.4.2): pick degree-2 vertices c with neighbours a, b, in vertex
// order, such that no vertex belongs to two triples; each triple runs a and b and derives c
// (one CTA), every other source runs as usual.  With `pruned` (both heuristics, after the
// 1-degree reduction) the triples are chosen on the residual graph, the sources are the
// non-removed vertices that have an edge or a leaf, and every run carries the leaf weights.
static bc_status run_deg2(Graph *g, bool pruned, double *d_bc, cudaStream_t st, bc_stats *acc) {
  Ctx *c = g->ctx;
  const DeviceGraph *dg = pruned ? &g->prune.res : &g->g;
  const int32_t n = dg->n;
  std::vector<int32_t> rp((size_t)n + 1), ci((size_t)dg->nnz), om;
  BC_CUDA_TRY(cudaMemcpy(rp.data(), dg->rp, rp.size() * 4, cudaMemcpyDeviceToHost));
  if (!ci.empty()) BC_CUDA_TRY(cudaMemcpy(ci.data(), dg->ci, ci.size() * 4, cudaMemcpyDeviceToHost));
  if (pruned) {
    om.resize((size_t)n);
    BC_CUDA_TRY(cudaMemcpy(om.data(), g->prune.omega, om.size() * 4, cudaMemcpyDeviceToHost));
  }
  std::vector<uint8_t> used((size_t)n, 0);
  std::vector<int32_t> tri, single;
  for (int32_t v = 0; v < n; v++) {
    if (rp[v + 1] - rp[v] != 2) continue;
    const int32_t a = ci[rp[v]], b = ci[rp[v] + 1];
    if (used[v] || used[a] || used[b]) continue;
    used[v] = used[a] = used[b] = 1;
    tri.push_back(a);
    tri.push_back(b);
    tri.push_back(v);
  }
  for (int32_t v = 0; v < n; v++)
    if (!used[v] && (rp[v + 1] > rp[v] || (pruned && om[v] > 0))) single.push_back(v);
  DevBuf sbuf, tbuf;
  bc_status s = sbuf.get(c, (single.size() + 1) * 4);
  if (!s) s = tbuf.get(c, (tri.size() + 3) * 4);
  if (s) return s;
  if (!single.empty())
    BC_CUDA_TRY(cudaMemcpyAsync(sbuf.p, single.data(), single.size() * 4, cudaMemcpyHostToDevice, st));
  if (!tri.empty())
    BC_CUDA_TRY(cudaMemcpyAsync(tbuf.p, tri.data(), tri.size() * 4, cudaMemcpyHostToDevice, st));
  PlainArgs pa{};
  pa.g = dg;
  pa.omega = pruned ? g->prune.omega : nullptr;
  pa.leaf_term = pruned;
  pa.src = (const int32_t *)sbuf.p;
  pa.nsrc = (int32_t)single.size();
  pa.tri = (const int32_t *)tbuf.p;
  pa.ntri = (int32_t)(tri.size() / 3);
  pa.bc = d_bc;
  pa.max_degree = g->max_degree;
  return cta_run(c, g, &g->cta, pa, st, acc);
}

static void finish_stats(Graph *g, bc_stats *acc, bc_stats *out) {
  if (!out) return;
  acc->edges = g->g.nnz / 2;
  acc->gteps = acc->seconds > 0 ? (double)acc->teps_sources * (double)acc->edges / acc->seconds / 1e9 : 0.0;
  *out = *acc;
}

bc_status bc_exact(bc_graph *graph, uint32_t flags, double *bc_out, void *cuda_stream,
                   bc_stats *stats) {
  Graph *g = as_graph(graph);
  if (!g || !bc_out) return fail(BC_EINVAL, "bc_exact: NULL argument");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
  const int32_t n = g->g.n;
  DevBuf bcbuf;
  double *d_bc = bc_out;
  if (!(flags & BC_DEVICE_PTRS)) {
    bc_status s = bcbuf.get(c, (size_t)n * 8);
    if (s) return s;
    d_bc = (double *)bcbuf.p;
  }
  BC_CUDA_TRY(cudaMemsetAsync(d_bc, 0, (size_t)n * 8, st));
  bc_stats acc{};
  bc_status s;
  if (flags & BC_DEG2) {
    if (flags & (BC_PATH_TILED | BC_PLAIN_GRID | BC_NO_CD_REUSE))
      return fail(BC_EINVAL, "bc_exact: BC_DEG2 runs on the per-source CTA kernel only");
    if (!cta_fits(n)) return fail(BC_EINVAL, "bc_exact: BC_DEG2 needs a graph of at most 65,536 vertices");
    if (flags & BC_PRUNE_DEG1) {
      s = prune_build(c, g, st);
      if (s) return s;
    }
    s = run_deg2(g, (flags & BC_PRUNE_DEG1) != 0, d_bc, st, &acc);
  } else if (flags & BC_PRUNE_DEG1) {
    s = prune_build(c, g, st);
    if (s) return s;
    s = run_sources(g, g->prune.src, g->prune.nsrc, flags, g->prune.omega, true, d_bc, st, &acc,
                    &g->prune.res);
  } else {
    DevBuf lbuf;
    int32_t *list = nullptr, cnt = 0;
    s = full_source_list(g, &g->g, &list, &cnt, lbuf, st);
    if (s) return s;
    s = run_sources(g, list, cnt, flags, nullptr, false, d_bc, st, &acc, &g->g);
  }
  if (s) return s;
  acc.teps_sources = g->n_nonisolated;
  if (!(flags & BC_DEVICE_PTRS)) {
    BC_CUDA_TRY(cudaMemcpyAsync(bc_out, d_bc, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  }
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  finish_stats(g, &acc, stats);
  return BC_OK;
}

bc_status bc_sources(bc_graph *graph, const int32_t *src, int32_t k, uint32_t flags,
                     double *bc_out, void *cuda_stream, bc_stats *stats) {
  Graph *g = as_graph(graph);
  if (!g || !bc_out || (k > 0 && !src)) return fail(BC_EINVAL, "bc_sources: NULL argument");
  if (k < 0) return fail(BC_EINVAL, "bc_sources: k < 0");
  if (flags & BC_PRUNE_DEG1)
    return fail(BC_EINVAL, "bc_sources: BC_PRUNE_DEG1 applies to bc_exact only (Eq. 4 needs every source)");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
  const int32_t n = g->g.n;
  DevBuf bcbuf, sbuf;
  double *d_bc = bc_out;
  const int32_t *d_src = src;
  if (!(flags & BC_DEVICE_PTRS)) {
    for (int32_t i = 0; i < k; i++)
      if (src[i] < 0 || src[i] >= n) return fail(BC_EINVAL, "bc_sources: source id out of range");
    bc_status s = bcbuf.get(c, (size_t)n * 8);
    if (!s && k) s = sbuf.get(c, (size_t)k * 4);
    if (s) return s;
    d_bc = (double *)bcbuf.p;
    if (k) {
      BC_CUDA_TRY(cudaMemcpyAsync(sbuf.p, src, (size_t)k * 4, cudaMemcpyHostToDevice, st));
      d_src = (const int32_t *)sbuf.p;
    }
  } else if (k) {
    // the graph's check word (calls on one graph are serialised by g->mu)
    BC_CUDA_TRY(cudaMemsetAsync(g->d_chk, 0, 4, st));
    k_check_sources<<<grid_for(k, c->num_sms), 256, 0, st>>>(n, src, k, g->d_chk);
    BC_CUDA_TRY(cudaGetLastError());
    int h = 0;
    BC_CUDA_TRY(cudaMemcpyAsync(&h, g->d_chk, 4, cudaMemcpyDeviceToHost, st));
    BC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) return fail(BC_EINVAL, "bc_sources: source id out of range");
  }
  BC_CUDA_TRY(cudaMemsetAsync(d_bc, 0, (size_t)n * 8, st));
  bc_stats acc{};
  bc_status s = run_sources(g, d_src, k, flags, nullptr, false, d_bc, st, &acc, &g->g);
  if (s) return s;
  acc.teps_sources = k;
  if (!(flags & BC_DEVICE_PTRS)) {
    BC_CUDA_TRY(cudaMemcpyAsync(bc_out, d_bc, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  }
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  finish_stats(g, &acc, stats);
  return BC_OK;
}

bc_status bc_sssp(bc_graph *graph, int32_t s, uint32_t flags, int32_t *depth, uint64_t *sigma,
                  uint8_t *sigma_ovf) {
  Graph *g = as_graph(graph);
  if (!g || !depth || !sigma || !sigma_ovf) return fail(BC_EINVAL, "bc_sssp: NULL argument");
  if (s < 0 || s >= g->g.n) return fail(BC_EINVAL, "bc_sssp: source out of range");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = c->own_stream;
  const size_t n = (size_t)g->g.n;
  const bool cta = !(flags & BC_PLAIN_GRID) &&
                   (cta_fits(g->g.n) || ((flags & BC_PLAIN_CTA) && g->g.n <= kCtaForcedMaxN));
  bc_status r = cta ? BC_OK : plain_ensure(c, &g->plain, g->g.n);
  if (r) return r;
  // one scratch block carved at 16-byte aligned offsets: sigma | depth | ovf | src
  const size_t o_dep = align16(n * 8), o_ovf = o_dep + align16(n * 4),
               o_src = o_ovf + align16(n), total = o_src + 16;
  DevBuf b;
  r = b.get(c, total);
  if (r) return r;
  char *base = (char *)b.p;
  unsigned long long *d_sig = (unsigned long long *)base;
  int32_t *d_dep = (int32_t *)(base + o_dep);
  uint8_t *d_ovf = (uint8_t *)(base + o_ovf);
  int32_t *d_src = (int32_t *)(base + o_src);
  BC_CUDA_TRY(cudaMemcpyAsync(d_src, &s, 4, cudaMemcpyHostToDevice, st));
  PlainArgs pa{};
  pa.g = &g->g;
  pa.src = d_src;
  pa.nsrc = 1;
  pa.out_depth = d_dep;
  pa.out_sigma = d_sig;
  pa.out_ovf = d_ovf;
  pa.max_degree = g->max_degree;
  pa.alpha = g->tune.ready ? g->tune.res.alpha : 0.5f;
  pa.beta = (g->tune.ready && g->tune.res.tile_width == 0 && g->tune.res.beta > 0.f) ? g->tune.res.beta : 24.f;
  pa.bc = nullptr;
  if (cta) {
    r = cta_run(c, g, &g->cta, pa, st, nullptr);
  } else {
    r = plain_run(c, &g->plain, pa, st, nullptr);
  }
  if (r) return r;
  cudaMemcpyKind kind = (flags & BC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  BC_CUDA_TRY(cudaMemcpyAsync(depth, d_dep, n * 4, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(sigma, d_sig, n * 8, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(sigma_ovf, d_ovf, n, kind, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  return BC_OK;
}

bc_status bc_tile_sssp(bc_graph *graph, const int32_t *src, int32_t k, uint32_t flags,
                       int32_t *depth, uint64_t *sigma, uint8_t *sigma_ovf) {
  Graph *g = as_graph(graph);
  if (!g || !src || !depth || !sigma || !sigma_ovf) return fail(BC_EINVAL, "bc_tile_sssp: NULL argument");
  if (k <= 0 || k > 256) return fail(BC_EINVAL, "bc_tile_sssp: k must be in [1, 256]");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = c->own_stream;
  const size_t n = (size_t)g->g.n;
  const bool dev = (flags & BC_DEVICE_PTRS) != 0;
  std::vector<int32_t> hs(k);
  if (dev) {
    BC_CUDA_TRY(cudaMemcpy(hs.data(), src, (size_t)k * 4, cudaMemcpyDeviceToHost));
  } else {
    memcpy(hs.data(), src, (size_t)k * 4);
  }
  for (int i = 0; i < k; i++)
    if (hs[i] < 0 || hs[i] >= g->g.n) return fail(BC_EINVAL, "bc_tile_sssp: source out of range");
  const size_t nk = n * (size_t)k;
  const size_t o_dep = align16(nk * 8), o_ovf = o_dep + align16(nk * 4),
               o_src = o_ovf + align16(nk), total = o_src + align16((size_t)k * 4);
  DevBuf b;
  bc_status r = b.get(c, total);
  if (r) return r;
  char *base = (char *)b.p;
  unsigned long long *d_sig = (unsigned long long *)base;
  int32_t *d_dep = (int32_t *)(base + o_dep);
  uint8_t *d_ovf = (uint8_t *)(base + o_ovf);
  int32_t *d_src = (int32_t *)(base + o_src);
  BC_CUDA_TRY(cudaMemcpyAsync(d_src, hs.data(), (size_t)k * 4, cudaMemcpyHostToDevice, st));
  int T = 32;
  while (T < k) T *= 2;
  uint32_t tsel = (flags & BC_TILE_MASK) >> BC_TILE_SHIFT;
  if (tsel >= 1 && tsel <= 4 && (32 << (tsel - 1)) >= k) T = 32 << (tsel - 1);
  TileArgs ta{};
  ta.g = &g->g;
  ta.src = d_src;
  ta.nsrc = k;
  ta.T = T;
  ta.loop_mode = (flags & BC_LOOP_LAUNCH) ? 1 : (flags & BC_LOOP_GRAPH) ? 2 : 0;
  ta.alpha = g->tune.ready ? g->tune.res.alpha : 0.5f;
  if (g->tune.ready && g->tune.res.tile_width > 0) {
    ta.beta = g->tune.res.beta;
    ta.hub = g->tune.res.hub_degree;
    ta.hub_chunk = g->tune.res.hub_chunk;
  }
  ta.out_depth = d_dep;
  ta.out_sigma = d_sig;
  ta.out_ovf = d_ovf;
  r = tile_run(c, g, &g->tile, ta, st, nullptr);
  if (r) return r;
  cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  BC_CUDA_TRY(cudaMemcpyAsync(depth, d_dep, n * k * 4, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(sigma, d_sig, n * k * 8, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(sigma_ovf, d_ovf, n * k, kind, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  return BC_OK;
}

bc_status bc_prune(bc_graph *graph, uint32_t flags, int32_t *omega, uint8_t *removed,
                   int32_t *res_row_ptr, int32_t *res_col_idx, int64_t *res_nnz) {
  Graph *g = as_graph(graph);
  if (!g || !omega || !removed || !res_row_ptr || !res_col_idx || !res_nnz)
    return fail(BC_EINVAL, "bc_prune: NULL argument");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = c->own_stream;
  bc_status r = prune_build(c, g, st);
  if (r) return r;
  const size_t n = (size_t)g->g.n;
  cudaMemcpyKind kind = (flags & BC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  BC_CUDA_TRY(cudaMemcpyAsync(omega, g->prune.omega, n * 4, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(removed, g->prune.removed, n, kind, st));
  BC_CUDA_TRY(cudaMemcpyAsync(res_row_ptr, g->prune.res.rp, (n + 1) * 4, kind, st));
  if (g->prune.res.nnz)
    BC_CUDA_TRY(cudaMemcpyAsync(res_col_idx, g->prune.res.ci, (size_t)g->prune.res.nnz * 4, kind, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  *res_nnz = g->prune.res.nnz;
  return BC_OK;
}

bc_status bc_destroy(void *handle);

}  // extern "C"

namespace bcl {
void server_stop(Ctx *c);  // bc_serve.cu
bool server_graph_busy(Ctx *c, Graph *g);
void server_forget_graph(Ctx *c, Graph *g);

static void graph_free(Graph *g) {
  Ctx *c = g->ctx;
  plain_free(c, &g->plain);
  prune_free(c, &g->prune);
  if (g->cta) {
    cta_free(c, g->cta);
    g->cta = nullptr;
  }
  if (g->tile) {
    tile_free(c, g->tile);
    g->tile = nullptr;
  }
  c->mem.release(g->g.rp, ((size_t)g->g.n + 1) * 4);
  c->mem.release(g->g.ci, (size_t)g->g.nnz * 4);
  if (g->d_chk) cudaFree(g->d_chk);
  order_free(c, g);
  g->magic = 0;
  delete g;
}
}  // namespace bcl

extern "C" bc_status bc_destroy(void *handle) {
  if (Graph *g = as_graph(handle)) {
    Ctx *c = g->ctx;
    if (g->inflight.load() > 0 || server_graph_busy(c, g))
      return fail(BC_EAGAIN, "bc_destroy: graph has requests in flight");
    cudaSetDevice(c->device);
    server_forget_graph(c, g);
    {
      std::lock_guard<std::mutex> lk(c->mu);
      for (size_t i = 0; i < c->graphs.size(); i++)
        if (c->graphs[i] == g) {
          c->graphs.erase(c->graphs.begin() + i);
          break;
        }
    }
    graph_free(g);
    return BC_OK;
  }
  if (Ctx *c = as_ctx(handle)) {
    cudaSetDevice(c->device);
    server_stop(c);
    std::vector<Graph *> gs;
    {
      std::lock_guard<std::mutex> lk(c->mu);
      gs.swap(c->graphs);
    }
    for (Graph *g : gs) graph_free(g);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    c->magic = 0;
    delete c;
    return BC_OK;
  }
  return fail(BC_EINVAL, "bc_destroy: not a bc handle");
}

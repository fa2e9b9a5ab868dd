// Locality order of the tile path's sources.
//
// A tile runs T sources through one shared traversal: every (vertex, level) pair that any
// of its sources reaches is an entry of the tile's active lists, and every edge between
// consecutive levels carries the bit mask of the sources it serves.  Sources that lie close
// together in the graph put most vertices at the same or neighbouring depths, so their
// masks coincide: fewer entries per vertex, denser masks per hit, fewer hit edges for the
// same work.  The sum over the sources (Alg. 1's outer loop, BC additive over sources) does
// not depend on how they are grouped, so the grouping is a scheduling choice.
//
// The order: every source gets its distances to L landmark vertices (a seeded sample of the
// non-isolated vertices, found once per graph by one forward-only tile and kept as bytes),
// and the sources are sorted by that profile, lexicographically (ties by position in the
// given list).  Sources with equal profiles sit next to each other in the sorted list and
// land in the same tiles.  The order depends only on the graph and the source list, so
// results still repeat bit for bit.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "bc_internal.h"

namespace bcl {

std::vector<int64_t> sample_distinct(int64_t N, int64_t k, uint64_t seed);  // bc_tune.cu

constexpr int kLandmarks = 32;
constexpr uint64_t kLandmarkSeed = 0x1A4D3A12C0FFEEull;

struct OrderCache {
  const int32_t *rp = nullptr;  // the graph the distances belong to
  int L = 0;                    // landmarks (0: nothing to order by)
  uint8_t *d = nullptr;         // [L][n] distances, 255 = unreached or >= 255
  size_t bytes = 0;
  std::vector<uint8_t> h;       // host copy, [n][L] (serving), filled on first use
};

namespace {

__global__ void k_lm_pack(const int32_t *depth, size_t total, uint8_t *out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int d = depth[i];
    out[i] = (d < 0 || d > 254) ? (uint8_t)255 : (uint8_t)d;
  }
}

// key[i * L + t] = distance of source i from landmark t
__global__ void k_lm_gather(const uint8_t *d, int L, int n, const int32_t *src, int k, uint8_t *key) {
  const size_t total = (size_t)k * L;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t si = i / L, t = i % L;
    key[i] = d[t * (size_t)n + src[si]];
  }
}

bc_status build_cache(Graph *g, const DeviceGraph *dg, int T, cudaStream_t st, TileWS **ws, OrderCache *oc) {
  Ctx *c = g->ctx;
  const int32_t n = dg->n;
  std::vector<int32_t> rp((size_t)n + 1);
  BC_CUDA_TRY(cudaMemcpyAsync(rp.data(), dg->rp, rp.size() * 4, cudaMemcpyDeviceToHost, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int32_t> pool;
  for (int32_t v = 0; v < n; v++)
    if (rp[v + 1] > rp[v]) pool.push_back(v);
  oc->rp = dg->rp;
  oc->L = 0;
  if (pool.empty()) return BC_OK;
  const int L = (int)std::min<size_t>(kLandmarks, pool.size());
  std::vector<int64_t> idx = sample_distinct((int64_t)pool.size(), L, kLandmarkSeed);
  std::vector<int32_t> lm((size_t)L);
  for (int i = 0; i < L; i++) lm[i] = pool[(size_t)idx[i]];
  int32_t *d_lm = nullptr, *d_depth = nullptr;
  const size_t b_lm = (size_t)L * 4, b_depth = (size_t)L * n * 4, b_out = (size_t)L * n;
  bc_status s = c->mem.alloc((void **)&d_lm, b_lm);
  if (!s) s = c->mem.alloc((void **)&d_depth, b_depth);
  if (!s) s = c->mem.alloc((void **)&oc->d, b_out);
  if (!s && cudaMemcpyAsync(d_lm, lm.data(), b_lm, cudaMemcpyHostToDevice, st) != cudaSuccess)
    s = fail(BC_ECUDA, "source order: copy of the landmarks");
  if (!s) {  // one forward-only tile from the landmarks: their distances to every vertex
    TileArgs ta{};
    ta.g = dg;
    ta.src = d_lm;
    ta.nsrc = L;
    ta.T = T;
    ta.loop_mode = 0;
    ta.alpha = 0.5f;
    ta.out_depth = d_depth;
    s = tile_run(c, g, ws, ta, st, nullptr);
  }
  if (!s) {
    k_lm_pack<<<c->num_sms * 4, 256, 0, st>>>(d_depth, (size_t)L * n, oc->d);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_fail(e, "source order: landmark distances");
  }
  if (!s) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "source order: landmark distances");
  }
  if (d_lm) c->mem.release(d_lm, b_lm);
  if (d_depth) c->mem.release(d_depth, b_depth);
  if (s) {
    if (oc->d) c->mem.release(oc->d, b_out);
    oc->d = nullptr;
    oc->rp = nullptr;
    return s;
  }
  oc->L = L;
  oc->bytes = b_out;
  return BC_OK;
}

}  // namespace

void order_free(Ctx *c, Graph *g) {
  for (OrderCache *&oc : g->order) {
    if (!oc) continue;
    if (oc->d) c->mem.release(oc->d, oc->bytes);
    delete oc;
    oc = nullptr;
  }
}

namespace {

// The graph's cache (built on first use)
bc_status cache_for(Graph *g, const DeviceGraph *dg, int T, cudaStream_t st, TileWS **ws, OrderCache **out) {
  Ctx *c = g->ctx;
  OrderCache *oc = nullptr;
  for (OrderCache *x : g->order)
    if (x && x->rp == dg->rp) oc = x;
  if (!oc) {
    // an empty slot, else the one not holding the handle's own graph (whose host copy serving
    // keeps using): a cache for an earlier residual graph is replaced
    int si = !g->order[0] ? 0 : !g->order[1] ? 1 : (g->order[0]->rp == g->g.rp ? 1 : 0);
    OrderCache *&slot = g->order[si];
    if (slot) {
      if (slot->d) c->mem.release(slot->d, slot->bytes);
      delete slot;
    }
    slot = new (std::nothrow) OrderCache();
    if (!slot) return fail(BC_ENOMEM, "source order: host allocation failed");
    oc = slot;
    bc_status s = build_cache(g, dg, T, st, ws, oc);
    if (s) return s;
  }
  *out = oc;
  return BC_OK;
}

}  // namespace

bc_status order_host_keys(Graph *g, const DeviceGraph *dg, int T, cudaStream_t st, TileWS **ws,
                          const uint8_t **keys, int *L) {
  *keys = nullptr;
  *L = 0;
  OrderCache *oc = nullptr;
  bc_status s = cache_for(g, dg, T, st, ws, &oc);
  if (s || oc->L == 0) return s;
  const size_t n = (size_t)dg->n, Lc = (size_t)oc->L;
  if (oc->h.empty()) {
    std::vector<uint8_t> t(Lc * n);
    cudaError_t e = cudaMemcpyAsync(t.data(), oc->d, t.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "source order: copy of the landmark distances");
    std::vector<uint8_t> h(Lc * n);
    for (size_t l = 0; l < Lc; l++)
      for (size_t v = 0; v < n; v++) h[v * Lc + l] = t[l * n + v];
    oc->h.swap(h);
  }
  *keys = oc->h.data();
  *L = oc->L;
  return BC_OK;
}

bc_status order_sources(Graph *g, const DeviceGraph *dg, const int32_t *d_src, int32_t k, int T, cudaStream_t st,
                        int32_t **out, size_t *out_bytes) {
  Ctx *c = g->ctx;
  *out = nullptr;
  *out_bytes = 0;
  OrderCache *oc = nullptr;
  {
    const bc_status s0 = cache_for(g, dg, T, st, &g->tile, &oc);
    if (s0) return s0;
  }
  if (oc->L == 0) return BC_OK;
  const int L = oc->L;
  uint8_t *d_key = nullptr;
  const size_t b_key = (size_t)k * L;
  bc_status s = c->mem.alloc((void **)&d_key, b_key);
  if (s) return s;
  std::vector<uint8_t> key(b_key);
  std::vector<int32_t> hsrc((size_t)k);
  k_lm_gather<<<c->num_sms * 4, 256, 0, st>>>(oc->d, L, dg->n, d_src, k, d_key);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(key.data(), d_key, b_key, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hsrc.data(), d_src, (size_t)k * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  c->mem.release(d_key, b_key);
  if (e != cudaSuccess) return cuda_fail(e, "source order: landmark profiles");
  std::vector<int32_t> perm((size_t)k);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
    return memcmp(&key[(size_t)a * L], &key[(size_t)b * L], (size_t)L) < 0;
  });
  std::vector<int32_t> sorted((size_t)k);
  for (int32_t i = 0; i < k; i++) sorted[i] = hsrc[perm[i]];
  int32_t *d_out = nullptr;
  s = c->mem.alloc((void **)&d_out, (size_t)k * 4);
  if (s) return s;
  e = cudaMemcpyAsync(d_out, sorted.data(), (size_t)k * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vector goes out of scope
  if (e != cudaSuccess) {
    c->mem.release(d_out, (size_t)k * 4);
    return cuda_fail(e, "source order: copy of the ordered sources");
  }
  *out = d_out;
  *out_bytes = (size_t)k * 4;
  return BC_OK;
}

}  // namespace bcl

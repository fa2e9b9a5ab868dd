// Autotuner: times candidate configurations on a seeded probe of the graph's sources and
// keeps the fastest on the graph: tile width, the direction-switch thresholds (top-down ->
// bottom-up alpha, bottom-up -> top-down beta), level-loop mode, the hub degree and hub
// chunk of the tile path's load balance, or the per-source path (and its beta).  Optionally
// persisted in a JSON-lines cache file (BC_TUNE_CACHE) keyed by GPU name and a graph
// signature.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

#include "bc_internal.h"

namespace bcl {

// SplitMix64 (Steele, Lea, Flood 2014): the generator behind seeded source draws.
uint64_t splitmix64_next(uint64_t &x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// k distinct indices of [0, N) (Floyd's algorithm), uniform given the seed; sorted.
std::vector<int64_t> sample_distinct(int64_t N, int64_t k, uint64_t seed) {
  std::vector<int64_t> out;
  if (k > N) k = N;
  std::unordered_set<int64_t> seen;
  seen.reserve((size_t)k * 2 + 1);
  uint64_t x = seed;
  for (int64_t j = N - k; j < N; j++) {
    const uint64_t r = splitmix64_next(x);
    const int64_t t = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(j + 1)) >> 64);
    if (seen.count(t)) {
      seen.insert(j);
      out.push_back(j);
    } else {
      seen.insert(t);
      out.push_back(t);
    }
  }
  std::sort(out.begin(), out.end());
  return out;
}

// Host list of the non-isolated vertices of g (cached on the graph).
bc_status nonisolated_host(Graph *g, std::vector<int32_t> &out) {
  if (g->h_deg_nonisolated.empty() && g->n_nonisolated > 0) {
    std::vector<int32_t> rp((size_t)g->g.n + 1);
    BC_CUDA_TRY(cudaMemcpy(rp.data(), g->g.rp, rp.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<int32_t> v;
    v.reserve((size_t)g->n_nonisolated);
    for (int32_t i = 0; i < g->g.n; i++)
      if (rp[i + 1] > rp[i]) v.push_back(i);
    g->h_deg_nonisolated.swap(v);
  }
  out = g->h_deg_nonisolated;
  return BC_OK;
}

namespace {

struct Probe {
  Graph *g;
  int32_t *d_src;
  int32_t k;
  double *d_bc;
  cudaStream_t st;
};

struct Cfg {
  int T;            // tile width; 0 = per-source path (kernel by size), -1 = one source per CTA
  float alpha;
  float beta;       // tile: 0 = no hysteresis; per-source path: n / beta frontier test
  int loop_mode;
  int hub, chunk;   // tile path load balance
};

// seconds per source of one configuration (best of two runs)
bc_status time_config(const Probe &pr, const Cfg &c, double *sec_per_src) {
  const int T = c.T;
  const float alpha = c.alpha;
  double best = 1e30;
  for (int rep = 0; rep < 2; rep++) {
    bc_stats s{};
    bc_status r;
    if (T <= 0) {  // per-source path: 0 = the kernel chosen by size, -1 = one source per CTA
      const bool cta = T < 0 || cta_fits(pr.g->g.n);
      PlainArgs pa{};
      pa.g = &pr.g->g;
      pa.src = pr.d_src;
      // the grid-wide kernel is timed on fewer sources; the per-CTA kernel needs enough
      // sources to fill the GPU
      pa.nsrc = cta ? pr.k : (pr.k < 32 ? pr.k : 32);
      pa.bc = pr.d_bc;
      pa.max_degree = pr.g->max_degree;
      pa.alpha = alpha;
      pa.beta = c.beta > 0.f ? c.beta : 24.f;
      if (cta) {
        r = cta_run(pr.g->ctx, pr.g, &pr.g->cta, pa, pr.st, &s);
      } else {
        r = plain_ensure(pr.g->ctx, &pr.g->plain, pr.g->g.n);
        if (!r) r = plain_run(pr.g->ctx, &pr.g->plain, pa, pr.st, &s);
      }
    } else {
      TileArgs ta{};
      ta.g = &pr.g->g;
      ta.src = pr.d_src;
      ta.nsrc = pr.k;
      ta.bc = pr.d_bc;
      ta.T = T;
      ta.loop_mode = c.loop_mode;
      ta.alpha = alpha;
      ta.beta = c.beta;
      ta.hub = c.hub;
      ta.hub_chunk = c.chunk;
      r = tile_run(pr.g->ctx, pr.g, &pr.g->tile, ta, pr.st, &s);
    }
    if (r) return r;
    if (s.sources > 0 && s.seconds / (double)s.sources < best) best = s.seconds / (double)s.sources;
  }
  *sec_per_src = best;
  return BC_OK;
}

std::string gpu_name(int dev) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  return prop.name;
}

std::string cache_key(Graph *g) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|n=%d|nnz=%lld|maxdeg=%d|nonisolated=%lld",
           gpu_name(g->ctx->device).c_str(), g->g.n, (long long)g->g.nnz, g->max_degree,
           (long long)g->n_nonisolated);
  return buf;
}

bool cache_lookup(const std::string &key, bc_tune_result *res) {
  const char *path = getenv("BC_TUNE_CACHE");
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    const char *k = strstr(line, "\"key\": \"");
    if (!k) continue;
    k += 8;
    if (strncmp(k, key.c_str(), key.size()) != 0 || k[key.size()] != '"') continue;
    bc_tune_result r{};
    const char *p;
    if ((p = strstr(line, "\"tile_width\": "))) r.tile_width = atoi(p + 14);
    if ((p = strstr(line, "\"alpha\": "))) r.alpha = (float)atof(p + 9);
    if ((p = strstr(line, "\"beta\": "))) r.beta = (float)atof(p + 8);
    if ((p = strstr(line, "\"loop_mode\": "))) r.loop_mode = atoi(p + 13);
    if ((p = strstr(line, "\"plain_cta\": "))) r.plain_cta = atoi(p + 13);
    if ((p = strstr(line, "\"hub_degree\": "))) r.hub_degree = atoi(p + 14);
    if ((p = strstr(line, "\"hub_chunk\": "))) r.hub_chunk = atoi(p + 13);
    *res = r;
    found = true;  // the last matching line wins
  }
  fclose(f);
  return found;
}

void cache_store(const std::string &key, const bc_tune_result &r) {
  const char *path = getenv("BC_TUNE_CACHE");
  if (!path) return;
  if (FILE *f = fopen(path, "a")) {
    fprintf(f, "{\"key\": \"%s\", \"tile_width\": %d, \"alpha\": %.4f, \"beta\": %.2f, \"loop_mode\": %d, \"plain_cta\": %d, \"hub_degree\": %d, \"hub_chunk\": %d, \"probe_seconds\": %.3f}\n",
            key.c_str(), r.tile_width, r.alpha, r.beta, r.loop_mode, r.plain_cta, r.hub_degree, r.hub_chunk,
            r.probe_seconds);
    fclose(f);
  }
}

}  // namespace
}  // namespace bcl

using namespace bcl;

extern "C" bc_status bc_autotune(bc_graph *graph, int32_t probe_sources, uint64_t seed,
                                 bc_tune_result *out) {
  Graph *g = (Graph *)graph;
  if (!g || g->magic != kGraphMagic || !out) return fail(BC_EINVAL, "bc_autotune: bad argument");
  if (probe_sources < 0) return fail(BC_EINVAL, "bc_autotune: probe_sources < 0");
  Ctx *c = g->ctx;
  BC_CUDA_TRY(cudaSetDevice(c->device));
  std::lock_guard<std::mutex> lk(g->mu);
  const std::string key = cache_key(g);
  bc_tune_result res{};
  if (cache_lookup(key, &res)) {
    g->tune.res = res;
    g->tune.ready = true;
    *out = res;
    return BC_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int32_t> pool;
  bc_status s = nonisolated_host(g, pool);
  if (s) return s;
  if (pool.empty()) {
    res.tile_width = 0;
    res.alpha = 0.5f;
    res.beta = 24.f;
    g->tune.res = res;
    g->tune.ready = true;
    *out = res;
    return BC_OK;
  }
  const int32_t k = (int32_t)std::min<int64_t>(probe_sources ? probe_sources : 256, (int64_t)pool.size());
  std::vector<int64_t> idx = sample_distinct((int64_t)pool.size(), k, seed ^ 0xB1CE5EEDull);
  std::vector<int32_t> hs(idx.size());
  for (size_t i = 0; i < idx.size(); i++) hs[i] = pool[(size_t)idx[i]];
  Probe pr{g, nullptr, (int32_t)hs.size(), nullptr, c->own_stream};
  s = c->mem.alloc((void **)&pr.d_src, hs.size() * 4 + 4);
  if (s) return s;
  s = c->mem.alloc((void **)&pr.d_bc, (size_t)g->g.n * 8);
  if (s) {
    c->mem.release(pr.d_src, hs.size() * 4 + 4);
    return s;
  }
  const cudaError_t ce = cudaMemcpy(pr.d_src, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    c->mem.release(pr.d_src, hs.size() * 4 + 4);
    c->mem.release(pr.d_bc, (size_t)g->g.n * 8);
    return cuda_fail(ce, "bc_autotune: copy of the probe sources");
  }
  {  // the tile path runs a call's sources grouped by locality: so do the probes
    int32_t *osrc = nullptr;
    size_t ob = 0;
    s = order_sources(g, &g->g, pr.d_src, pr.k, 64, pr.st, &osrc, &ob);
    if (!s && osrc) {
      const cudaError_t oe = cudaMemcpyAsync(pr.d_src, osrc, (size_t)pr.k * 4, cudaMemcpyDeviceToDevice, pr.st);
      cudaStreamSynchronize(pr.st);
      c->mem.release(osrc, ob);
      if (oe != cudaSuccess) s = cuda_fail(oe, "bc_autotune: ordered probe sources");
    }
    if (s) {
      c->mem.release(pr.d_src, hs.size() * 4 + 4);
      c->mem.release(pr.d_bc, (size_t)g->g.n * 8);
      return s;
    }
  }
  double best = 1e30, t;
  Cfg cur{64, 0.2f, 0.f, 0, 512, 256};
  // a later stage's value replaces the current one only when it is clearly faster (2%):
  // timing noise must not pick a threshold
  auto stage = [&](auto set, std::initializer_list<double> vals, double margin) {
    for (double v : vals) {
      if (s) return;
      Cfg c = cur;
      set(c, v);
      s = time_config(pr, c, &t);
      if (!s && t < best * margin) best = t, cur = c;
    }
  };
  // stage 1: tile width
  stage([](Cfg &c, double v) { c.T = (int)v; }, {32, 64, 128, 256}, 1.0);
  // stage 2: top-down -> bottom-up threshold of the tile path
  stage([](Cfg &c, double v) { c.alpha = (float)v; }, {0.02, 0.05, 0.5, 2.0}, 1.0);
  // stage 3: level-loop mode (matters on long-diameter graphs)
  stage([](Cfg &c, double v) { c.loop_mode = (int)v; }, {1, 2}, 0.97);
  // stage 4: bottom-up -> top-down hysteresis (0 = none)
  stage([](Cfg &c, double v) { c.beta = (float)v; }, {4, 16}, 0.98);
  // stage 5: load balance of high-degree vertices (forward: degree from which a candidate is
  // split into warp work items; backward: edges per work item of a split entry)
  stage([](Cfg &c, double v) { c.hub = (int)v; }, {1024, 2048}, 0.98);
  stage([](Cfg &c, double v) { c.chunk = (int)v; }, {512, 1024}, 0.98);
  // stage 6: the per-source path (the kernel chosen by size, and on larger graphs also one
  // source per CTA, which suits sparse high-diameter graphs); the grid-wide kernel's beta
  double tplain = 1e30, tcta = 1e30;
  float pbeta = 24.f;
  if (!s) s = time_config(pr, Cfg{0, 0.5f, 24.f, 0, 0, 0}, &tplain);
  const bool grid_kernel = !cta_fits(g->g.n);
  if (!s && grid_kernel && tplain < best) {
    for (float b : {8.f, 64.f}) {
      if (s) break;
      s = time_config(pr, Cfg{0, 0.5f, b, 0, 0, 0}, &t);
      if (!s && t < tplain * 0.98) tplain = t, pbeta = b;
    }
  }
  if (!s && grid_kernel && g->g.n <= kCtaForcedMaxN) s = time_config(pr, Cfg{-1, 0.5f, 24.f, 0, 0, 0}, &tcta);
  c->mem.release(pr.d_src, hs.size() * 4 + 4);
  c->mem.release(pr.d_bc, (size_t)g->g.n * 8);
  if (s) return s;
  if (std::min(tplain, tcta) < best) {
    res.tile_width = 0;
    res.alpha = 0.5f;
    res.beta = pbeta;
    res.loop_mode = 0;
    res.plain_cta = tcta < tplain ? 1 : 0;
  } else {
    res.tile_width = cur.T;
    res.alpha = cur.alpha;
    res.beta = cur.beta;
    res.loop_mode = cur.loop_mode;
    res.hub_degree = cur.hub;
    res.hub_chunk = cur.chunk;
  }
  res.probe_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  g->tune.res = res;
  g->tune.ready = true;
  cache_store(key, res);
  *out = res;
  return BC_OK;
}

extern "C" bc_status bc_sample_sources(bc_graph *graph, int32_t k, uint64_t seed, int32_t *src_out) {
  Graph *g = (Graph *)graph;
  if (!g || g->magic != kGraphMagic || !src_out || k < 0)
    return fail(BC_EINVAL, "bc_sample_sources: bad argument");
  std::vector<int32_t> pool;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    BC_CUDA_TRY(cudaSetDevice(g->ctx->device));
    bc_status s = nonisolated_host(g, pool);
    if (s) return s;
  }
  if ((int64_t)k > (int64_t)pool.size())
    return fail(BC_EINVAL, "bc_sample_sources: k exceeds the number of non-isolated vertices");
  std::vector<int64_t> idx = sample_distinct((int64_t)pool.size(), k, seed);
  for (int32_t i = 0; i < k; i++) src_out[i] = pool[(size_t)idx[i]];
  return BC_OK;
}

// Host-side internals of libbc.so (product code only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bc.h"
#include "bc_common.cuh"

namespace bcl {

constexpr uint32_t kCtxMagic = 0xBC0C7A11u;
constexpr uint32_t kGraphMagic = 0xBC06AF11u;

void set_error(const std::string &msg);
bc_status fail(bc_status st, const std::string &msg);
bc_status cuda_fail(cudaError_t e, const char *what);

#define BC_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return bcl::cuda_fail(e_, #expr); \
  } while (0)

// Tracks the library's own device memory against the context budget.
struct DevMem {
  std::atomic<size_t> used{0};
  size_t budget = 0;  // 0 = unlimited
  bc_status alloc(void **p, size_t bytes);  // p == nullptr: reserve only
  void release(void *p, size_t bytes);      // p == nullptr: unreserve only
};

// Control block of one traversal workspace (device memory).
constexpr int kPlainScanBlocks = 1024;  // CTAs of the per-source kernel the rescan supports
struct PlainCtl {
  unsigned long long qpack;  // packed queue/edge append counter
  unsigned long long ns;     // component size incl. removed leaves (Eq. 3's n)
  GridSync bar;
  unsigned long long sigmax[2];  // largest sigma of level l (slot l & 1)
  int level_ovf[2];          // some vertex of level l overflowed 2^64 (slot l & 1)
  int src_ovf;               // some vertex of the current source overflowed
  int max_depth;
  long long ovf_sources;
  long long levels;
  long long reached;
  long long reached_arcs;
  int trace_n;
  int pad1;
  int scan_blk[kPlainScanBlocks];  // per-CTA degree sums of a level (BC_NO_CD_REUSE)
};

// Per-source path workspace for a graph of n vertices (Sec. 3.1/3.2 data structures:
// queue Q with level offsets Q_off, degree prefix CD, depth d, sigma, bitmaps, delta).
struct PlainWS {
  int32_t n = 0;
  int32_t *depth = nullptr;    // [n]  -1 = unvisited
  int32_t *Q = nullptr;        // [n]  BFS queue, also the stack of Alg. 1
  int32_t *CD = nullptr;       // [n]  exclusive prefix of degrees in Q order
  int32_t *lvl_off = nullptr;  // [n+2] Q offset of each level
  int32_t *lvl_eoff = nullptr; // [n+2] CD value at each level start
  unsigned long long *sig = nullptr;  // [n] sigma mod 2^64
  uint32_t *ovf = nullptr;     // [nw] overflow bits
  uint32_t *vis = nullptr;     // [nw] visited-before-this-level bits
  uint32_t *front = nullptr;   // [nw] frontier bits (bottom-up)
  unsigned long long *acc = nullptr;  // [2n] successor sums of Alg. 5 (64.64 fixed point)
  double *r = nullptr;         // [n] (1 + delta + omega) / sigma
  double *xm = nullptr;        // [n] extended-range sigma: mantissa
  int32_t *xe = nullptr;       // [n] extended-range sigma: exponent
  PlainCtl *ctl = nullptr;
  size_t bytes = 0;
};

struct DeviceGraph {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t *rp = nullptr;
  int32_t *ci = nullptr;
};

struct TileWS;      // bc_tile.cu
struct CtaWS;       // bc_cta.cu
struct OrderCache;  // bc_order.cu

struct PruneCache {
  bool ready = false;
  DeviceGraph res;        // residual CSR (same vertex ids)
  int32_t *omega = nullptr;
  uint8_t *removed = nullptr;
  int32_t *src = nullptr; // non-removed vertices (the sources of the pruned run)
  int32_t nsrc = 0;
  int64_t n_removed = 0;
};

struct TuneCache {
  bool ready = false;
  bc_tune_result res{};
};

struct Ctx;

struct Graph {
  uint32_t magic = kGraphMagic;
  Ctx *ctx = nullptr;
  DeviceGraph g;
  int64_t n_nonisolated = 0;
  int32_t max_degree = 0;
  std::mutex mu;           // serialises direct calls on this graph's workspaces
  std::atomic<int> inflight{0};
  PlainWS plain;
  PruneCache prune;
  TuneCache tune;
  TileWS *tile = nullptr;  // tile-path workspace (bc_tile.cu)
  CtaWS *cta = nullptr;    // per-source path on small graphs (bc_cta.cu)
  std::vector<int32_t> h_deg_nonisolated;  // host copy for sampled requests
  int *d_chk = nullptr;    // device words for argument checks (16 bytes, graph's lifetime)
  OrderCache *order[2] = {nullptr, nullptr};  // landmark distances (graph, residual graph)
};

struct Server;  // bc_serve.cu

struct Ctx {
  uint32_t magic = kCtxMagic;
  int device = 0;
  int num_sms = 0;
  DevMem mem;
  uint64_t wait_limit_ns = 20ull * 1000 * 1000 * 1000;
  std::mutex mu;
  std::vector<Graph *> graphs;
  Server *server = nullptr;
  cudaStream_t own_stream = nullptr;
};

// ---- per-source path (bc_plain.cu)
struct PlainArgs {
  const DeviceGraph *g;
  const int32_t *omega;   // nullable: Eq. 4 weights (pruned run)
  const int32_t *src;     // device
  int32_t nsrc;
  double *bc;             // device [n], accumulated into
  bool leaf_term;
  int32_t max_degree;     // bound used to prove a level cannot overflow 2^64
  // bc_sssp outputs (device), non-null => forward only for src[0]
  int32_t *out_depth;
  unsigned long long *out_sigma;
  uint8_t *out_ovf;
  float alpha;
  float beta;
  // per-source path on small graphs only: 2-degree triples (a, b, c) run as one unit,
  // c's DAG derived from those of a and b (device, 3 ints each)
  const int32_t *tri;
  int32_t ntri;
  // grid-wide kernel only: rescan each level's degree prefix in the backward sweep
  // instead of reusing the forward's (ablation of Sec. 3.1's reuse)
  bool no_cd_reuse;
  // per-CTA kernel (serving): the sources of nreq requests in one call, request q's being
  // the next h_req_k[q] entries of src (host array); each request gets its own CTAs and
  // its BC goes to req_bc[q] (device array of nreq device pointers); bc is then unused
  int32_t nreq;
  const int32_t *h_req_k;
  double *const *req_bc;
};
bc_status plain_ensure(Ctx *ctx, PlainWS *ws, int32_t n);
void plain_free(Ctx *ctx, PlainWS *ws);
bc_status plain_run(Ctx *ctx, PlainWS *ws, const PlainArgs &a, cudaStream_t st, bc_stats *acc);
bc_status plain_run_view(const PlainWS &ws, const PlainArgs &a, int num_sms, uint64_t limit_ns,
                         cudaStream_t st, int *dev_err);

// ---- per-source path on small graphs: one CTA per source (bc_cta.cu)
constexpr int32_t kCtaMaxN = 65536;        // default for the per-source path up to this size
constexpr int32_t kCtaForcedMaxN = 1 << 24;  // BC_PLAIN_CTA / tuned: up to this size
constexpr int kCtaMaxReq = 32;  // requests per per-CTA launch (serving)
bool cta_fits(int32_t n);
// Runs a.src, one source per CTA (a.out_depth set: forward only for a.src[0], depth / sigma /
// overflow exported).
bc_status cta_run(Ctx *ctx, Graph *g, CtaWS **ws, const PlainArgs &a, cudaStream_t st, bc_stats *acc);
void cta_free(Ctx *ctx, CtaWS *ws);

// ---- device 1-degree preprocessing (bc_prune.cu)
bc_status prune_build(Ctx *ctx, Graph *g, cudaStream_t st);
void prune_free(Ctx *ctx, PruneCache *p);

// ---- tile path (bc_tile.cu)
struct TileArgs {
  const DeviceGraph *g;
  const int32_t *omega;
  const int32_t *src;     // device
  int32_t nsrc;
  double *bc;
  int32_t T;              // 32..256
  int32_t loop_mode;      // 0 persistent, 1 per-level launches, 2 CUDA graph
  float alpha;
  float beta;             // > 0: bottom-up hysteresis (see bc_tune_result); 0: alpha alone
  int32_t hub;            // 0 = default: degree from which CTAs split an adjacency
  int32_t hub_chunk;      // 0 = default: edges per backward hub work item
  int32_t *out_depth;     // tile sssp hook: [nsrc][n]
  unsigned long long *out_sigma;
  uint8_t *out_ovf;
  // serving: sources of several requests share a tile; lane_req[i] (device, aligned with
  // src) is the request slot of source i, req_bc[slot] (device) its BC buffer.  A tile's
  // lanes may only refer to slots < nreq (nreq = 0: everything goes to bc).
  int32_t nreq;
  const uint8_t *lane_req;
  double *const *req_bc;
};
bc_status tile_run(Ctx *ctx, Graph *g, TileWS **ws, const TileArgs &a, cudaStream_t st,
                   bc_stats *acc);
void tile_free(Ctx *ctx, TileWS *ws);

// ---- locality order of the tile path's sources (bc_order.cu)
// Sources sorted by their distances to seeded landmark vertices (computed once per graph):
// *out (k ints, device, allocated from the context budget; release *out_bytes) or nullptr
// when there is nothing to order by.
bc_status order_sources(Graph *g, const DeviceGraph *dg, const int32_t *d_src, int32_t k, int T,
                        cudaStream_t st, int32_t **out, size_t *out_bytes);
void order_free(Ctx *c, Graph *g);
// Host copy of the same profiles, [n][*L] bytes (source v's L distances at v * L), built on
// first use with tile workspace *ws (the caller holds g->mu); *keys = nullptr, *L = 0 when
// there is nothing to order by.  Valid until the graph is destroyed.
bc_status order_host_keys(Graph *g, const DeviceGraph *dg, int T, cudaStream_t st, TileWS **ws,
                          const uint8_t **keys, int *L);

// ---- common helpers (bc_api.cu)
int64_t plain_bytes(int32_t n);
bc_status run_sources(Graph *g, const int32_t *d_src, int32_t k, uint32_t flags,
                      const int32_t *omega, bool leaf_term, double *d_bc,
                      cudaStream_t st, bc_stats *stats, const DeviceGraph *dg);

}  // namespace bcl

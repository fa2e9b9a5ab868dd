// Device 1-degree preprocessing (Alg. 6 on one GPU; Eq. 3's omega).
//
// A vertex u with deg(u) = 1 whose only neighbour v has deg(v) >= 2 is removed and
// omega[v] counts it; both arcs (u,v) and (v,u) leave the graph (Sec. 3.4.1).  A K2
// component keeps both ends (removing both would lose the pair).  One removal round
// only (Sec. 3.4.1 footnote 1).  The residual CSR keeps the original vertex ids, so
// depths, sigma and BC of residual vertices are indexed as in the input graph.
#include "bc_internal.h"
#include "bc_scan.cuh"

namespace bcl {

namespace {

__global__ void k_mark_leaves(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *omega,
                              uint8_t *removed) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = rp[u];
    uint8_t rem = 0;
    if (rp[u + 1] - a == 1) {
      int32_t v = ci[a];
      if (rp[v + 1] - rp[v] >= 2) {
        rem = 1;
        atomicAdd(omega + v, 1);
      }
    }
    removed[u] = rem;
  }
}

__global__ void k_residual_degree(int32_t n, const int32_t *rp, const int32_t *ci,
                                  const uint8_t *removed, int32_t *rdeg) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = 0;
    if (!removed[u])
      for (int32_t e = rp[u]; e < rp[u + 1]; e++) c += !removed[ci[e]];
    rdeg[u] = c;
  }
}

__global__ void k_residual_fill(int32_t n, const int32_t *rp, const int32_t *ci,
                                const uint8_t *removed, const int32_t *rrp, int32_t *rci) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (removed[u]) continue;
    int32_t o = rrp[u];
    for (int32_t e = rp[u]; e < rp[u + 1]; e++) {
      int32_t v = ci[e];
      if (!removed[v]) rci[o++] = v;
    }
  }
}

// Sources of the pruned run: every non-removed vertex that has a residual edge or
// removed leaves (the latter still owes its deferred leaf term).
__global__ void k_pruned_sources(int32_t n, const uint8_t *removed, const int32_t *rrp,
                                 const int32_t *omega, int32_t *out, int *count) {
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = base + threadIdx.x;
    bool keep = u < n && !removed[u] && (rrp[u + 1] > rrp[u] || omega[u] > 0);
    unsigned m = __ballot_sync(BC_FULL, keep);
    int pos = 0;
    if ((threadIdx.x & 31) == 0 && m) pos = atomicAdd(count, __popc(m));
    pos = __shfl_sync(BC_FULL, pos, 0);
    if (keep) out[pos + __popc(m & lanemask_lt())] = (int32_t)u;
  }
}

int blocks_for(int64_t work, Ctx *c) {
  int64_t b = (work + 255) / 256, cap = (int64_t)c->num_sms * 16;
  return (int)(b < 1 ? 1 : b > cap ? cap : b);
}

}  // namespace

void prune_free(Ctx *ctx, PruneCache *p) {
  if (!p->omega) return;
  const size_t n = (size_t)p->res.n;
  ctx->mem.release(p->omega, n * 4);
  ctx->mem.release(p->removed, n);
  ctx->mem.release(p->src, n * 4 + 4);
  ctx->mem.release(p->res.rp, (n + 1) * 4);
  if (p->res.ci) ctx->mem.release(p->res.ci, (size_t)p->res.nnz * 4 + 4);
  *p = PruneCache();
}

bc_status prune_build(Ctx *ctx, Graph *g, cudaStream_t st) {
  if (g->prune.ready) return BC_OK;
  prune_free(ctx, &g->prune);
  PruneCache &p = g->prune;
  const int32_t n = g->g.n;
  const size_t N = (size_t)n;
  p.res.n = n;
  bc_status s = ctx->mem.alloc((void **)&p.omega, N * 4);
  if (!s) s = ctx->mem.alloc((void **)&p.removed, N);
  if (!s) s = ctx->mem.alloc((void **)&p.src, N * 4 + 4);
  if (!s) s = ctx->mem.alloc((void **)&p.res.rp, (N + 1) * 4);
  if (s) {
    if (p.omega) ctx->mem.release(p.omega, N * 4);
    if (p.removed) ctx->mem.release(p.removed, N);
    if (p.src) ctx->mem.release(p.src, N * 4 + 4);
    p = PruneCache();
    return s;
  }
  int32_t *rdeg = nullptr;
  int *d_cnt = nullptr;
  void *scratch = nullptr;
  size_t scratch_bytes = scan_scratch_bytes(n + 1);
  cudaError_t e = cudaMalloc(&rdeg, (N + 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_cnt, 16);
  if (e == cudaSuccess) e = cudaMalloc(&scratch, scratch_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.omega, 0, N * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rdeg, 0, (N + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 16, st);
  const int nb = blocks_for(n, ctx);
  if (e == cudaSuccess) {
    k_mark_leaves<<<nb, 256, 0, st>>>(n, g->g.rp, g->g.ci, p.omega, p.removed);
    k_residual_degree<<<nb, 256, 0, st>>>(n, g->g.rp, g->g.ci, p.removed, rdeg);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_exclusive_i32(rdeg, p.res.rp, n + 1, scratch, st);
  int32_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, p.res.rp + n, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    p.res.nnz = total;
    s = ctx->mem.alloc((void **)&p.res.ci, (size_t)total * 4 + 4);
    if (s) {
      cudaFree(rdeg);
      cudaFree(d_cnt);
      cudaFree(scratch);
      prune_free(ctx, &p);
      return s;
    }
    k_residual_fill<<<nb, 256, 0, st>>>(n, g->g.rp, g->g.ci, p.removed, p.res.rp, p.res.ci);
    k_pruned_sources<<<nb, 256, 0, st>>>(n, p.removed, p.res.rp, p.omega, p.src, d_cnt);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(rdeg);
  cudaFree(d_cnt);
  cudaFree(scratch);
  if (e != cudaSuccess) {
    prune_free(ctx, &p);
    return cuda_fail(e, "1-degree preprocessing");
  }
  // Sort the source list (the compaction order depends on warp scheduling): not needed
  // for correctness, but every call then gives the same sources to the same tiles and
  // CTAs.
  p.nsrc = h;
  std::vector<int32_t> hs(h);
  if (h) {
    BC_CUDA_TRY(cudaMemcpy(hs.data(), p.src, (size_t)h * 4, cudaMemcpyDeviceToHost));
    std::sort(hs.begin(), hs.end());
    BC_CUDA_TRY(cudaMemcpy(p.src, hs.data(), (size_t)h * 4, cudaMemcpyHostToDevice));
  }
  int64_t removed_cnt = 0;
  {
    std::vector<uint8_t> hr(N);
    BC_CUDA_TRY(cudaMemcpy(hr.data(), p.removed, N, cudaMemcpyDeviceToHost));
    for (uint8_t x : hr) removed_cnt += x;
  }
  p.n_removed = removed_cnt;
  p.ready = true;
  return BC_OK;
}

}  // namespace bcl

// Per-source path for small graphs: every CTA runs whole sources on its own.
//
// The method is Brandes' (Alg. 1) with the level-synchronous forward sweep of Alg. 2 /
// Alg. 3 and the successor-checking backward sweep of Alg. 4 / Alg. 5, one source at a
// time.  On a graph of a few thousand vertices a level holds far too little work for the
// whole GPU, and the grid-wide barriers of the per-source kernel dominate.  Here the loop
// over sources of Alg. 1 is spread over the CTAs (the coarse-grained parallelism of
// Sec. 3.3, applied to the SMs of one GPU): a CTA takes sources blockIdx.x, blockIdx.x +
// gridDim.x, ..., runs each with CTA barriers only, and keeps the source's depth, sigma,
// r and queue in shared memory when they fit (else in a per-CTA slice of global memory).
//
// Forward level l: a warp per frontier vertex v, lanes over its edges.  The
// compare-and-swap that discovers w returns the previous depth, and sigma[w] += sigma[v]
// (64-bit integer atomics, exact) whenever it was -1 or l, with a sticky overflow bit on a
// carry or an overflowed parent.  When a level overflowed, each overflowed vertex of it
// also gets its extended-range sigma (mantissa, exponent) summed over its parents.
// Backward level d: sigma of w is taken as m 2^e (m in [0.5, 1)), r is stored scaled by
// 2^e; a warp per vertex w of level d sums its successors' r, rescaled to w's exponent, in
// float-float arithmetic (lanes in edge order, then a fixed-order warp reduction); then
// delta = m * sum, r[w] = (1 + omega) / m + sum, and the CTA's BC partial of w grows by
// (omega[s] + 1) * delta.  A second kernel sums the partials in CTA order, so the result is
// deterministic.
#include <algorithm>
#include <cstring>

#include "bc_ff.cuh"
#include "bc_internal.h"

namespace bcl {

namespace {

constexpr int kCtaThreads = 512;
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr size_t kCtaSmemMax = 200 * 1024;  // per-CTA state kept in shared memory up to this

struct CtaK {
  int n;
  const int32_t *__restrict__ rp;
  const int32_t *__restrict__ ci;
  const int32_t *__restrict__ omega;
  const int32_t *__restrict__ src;
  int nsrc;
  int leaf_term;
  double *bcp;        // [gridDim.x][n] per-CTA BC partials
  char *gws;          // per-CTA global slices (state when not in shared memory, level offsets)
  size_t slice;       // bytes per slice
  int in_smem;        // state arrays in shared memory
  unsigned long long *stats;  // reached pairs, their arcs, levels, deepest level (max),
                              // sources whose sigma passed 2^64
  int32_t *out_depth;         // forward-only export of src[0] (sssp), or null
  unsigned long long *out_sigma;
  uint8_t *out_ovf;
};

// State of one source, n vertices: sigma u64 | r float2 | depth i32 | queue i32 | overflow
// bits.  The global slice of a CTA holds this state when it is not in shared memory, then
// the level offsets and the extended-range sigma (mantissa f64, exponent i32), touched
// only for overflowed vertices.
__host__ __device__ inline size_t cta_state_bytes(int n) {
  return ((size_t)n * 24 + ((size_t)(n + 31) / 32) * 4 + 16 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t cta_extra_bytes(int n) {
  return ((size_t)(n + 2) * 4 + 15) / 16 * 16 + (size_t)n * 12;
}

// sigma of v as m 2^e with m in [0.5, 1)
__device__ __forceinline__ XS cta_sigma(const unsigned long long *sig, const uint32_t *ovf,
                                        const double *xm, const int32_t *xe, int v) {
  if ((ovf[v >> 5] >> (v & 31)) & 1u) {
    XS x;
    x.m = xm[v];
    x.e = xe[v];
    return x;
  }
  return xs_u64(sig[v]);
}

__global__ void __launch_bounds__(kCtaThreads) k_cta_sources(CtaK p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = p.n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  char *gslice = p.gws + (size_t)blockIdx.x * p.slice;
  char *base = p.in_smem ? (char *)smem : gslice;
  unsigned long long *sig = (unsigned long long *)base;
  float2 *r = (float2 *)(base + (size_t)n * 8);
  int32_t *d = (int32_t *)(base + (size_t)n * 16);
  int32_t *Q = d + n;
  uint32_t *ovf = (uint32_t *)(Q + n);
  char *extra = gslice + (p.in_smem ? 0 : cta_state_bytes(n));
  int32_t *loff = (int32_t *)extra;
  double *xm = (double *)(extra + ((size_t)(n + 2) * 4 + 15) / 16 * 16);
  int32_t *xe = (int32_t *)(xm + n);
  double *bcp = p.bcp + (size_t)blockIdx.x * n;

  __shared__ int s_q, s_ovf, s_lovf[2];
  __shared__ unsigned long long s_ns;

  for (int v = tid; v < n; v += kCtaThreads) {
    sig[v] = 0ull;
    d[v] = -1;
    bcp[v] = 0.0;
  }
  for (int i = tid; i < (n + 31) / 32; i += kCtaThreads) ovf[i] = 0u;
  unsigned long long my_arcs = 0, my_reached = 0, my_levels = 0, my_deep = 0, my_ovf = 0;
  __syncthreads();

  for (int si = blockIdx.x; si < p.nsrc; si += gridDim.x) {
    const int s = p.src[si];
    if (tid == 0) {
      d[s] = 0;
      sig[s] = 1ull;
      Q[0] = s;
      loff[0] = 0;
      loff[1] = 1;
      s_q = 1;
      s_ovf = 0;
      s_lovf[1] = 0;
      s_ns = 1ull + (p.omega ? (unsigned long long)p.omega[s] : 0ull);
    }
    __syncthreads();
    // ---------------------------------------------------------------- forward
    int level = 1, q0 = 0, q1 = 1;
    unsigned long long src_arcs = 0;
    while (q1 > q0) {
      for (int i = q0 + wid; i < q1; i += kCtaWarps) {
        const int v = Q[i];
        const unsigned long long sv = sig[v];
        const bool ov = (ovf[v >> 5] >> (v & 31)) & 1u;
        const int e0 = p.rp[v], e1 = p.rp[v + 1];
        if (lane == 0) src_arcs += (unsigned long long)(e1 - e0);
        for (int e = e0 + lane; e < e1; e += 32) {
          const int w = p.ci[e];
          int dw = *(volatile int32_t *)&d[w];
          if (dw < 0) {
            const int old = atomicCAS(&d[w], -1, level);
            if (old < 0) {
              Q[atomicAdd(&s_q, 1)] = w;
              if (p.leaf_term && p.omega) atomicAdd(&s_ns, 1ull + (unsigned long long)p.omega[w]);
              dw = level;
            } else {
              dw = old;
            }
          }
          if (dw == level) {
            const unsigned long long old = atomicAdd(&sig[w], sv);
            if (old + sv < old || ov) {
              atomicOr(&ovf[w >> 5], 1u << (w & 31));
              s_ovf = 1;
              s_lovf[level & 1] = 1;
            }
          }
        }
      }
      __syncthreads();
      const int q2 = s_q;
      const bool lovf = s_lovf[level & 1] != 0;
      if (tid == 0) s_lovf[(level + 1) & 1] = 0;
      __syncthreads();
      if (tid == 0) loff[level + 1] = q2;
      if (lovf) {
        // extended-range sigma of the overflowed vertices of this level: the sum over the
        // parents (level - 1), lanes in edge order, then a fixed-order warp reduction
        for (int i = q1 + wid; i < q2; i += kCtaWarps) {
          const int w = Q[i];
          if (!((ovf[w >> 5] >> (w & 31)) & 1u)) continue;
          XS acc;
          acc.m = 0.0;
          acc.e = 0;
          const int e1 = p.rp[w + 1];
          for (int e = p.rp[w] + lane; e < e1; e += 32) {
            const int v = p.ci[e];
            if (d[v] == level - 1) xs_add(acc, cta_sigma(sig, ovf, xm, xe, v));
          }
#pragma unroll
          for (int off = 16; off >= 1; off >>= 1) {
            XS o;
            o.m = __shfl_down_sync(BC_FULL, acc.m, off);
            o.e = __shfl_down_sync(BC_FULL, acc.e, off);
            xs_add(acc, o);
          }
          if (lane == 0) {
            acc = xs_norm(acc);
            xm[w] = acc.m;
            xe[w] = acc.e;
          }
        }
        __syncthreads();
      }
      q0 = q1;
      q1 = q2;
      level++;
    }
    const int lmax = level - 2;  // deepest non-empty level
    const int qtot = q1;
    my_arcs += src_arcs;
    my_reached += (unsigned long long)qtot;
    my_levels += (unsigned long long)(level - 1);
    if ((unsigned long long)lmax > my_deep) my_deep = (unsigned long long)lmax;
    if (s_ovf) my_ovf++;

    if (p.out_depth) {  // forward-only export (sssp of src[0])
      for (int v = tid; v < n; v += kCtaThreads) {
        p.out_depth[v] = d[v];
        p.out_sigma[v] = sig[v];
        p.out_ovf[v] = (uint8_t)((ovf[v >> 5] >> (v & 31)) & 1u);
      }
    } else {
      // -------------------------------------------------------------- backward
      const float2 wsrc = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[s] : 0ull));
      for (int dd = lmax; dd >= 1; --dd) {
        const int a0 = loff[dd], a1 = loff[dd + 1];
        for (int i = a0 + wid; i < a1; i += kCtaWarps) {
          const int w = Q[i];
          const XS sw = cta_sigma(sig, ovf, xm, xe, w);
          float2 acc = make_float2(0.0f, 0.0f);
          if (dd < lmax) {
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w] + lane; e < e1; e += 32) {
              const int v = p.ci[e];
              if (d[v] != dd + 1) continue;
              const int ev = ((ovf[v >> 5] >> (v & 31)) & 1u) ? xe[v] : 64 - __clzll((long long)sig[v]);
              ff_add(acc, ff_scale(r[v], sw.e - ev));
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) ff_add(acc, ff_shfl_xor(acc, m));
          }
          if (lane == 0) {
            const float2 mw = ff_mant(sw.m);
            const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
            float2 rw = ff_mul(om1, ff_rcp(mw));
            ff_add(rw, acc);
            r[w] = rw;  // r scaled by 2^e of w
            const float2 dl = ff_mul(wsrc, ff_mul(mw, acc));
            if (!ff_zero(dl)) bcp[w] += ff_to(dl);
          }
        }
        __syncthreads();
      }
      if (tid == 0 && p.leaf_term && p.omega && p.omega[s] > 0) {
        const double om = (double)p.omega[s];
        bcp[s] += om * (2.0 * (double)s_ns - om - 3.0);
      }
    }
    // reset the reached vertices for the next source
    __syncthreads();
    for (int i = tid; i < qtot; i += kCtaThreads) {
      const int w = Q[i];
      d[w] = -1;
      sig[w] = 0ull;
      ovf[w >> 5] = 0u;
    }
    __syncthreads();
  }
  // statistics
  for (int m = 16; m >= 1; m >>= 1) my_arcs += __shfl_xor_sync(BC_FULL, my_arcs, m);
  if (lane == 0 && my_arcs) atomicAdd(&p.stats[1], my_arcs);
  if (tid == 0) {
    atomicAdd(&p.stats[0], my_reached);
    atomicAdd(&p.stats[2], my_levels);
    atomicMax(&p.stats[3], my_deep);
    if (my_ovf) atomicAdd(&p.stats[4], my_ovf);
  }
}

// bc[v] += sum over CTAs c (in order) of bcp[c][v]
__global__ void k_cta_reduce(const double *bcp, int ncta, int n, double *bc) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int c = 0; c < ncta; c++) sum += bcp[(size_t)c * n + v];
    if (sum != 0.0) bc[v] += sum;
  }
}

}  // namespace

struct CtaWS {
  int n = 0, ncta = 0, in_smem = 0;
  size_t slice = 0, smem = 0;
  double *bcp = nullptr;
  char *gws = nullptr;
  unsigned long long *stats = nullptr;
  size_t bytes = 0;
};

void cta_free(Ctx *ctx, CtaWS *ws) {
  if (!ws) return;
  cudaFree(ws->bcp);
  cudaFree(ws->gws);
  cudaFree(ws->stats);
  ctx->mem.release(nullptr, ws->bytes);
  delete ws;
}

static bc_status cta_ensure(Ctx *ctx, CtaWS **wsp, int n) {
  CtaWS *ws = *wsp;
  const size_t st = cta_state_bytes(n);
  const int in_smem = st <= kCtaSmemMax;
  const size_t smem = in_smem ? st : 0;
  int bps = 0;
  if (smem > 48 * 1024) {
    BC_CUDA_TRY(cudaFuncSetAttribute(k_cta_sources, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  BC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cta_sources, kCtaThreads, smem));
  if (bps < 1) return fail(BC_ECUDA, "CTA per-source kernel does not fit on an SM");
  if (!in_smem) bps = std::min(bps, 2);  // slices live in L2 / HBM: keep their total small
  int ncta = ctx->num_sms * bps;
  const size_t slice = ((in_smem ? 0 : st) + cta_extra_bytes(n) + 255) & ~(size_t)255;
  const size_t per_cta = (size_t)n * 8 + slice;
  if (ctx->mem.budget) {  // fewer CTAs when the context's HBM budget is tight
    const size_t used = ctx->mem.used.load() - (ws ? ws->bytes : 0);
    const size_t avail = ctx->mem.budget > used + 64 ? ctx->mem.budget - used - 64 : 0;
    ncta = (int)std::min<size_t>((size_t)ncta, avail / per_cta);
    if (ncta < 1) return fail(BC_ENOMEM, "CTA per-source workspace exceeds the context HBM budget");
  }
  if (ws && ws->n == n && ws->ncta == ncta) return BC_OK;
  if (ws) {
    cta_free(ctx, ws);
    *wsp = nullptr;
  }
  ws = new CtaWS();
  ws->n = n;
  ws->ncta = ncta;
  ws->in_smem = in_smem;
  ws->smem = smem;
  ws->slice = slice;
  const size_t b_bcp = (size_t)ncta * n * 8, b_gws = ws->slice * ncta;
  ws->bytes = b_bcp + b_gws + 64;
  bc_status s = ctx->mem.alloc(nullptr, ws->bytes);
  if (s) {
    delete ws;
    return s;
  }
  cudaError_t e = cudaMalloc((void **)&ws->bcp, b_bcp);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->gws, b_gws);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->stats, 64);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cta_free(ctx, ws);
    return fail(BC_ENOMEM, "CTA per-source workspace allocation failed");
  }
  *wsp = ws;
  return BC_OK;
}

bool cta_fits(int32_t n) { return n > 0 && n <= kCtaMaxN; }

bc_status cta_run(Ctx *ctx, Graph *g, CtaWS **wsp, const PlainArgs &a, cudaStream_t st, bc_stats *acc) {
  const DeviceGraph *dg = a.g;
  const int n = dg->n;
  const bool sssp = a.out_depth != nullptr;
  if (a.nsrc <= 0) return BC_OK;
  bc_status s = cta_ensure(ctx, wsp, n);
  if (s) return s;
  CtaWS *ws = *wsp;
  (void)g;
  CtaK p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.rp = dg->rp;
  p.ci = dg->ci;
  p.omega = a.omega;
  p.src = a.src;
  p.nsrc = sssp ? 1 : a.nsrc;
  p.leaf_term = a.leaf_term ? 1 : 0;
  p.bcp = ws->bcp;
  p.gws = ws->gws;
  p.slice = ws->slice;
  p.in_smem = ws->in_smem;
  p.stats = ws->stats;
  p.out_depth = a.out_depth;
  p.out_sigma = a.out_sigma;
  p.out_ovf = a.out_ovf;
  const int ncta = std::min(ws->ncta, p.nsrc);
  BC_CUDA_TRY(cudaMemsetAsync(ws->stats, 0, 64, st));
  cudaEvent_t e0, e1;
  BC_CUDA_TRY(cudaEventCreate(&e0));
  BC_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  k_cta_sources<<<ncta, kCtaThreads, ws->smem, st>>>(p);
  cudaError_t le = cudaGetLastError();
  if (le == cudaSuccess && !sssp && a.bc) {
    k_cta_reduce<<<ctx->num_sms * 4, 256, 0, st>>>(ws->bcp, ncta, n, a.bc);
    le = cudaGetLastError();
  }
  cudaEventRecord(e1, st);
  if (le != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(le, "CTA per-source kernel launch");
  }
  unsigned long long hs[5];
  cudaMemcpyAsync(hs, ws->stats, sizeof(hs), cudaMemcpyDeviceToHost, st);
  const cudaError_t se = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (se == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (se != cudaSuccess) return cuda_fail(se, "CTA per-source kernel");
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  if (acc) {
    acc->seconds += ms * 1e-3;
    acc->sources += p.nsrc;
    acc->sigma_overflow_sources += (int64_t)hs[4];
    acc->reached_vertices += (int64_t)hs[0];
    acc->reached_arcs += (int64_t)hs[1];
    acc->levels += (int64_t)hs[2];
    if ((int32_t)hs[3] > acc->max_depth) acc->max_depth = (int32_t)hs[3];
    acc->kernel_launches += sssp ? 1 : 2;
    if (acc->tile_width == 0) acc->tile_width = 1;
  }
  return BC_OK;
}

}  // namespace bcl

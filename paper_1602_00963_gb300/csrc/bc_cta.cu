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
// (omega[s] + 1) * delta.  A second kernel sums the partials in CTA order.  Every sum has a
// fixed order (a vertex's path depends on its degree only), so the result repeats bit for
// bit from run to run.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

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
  int clean;          // state in global memory already cleared (left clean by the last call)
  unsigned long long *stats;  // reached pairs, their arcs, levels, deepest level (max),
                              // sources whose sigma passed 2^64
  const int32_t *tri;         // 2-degree triples (a, b, c), 3 ints each
  int ntri;
  int32_t *out_depth;         // forward-only export of src[0] (sssp), or null
  unsigned long long *out_sigma;
  uint8_t *out_ovf;
  // several requests in one launch (nreq > 0): request q owns the sources
  // [req[q], req[q + 1]) and the CTAs [req[R + q], req[R + q + 1]), R = nreq + 1
  int nreq;
  const int32_t *req;
};

// State of one source, n vertices: sigma u64 | r float2 | depth i32 | queue i32 | overflow
// bits.  The global slice of a CTA holds this state when it is not in shared memory, then
// the level offsets and the extended-range sigma (mantissa f64, exponent i32), touched
// only for overflowed vertices.
__host__ __device__ inline size_t cta_state_bytes(int n) {
  return ((size_t)n * 24 + ((size_t)(n + 31) / 32) * 4 + 16 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t cta_extra_bytes(int n) {  // a multiple of 16: states follow
  return (((size_t)(n + 2) * 4 + 15) / 16 * 16 + (size_t)n * 12 + 15) & ~(size_t)15;
}

// One source's state: per-vertex arrays plus the level offsets and extended-range sigma.
struct CtaState {
  unsigned long long *sig;
  float2 *r;
  int32_t *d;
  int32_t *Q;
  uint32_t *ovf;
  int32_t *loff;
  double *xm;
  int32_t *xe;
};

// Carve a state: the per-vertex block at blk (cta_state_bytes), the rest at extra
// (cta_extra_bytes).
__device__ __forceinline__ CtaState cta_carve(char *blk, char *extra, int n) {
  CtaState S;
  S.sig = (unsigned long long *)blk;
  S.r = (float2 *)(blk + (size_t)n * 8);
  S.d = (int32_t *)(blk + (size_t)n * 16);
  S.Q = S.d + n;
  S.ovf = (uint32_t *)(S.Q + n);
  S.loff = (int32_t *)extra;
  S.xm = (double *)(extra + ((size_t)(n + 2) * 4 + 15) / 16 * 16);
  S.xe = (int32_t *)(S.xm + n);
  return S;
}

constexpr int kCtaLaneDeg = 32;  // vertices of degree <= this are handled by one thread
constexpr int kStage = 4;        // state in global memory: a thread's edges are loaded
                                 // kStage at a time (their latencies overlap)
constexpr int kStage2 = 2;       // the same for the 2-degree backward sweep
constexpr int kCtaBig = 512;     // higher-degree vertices listed per pass for whole warps

struct CtaShared {
  int q, ovf, lovf[2], nbig;
  unsigned long long ns;
  int big[kCtaBig];
};

// Entries Q[i0, i1): a vertex of degree <= kCtaLaneDeg is handled by one thread (a level of
// a sparse, high-diameter graph then keeps every thread busy), a larger one by a whole warp
// (lanes over its edges) from a shared list.  The entries are taken in windows of one per
// thread, so the list (kCtaBig >= kCtaThreads) never fills: which path handles a vertex, and
// so the order of its floating-point sums, depends on its degree only.
static_assert(kCtaBig >= kCtaThreads, "a window's high-degree vertices must fit the list");
template <typename LaneF, typename WarpF>
__device__ __forceinline__ void cta_split(const CtaK &p, const int32_t *Q, int i0, int i1, CtaShared &sh,
                                          LaneF &&lane_f, WarpF &&warp_f) {
  for (int b = i0; b < i1; b += kCtaThreads) {  // uniform over the CTA
    const int i = b + (int)threadIdx.x;
    if (i < i1) {
      const int v = Q[i];
      if (p.rp[v + 1] - p.rp[v] > kCtaLaneDeg)
        sh.big[atomicAdd(&sh.nbig, 1)] = v;
      else
        lane_f(v);
    }
    __syncthreads();
    const int nb = sh.nbig;
    __syncthreads();
    if (threadIdx.x == 0) sh.nbig = 0;
    for (int j = (int)(threadIdx.x >> 5); j < nb; j += kCtaWarps) warp_f(sh.big[j]);
    __syncthreads();
  }
}

// sigma of v as m 2^e with m in [0.5, 1)
__device__ __forceinline__ XS cta_sigma(const CtaState &S, int v) {
  if ((S.ovf[v >> 5] >> (v & 31)) & 1u) {
    XS x;
    x.m = S.xm[v];
    x.e = S.xe[v];
    return x;
  }
  return xs_u64(S.sig[v]);
}
__device__ __forceinline__ int cta_exp(const CtaState &S, int v) {
  return ((S.ovf[v >> 5] >> (v & 31)) & 1u) ? S.xe[v] : 64 - __clzll((long long)S.sig[v]);
}

__device__ void cta_clear(const CtaState &S, int n) {
  for (int v = threadIdx.x; v < n; v += kCtaThreads) {
    S.sig[v] = 0ull;
    S.d[v] = -1;
  }
  for (int i = threadIdx.x; i < (n + 31) / 32; i += kCtaThreads) S.ovf[i] = 0u;
}

// Forward sweep from s (Alg. 2 / Alg. 3, CTA barriers).  Returns the deepest non-empty
// level; *qtot = reached vertices, *arcs += their adjacency entries (lane 0 of each warp).
__device__ int cta_forward(const CtaK &p, const CtaState &S, int s, CtaShared &sh, int *qtot,
                           unsigned long long *arcs) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    S.d[s] = 0;
    S.sig[s] = 1ull;
    S.Q[0] = s;
    S.loff[0] = 0;
    S.loff[1] = 1;
    sh.q = 1;
    sh.ovf = 0;
    sh.lovf[1] = 0;
  }
  __syncthreads();
  int level = 1, q0 = 0, q1 = 1;
  while (q1 > q0) {
    // discover w from v (the compare-and-swap returns the previous depth) and add sigma
    auto edge = [&](int w, unsigned long long sv, bool ov) {
      int dw = *(volatile int32_t *)&S.d[w];
      if (dw < 0) {
        const int old = atomicCAS(&S.d[w], -1, level);
        if (old < 0) {
          S.Q[atomicAdd(&sh.q, 1)] = w;
          dw = level;
        } else {
          dw = old;
        }
      }
      if (dw == level) {
        const unsigned long long old = atomicAdd(&S.sig[w], sv);
        if (old + sv < old || ov) {
          atomicOr(&S.ovf[w >> 5], 1u << (w & 31));
          sh.ovf = 1;
          sh.lovf[level & 1] = 1;
        }
      }
    };
    cta_split(
        p, S.Q, q0, q1, sh,
        [&](int v) {
          // one thread: the edges in groups of kStage, each stage's loads and atomics of
          // the group in flight together
          const unsigned long long sv = S.sig[v];
          const bool ov = (S.ovf[v >> 5] >> (v & 31)) & 1u;
          const int e0 = p.rp[v], e1 = p.rp[v + 1];
          *arcs += (unsigned long long)(e1 - e0);
          if (p.in_smem) {  // state in shared memory: loads are cheap, no staging
            for (int e = e0; e < e1; e++) edge(p.ci[e], sv, ov);
            return;
          }
          for (int e = e0; e < e1; e += kStage) {
            int w[kStage], dw[kStage];
#pragma unroll
            for (int j = 0; j < kStage; j++) w[j] = e + j < e1 ? p.ci[e + j] : -1;
#pragma unroll
            for (int j = 0; j < kStage; j++) dw[j] = w[j] >= 0 ? *(volatile int32_t *)&S.d[w[j]] : INT_MAX;
#pragma unroll
            for (int j = 0; j < kStage; j++) {
              if (w[j] < 0 || dw[j] >= 0) continue;
              const int old = atomicCAS(&S.d[w[j]], -1, level);
              if (old < 0) {
                S.Q[atomicAdd(&sh.q, 1)] = w[j];
                dw[j] = level;
              } else {
                dw[j] = old;
              }
            }
            unsigned long long old[kStage];
#pragma unroll
            for (int j = 0; j < kStage; j++) old[j] = (w[j] >= 0 && dw[j] == level) ? atomicAdd(&S.sig[w[j]], sv) : 0ull;
#pragma unroll
            for (int j = 0; j < kStage; j++) {
              if (w[j] < 0 || dw[j] != level) continue;
              if (old[j] + sv < old[j] || ov) {
                atomicOr(&S.ovf[w[j] >> 5], 1u << (w[j] & 31));
                sh.ovf = 1;
                sh.lovf[level & 1] = 1;
              }
            }
          }
        },
        [&](int v) {
          const unsigned long long sv = S.sig[v];
          const bool ov = (S.ovf[v >> 5] >> (v & 31)) & 1u;
          const int e0 = p.rp[v], e1 = p.rp[v + 1];
          if (lane == 0) *arcs += (unsigned long long)(e1 - e0);
          for (int e = e0 + lane; e < e1; e += 32) edge(p.ci[e], sv, ov);
        });
    const int q2 = sh.q;
    const bool lovf = sh.lovf[level & 1] != 0;
    if (tid == 0) sh.lovf[(level + 1) & 1] = 0;
    __syncthreads();
    if (tid == 0) S.loff[level + 1] = q2;
    if (lovf) {
      // extended-range sigma of the overflowed vertices of this level: the sum over the
      // parents (level - 1) in edge order (warps: lanes in edge order, then a fixed-order
      // reduction)
      cta_split(
          p, S.Q, q1, q2, sh,
          [&](int w) {
            if (!((S.ovf[w >> 5] >> (w & 31)) & 1u)) return;
            XS acc;
            acc.m = 0.0;
            acc.e = 0;
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w]; e < e1 && p.in_smem; e++) {
              const int v = p.ci[e];
              if (S.d[v] == level - 1) xs_add(acc, cta_sigma(S, v));
            }
            for (int e = p.rp[w]; e < e1 && !p.in_smem; e += kStage) {
              int v[kStage];
              bool par[kStage];
              XS x[kStage];
#pragma unroll
              for (int j = 0; j < kStage; j++) v[j] = e + j < e1 ? p.ci[e + j] : -1;
#pragma unroll
              for (int j = 0; j < kStage; j++) par[j] = v[j] >= 0 && S.d[v[j]] == level - 1;
#pragma unroll
              for (int j = 0; j < kStage; j++)
                if (par[j]) x[j] = cta_sigma(S, v[j]);
#pragma unroll
              for (int j = 0; j < kStage; j++)
                if (par[j]) xs_add(acc, x[j]);
            }
            acc = xs_norm(acc);
            S.xm[w] = acc.m;
            S.xe[w] = acc.e;
          },
          [&](int w) {
            if (!((S.ovf[w >> 5] >> (w & 31)) & 1u)) return;
            XS acc;
            acc.m = 0.0;
            acc.e = 0;
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w] + lane; e < e1; e += 32) {
              const int v = p.ci[e];
              if (S.d[v] == level - 1) xs_add(acc, cta_sigma(S, v));
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
              S.xm[w] = acc.m;
              S.xe[w] = acc.e;
            }
          });
    }
    q0 = q1;
    q1 = q2;
    level++;
  }
  *qtot = q1;
  return level - 2;
}

// Backward sweep of s (Alg. 4 / Alg. 5): sigma of w taken as m 2^e, r stored scaled by 2^e.
__device__ void cta_backward(const CtaK &p, const CtaState &S, int s, int lmax, double *bcp,
                             CtaShared &sh) {
  const int tid = threadIdx.x, lane = tid & 31;
  const float2 wsrc = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[s] : 0ull));
  for (int dd = lmax; dd >= 1; --dd) {
    // commit of w from the sum of its successors' r (rescaled to w's exponent)
    auto commit = [&](int w, const XS &sw, float2 acc) {
      const float2 mw = ff_mant(sw.m);
      const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
      float2 rw = ff_mul(om1, ff_rcp(mw));
      ff_add(rw, acc);
      S.r[w] = rw;  // r scaled by 2^e of w
      const float2 dl = ff_mul(wsrc, ff_mul(mw, acc));
      if (!ff_zero(dl)) bcp[w] += ff_to(dl);
    };
    cta_split(
        p, S.Q, S.loff[dd], S.loff[dd + 1], sh,
        [&](int w) {
          const XS sw = cta_sigma(S, w);
          float2 acc = make_float2(0.0f, 0.0f);
          if (dd < lmax && p.in_smem) {
            for (int e = p.rp[w]; e < p.rp[w + 1]; e++) {
              const int v = p.ci[e];
              if (S.d[v] == dd + 1) ff_add(acc, ff_scale(S.r[v], sw.e - cta_exp(S, v)));
            }
          } else if (dd < lmax) {
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w]; e < e1; e += kStage) {
              int v[kStage];
              bool suc[kStage];
              float2 x[kStage];
              int ev[kStage];
#pragma unroll
              for (int j = 0; j < kStage; j++) v[j] = e + j < e1 ? p.ci[e + j] : -1;
#pragma unroll
              for (int j = 0; j < kStage; j++) suc[j] = v[j] >= 0 && S.d[v[j]] == dd + 1;
#pragma unroll
              for (int j = 0; j < kStage; j++) {
                x[j] = suc[j] ? S.r[v[j]] : make_float2(0.0f, 0.0f);
                ev[j] = suc[j] ? cta_exp(S, v[j]) : 0;
              }
#pragma unroll
              for (int j = 0; j < kStage; j++)
                if (suc[j]) ff_add(acc, ff_scale(x[j], sw.e - ev[j]));
            }
          }
          commit(w, sw, acc);
        },
        [&](int w) {
          const XS sw = cta_sigma(S, w);
          float2 acc = make_float2(0.0f, 0.0f);
          if (dd < lmax) {
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w] + lane; e < e1; e += 32) {
              const int v = p.ci[e];
              if (S.d[v] == dd + 1) ff_add(acc, ff_scale(S.r[v], sw.e - cta_exp(S, v)));
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) ff_add(acc, ff_shfl_xor(acc, m));
          }
          if (lane == 0) commit(w, sw, acc);
        });
  }
  if (tid == 0 && p.leaf_term && p.omega && p.omega[s] > 0) {
    const double om = (double)p.omega[s];
    bcp[s] += om * (2.0 * (double)sh.ns - om - 3.0);
  }
}

// n_s of Eq. 3: the reached vertices Q[0, qtot) weighted by 1 + omega (a source with
// omega(s) > 0 only; the sum is an integer, so its order does not matter).  Ends with a barrier.
__device__ void cta_weighted_size(const CtaK &p, const CtaState &S, int qtot, CtaShared &sh) {
  if (threadIdx.x == 0) sh.ns = 0ull;
  __syncthreads();
  unsigned long long part = 0ull;
  for (int i = threadIdx.x; i < qtot; i += kCtaThreads) part += 1ull + (unsigned long long)p.omega[S.Q[i]];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) part += __shfl_xor_sync(BC_FULL, part, m);
  if ((threadIdx.x & 31) == 0 && part) atomicAdd(&sh.ns, part);
  __syncthreads();
}

__device__ void cta_reset(const CtaState &S, int qtot) {
  __syncthreads();
  for (int i = threadIdx.x; i < qtot; i += kCtaThreads) {
    const int w = S.Q[i];
    S.d[w] = -1;
    S.sig[w] = 0ull;
    S.ovf[w >> 5] = 0u;
  }
  __syncthreads();
}

// ---- 2-degree vertex c with neighbours a, b (Sec. 3.4.2): its shortest-path DAG follows
// from those of a and b.  For v != c: level_c(v) = 1 + min(level_a(v), level_b(v)) and
// sigma_c(v) = sigma_a(v), sigma_b(v) or their sum as the smaller level comes from a, from b
// or from both (Eq. in Sec. 3.4.2, by the Bellman criterion); level_c(c) = 0, sigma_c(c) = 1.
__device__ __forceinline__ int deg2_level(const CtaState &A, const CtaState &B, int c, int v) {
  if (v == c) return 0;
  const int da = A.d[v], db = B.d[v];
  if (da < 0 && db < 0) return -1;
  if (da < 0) return db + 1;
  if (db < 0) return da + 1;
  return (da < db ? da : db) + 1;
}
__device__ __forceinline__ XS deg2_sigma(const CtaState &A, const CtaState &B, int c, int v) {
  if (v == c) return xs_u64(1ull);
  const int da = A.d[v], db = B.d[v];
  if (db < 0 || (da >= 0 && da < db)) return cta_sigma(A, v);
  if (da < 0 || db < da) return cta_sigma(B, v);
  XS x = cta_sigma(A, v);
  xs_add(x, cta_sigma(B, v));
  return xs_norm(x);
}

// exponent of sigma_c(v) as m 2^e (v != c)
__device__ __forceinline__ int deg2_exp(const CtaState &A, const CtaState &B, int v) {
  const int da = A.d[v], db = B.d[v];
  if (db < 0 || (da >= 0 && da < db)) return cta_exp(A, v);
  if (da < 0 || db < da) return cta_exp(B, v);
  XS x = cta_sigma(A, v);
  xs_add(x, cta_sigma(B, v));
  return xs_norm(x).e;
}

// Backward sweep of the 2-degree vertex c on its derived DAG, level by level (the dynamic
// merging of frontiers, Alg. 8 / Alg. 9): c's level D holds the vertices of a's level D - 1
// whose level from b is not smaller, and those of b's level D - 1 whose level from a is
// larger.  rc holds c's r values (scaled by 2^e of sigma_c).  On a residual graph (1-degree
// reduction) the leaf weights enter as in cta_backward; c, a and b share a component, so the
// weighted component size in sh.ns (set for the triple) is also c's.
__device__ void cta_backward_deg2(const CtaK &p, const CtaState &A, const CtaState &B, int lmaxA, int lmaxB,
                                  int c, float2 *rc, double *bcp, CtaShared &sh) {
  const int lane = threadIdx.x & 31;
  const int lmax = 1 + (lmaxA > lmaxB ? lmaxA : lmaxB);
  const float2 wsrc = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[c] : 0ull));
  auto commit = [&](int w, const XS &sw, float2 acc) {
    const float2 mw = ff_mant(sw.m);
    const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
    float2 rw = ff_mul(om1, ff_rcp(mw));
    ff_add(rw, acc);
    rc[w] = rw;
    const float2 dl = ff_mul(wsrc, ff_mul(mw, acc));
    if (!ff_zero(dl)) bcp[w] += ff_to(dl);
  };
  for (int D = lmax; D >= 1; --D) {
#pragma unroll 1
    for (int side = 0; side < 2; side++) {
      const CtaState &S = side ? B : A;
      const int lm = side ? lmaxB : lmaxA;
      if (D - 1 > lm) continue;
      // w belongs to c's level D through this side (ties go to a)
      auto mine = [&](int w) {
        if (w == c) return false;
        const int da = A.d[w], db = B.d[w];
        return side == 0 ? (db < 0 || da <= db) : (da < 0 || db < da);
      };
      cta_split(
          p, S.Q, S.loff[D - 1], S.loff[D], sh,
          [&](int w) {
            if (!mine(w)) return;
            const XS sw = deg2_sigma(A, B, c, w);
            float2 acc = make_float2(0.0f, 0.0f);
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w]; e < e1; e += kStage2) {
              int v[kStage2];
              bool suc[kStage2];
#pragma unroll
              for (int j = 0; j < kStage2; j++) v[j] = e + j < e1 ? p.ci[e + j] : -1;
#pragma unroll
              for (int j = 0; j < kStage2; j++) suc[j] = v[j] >= 0 && deg2_level(A, B, c, v[j]) == D + 1;
#pragma unroll
              for (int j = 0; j < kStage2; j++)
                if (suc[j]) ff_add(acc, ff_scale(rc[v[j]], sw.e - deg2_exp(A, B, v[j])));
            }
            commit(w, sw, acc);
          },
          [&](int w) {
            if (!mine(w)) return;
            const XS sw = deg2_sigma(A, B, c, w);
            float2 acc = make_float2(0.0f, 0.0f);
            const int e1 = p.rp[w + 1];
            for (int e = p.rp[w] + lane; e < e1; e += 32) {
              const int v = p.ci[e];
              if (deg2_level(A, B, c, v) != D + 1) continue;
              ff_add(acc, ff_scale(rc[v], sw.e - deg2_exp(A, B, v)));
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) ff_add(acc, ff_shfl_xor(acc, m));
            if (lane == 0) commit(w, sw, acc);
          });
    }
  }
  if (threadIdx.x == 0 && p.leaf_term && p.omega && p.omega[c] > 0) {
    const double om = (double)p.omega[c];
    bcp[c] += om * (2.0 * (double)sh.ns - om - 3.0);
  }
}

__global__ void __launch_bounds__(kCtaThreads, 2) k_cta_sources(CtaK p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = p.n;
  const int tid = threadIdx.x, lane = tid & 31;
  char *gslice = p.gws + (size_t)blockIdx.x * p.slice;
  const size_t sb = cta_state_bytes(n), xb = cta_extra_bytes(n);
  // state A: shared memory when it fits; state B and c's r (2-degree triples) after it
  char *g = gslice;
  char *blkA = p.in_smem ? (char *)smem : g;
  if (!p.in_smem) g += sb;
  const CtaState A = cta_carve(blkA, g, n);
  g += xb;
  CtaState B = A;
  float2 *rc = nullptr;
  if (p.ntri) {
    B = cta_carve(g, g + sb, n);
    rc = (float2 *)(g + sb + xb);
  }
  double *bcp = p.bcp + (size_t)blockIdx.x * n;
  __shared__ CtaShared sh;

  for (int v = tid; v < n; v += kCtaThreads) bcp[v] = 0.0;
  if (tid == 0) sh.nbig = 0;  // the big-vertex list of cta_split starts empty
  // every source resets the vertices it reached, so state in global memory stays clean from
  // one call to the next; shared memory starts undefined
  if (p.in_smem || !p.clean) cta_clear(A, n);
  if (p.ntri && !p.clean) cta_clear(B, n);
  unsigned long long my_arcs = 0, my_reached = 0, my_levels = 0, my_deep = 0, my_ovf = 0;
  __syncthreads();

  auto account = [&](int lmax, int qtot) {
    my_reached += (unsigned long long)qtot;
    my_levels += (unsigned long long)(lmax + 1);
    if ((unsigned long long)lmax > my_deep) my_deep = (unsigned long long)lmax;
    if (sh.ovf) my_ovf++;
  };
  int s0 = (int)blockIdx.x, s1 = p.nsrc, sstep = (int)gridDim.x;
  if (p.nreq > 0) {  // the sources of this CTA's request, strided over the request's CTAs
    const int32_t *rc = p.req + p.nreq + 1;
    int q = 0;
    while (q + 1 < p.nreq && (int)blockIdx.x >= rc[q + 1]) q++;
    s0 = p.req[q] + ((int)blockIdx.x - rc[q]);
    s1 = p.req[q + 1];
    sstep = rc[q + 1] - rc[q];
  }
  for (int si = s0; si < s1; si += sstep) {
    const int s = p.src[si];
    int qtot = 0;
    const int lmax = cta_forward(p, A, s, sh, &qtot, &my_arcs);
    account(lmax, qtot);
    if (p.leaf_term && p.omega && p.omega[s] > 0) cta_weighted_size(p, A, qtot, sh);
    if (p.out_depth) {  // forward-only export (sssp of src[0])
      for (int v = tid; v < n; v += kCtaThreads) {
        p.out_depth[v] = A.d[v];
        p.out_sigma[v] = A.sig[v];
        p.out_ovf[v] = (uint8_t)((A.ovf[v >> 5] >> (v & 31)) & 1u);
      }
    } else {
      cta_backward(p, A, s, lmax, bcp, sh);
    }
    cta_reset(A, qtot);
  }
  // 2-degree triples (a, b, c): a and b as usual, c from their two DAGs
  for (int ti = blockIdx.x; ti < p.ntri; ti += gridDim.x) {
    const int a = p.tri[3 * ti], b = p.tri[3 * ti + 1], c = p.tri[3 * ti + 2];
    int qa = 0, qb = 0;
    const int la = cta_forward(p, A, a, sh, &qa, &my_arcs);
    account(la, qa);
    // a, b and c share a component: one weighted size serves all three
    if (p.leaf_term && p.omega && (p.omega[a] > 0 || p.omega[b] > 0 || p.omega[c] > 0))
      cta_weighted_size(p, A, qa, sh);
    cta_backward(p, A, a, la, bcp, sh);
    const int lb = cta_forward(p, B, b, sh, &qb, &my_arcs);
    account(lb, qb);
    cta_backward(p, B, b, lb, bcp, sh);
    cta_backward_deg2(p, A, B, la, lb, c, rc, bcp, sh);
    cta_reset(A, qa);
    cta_reset(B, qb);
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

// Several requests: req_bc[q][v] += sum over request q's CTAs c (in order) of bcp[c][v]
// (rc: the requests' CTA ranges, nreq + 1 offsets).
__global__ void k_cta_reduce_req(const double *bcp, int nreq, const int32_t *rc, double *const *req_bc, int n) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    for (int q = 0; q < nreq; q++) {
      double sum = 0.0;
      for (int c = rc[q]; c < rc[q + 1]; c++) sum += bcp[(size_t)c * n + v];
      if (sum != 0.0) req_bc[q][v] += sum;
    }
  }
}

}  // namespace

struct CtaWS {
  int n = 0, ncta = 0, in_smem = 0, tri = 0;
  bool clean = false;  // global-memory state left cleared by a completed launch
  size_t slice = 0, smem = 0;
  double *bcp = nullptr;
  char *gws = nullptr;
  unsigned long long *stats = nullptr;
  int32_t *req = nullptr;  // request offsets of a launch with several requests
  size_t bytes = 0;
};

void cta_free(Ctx *ctx, CtaWS *ws) {
  if (!ws) return;
  cudaFree(ws->bcp);
  cudaFree(ws->gws);
  cudaFree(ws->stats);
  cudaFree(ws->req);
  ctx->mem.release(nullptr, ws->bytes);
  delete ws;
}

static bc_status cta_ensure(Ctx *ctx, CtaWS **wsp, int n, bool tri) {
  CtaWS *ws = *wsp;
  const size_t st = cta_state_bytes(n);
  const int in_smem = st <= kCtaSmemMax;
  const size_t smem = in_smem ? st : 0;
  int bps = 0;
  {
    // the attribute is per function and device: set it once, to the largest size used, so
    // that concurrent callers (serving workers on graphs of different sizes) never lower it
    // under another's launch
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    BC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      BC_CUDA_TRY(cudaFuncSetAttribute(k_cta_sources, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kCtaSmemMax));
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  BC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_cta_sources, kCtaThreads, smem));
  if (bps < 1) return fail(BC_ECUDA, "CTA per-source kernel does not fit on an SM");
  if (!in_smem) bps = std::min(bps, 2);  // slices live in L2 / HBM: keep their total small
  int ncta = ctx->num_sms * bps;
  // slice: state A (unless in shared memory) and its extras; with triples also state B,
  // its extras and c's r values
  const size_t slice = ((in_smem ? 0 : st) + cta_extra_bytes(n) +
                        (tri ? st + cta_extra_bytes(n) + (size_t)n * 8 : 0) + 255) & ~(size_t)255;
  const size_t per_cta = (size_t)n * 8 + slice;
  if (ctx->mem.budget) {  // fewer CTAs when the context's HBM budget is tight: at most half
    // of what is free, so that requests arriving meanwhile still find room (serving)
    const size_t used = ctx->mem.used.load() - (ws ? ws->bytes : 0);
    const size_t avail = ctx->mem.budget > used + 64 ? ctx->mem.budget - used - 64 : 0;
    ncta = (int)std::min<size_t>((size_t)ncta, std::max<size_t>(avail / 2 / per_cta, avail >= per_cta ? 1 : 0));
    if (ncta < 1) return fail(BC_ENOMEM, "CTA per-source workspace exceeds the context HBM budget");
  }
  if (ws && ws->n == n && ws->ncta == ncta && ws->tri >= (int)tri) return BC_OK;
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
  ws->tri = tri ? 1 : 0;
  const size_t b_bcp = (size_t)ncta * n * 8, b_gws = ws->slice * ncta;
  ws->bytes = b_bcp + b_gws + 64 + 2 * (kCtaMaxReq + 1) * sizeof(int32_t);
  bc_status s = ctx->mem.alloc(nullptr, ws->bytes);
  if (s) {
    delete ws;
    return s;
  }
  cudaError_t e = cudaMalloc((void **)&ws->bcp, b_bcp);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->gws, b_gws);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->stats, 64);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->req, 2 * (kCtaMaxReq + 1) * sizeof(int32_t));
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
  if (a.nsrc <= 0 && a.ntri <= 0) return BC_OK;
  bc_status s = cta_ensure(ctx, wsp, n, a.ntri > 0);
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
  p.clean = ws->clean ? 1 : 0;
  p.stats = ws->stats;
  p.out_depth = a.out_depth;
  p.out_sigma = a.out_sigma;
  p.out_ovf = a.out_ovf;
  p.tri = a.tri;
  p.ntri = sssp ? 0 : a.ntri;
  if (a.nreq > 0 && (sssp || p.ntri || a.nreq > kCtaMaxReq || !a.h_req_k || !a.req_bc))
    return fail(BC_EINVAL, "CTA per-source kernel: bad request list");
  // requests per launch: groups of consecutive requests, each request with CTAs of its own
  // (at most ws->ncta requests per launch)
  std::vector<std::vector<int32_t>> hreq;
  int nlaunch = 0, launched_max = 0;
  BC_CUDA_TRY(cudaMemsetAsync(ws->stats, 0, 64, st));
  cudaEvent_t e0, e1;
  BC_CUDA_TRY(cudaEventCreate(&e0));
  BC_CUDA_TRY(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  const bool was_clean = ws->clean;
  ws->clean = false;  // until the launches are known to have completed
  cudaError_t le = cudaSuccess;
  auto launch = [&](const CtaK &kp, int ncta, const int32_t *rc, double *const *rbc) {
    CtaK q = kp;
    q.clean = (was_clean || launched_max >= ncta) ? 1 : 0;
    k_cta_sources<<<ncta, kCtaThreads, ws->smem, st>>>(q);
    le = cudaGetLastError();
    launched_max = std::max(launched_max, ncta);
    nlaunch++;
    if (le == cudaSuccess && !sssp && q.nreq > 0) {
      k_cta_reduce_req<<<ctx->num_sms * 4, 256, 0, st>>>(ws->bcp, q.nreq, rc, rbc, n);
      le = cudaGetLastError();
    } else if (le == cudaSuccess && !sssp && a.bc) {
      k_cta_reduce<<<ctx->num_sms * 4, 256, 0, st>>>(ws->bcp, ncta, n, a.bc);
      le = cudaGetLastError();
    }
  };
  if (a.nreq <= 0) {
    launch(p, std::max(1, std::min(ws->ncta, std::max(p.nsrc, p.ntri))), nullptr, nullptr);
  } else {
    int q0 = 0, soff = 0;
    while (q0 < a.nreq && le == cudaSuccess) {
      const int q1 = std::min(a.nreq, q0 + ws->ncta);
      const int R = q1 - q0;
      long long K = 0;
      for (int q = q0; q < q1; q++) K += a.h_req_k[q];
      const int C = (int)std::max<long long>(R, std::min<long long>(ws->ncta, K));
      // CTAs in proportion to the sources (at least one each, at most one per source), then
      // the rest, one at a time, to the request with the most rounds of sources per CTA
      std::vector<int> c(R);
      int used = 0;
      for (int j = 0; j < R; j++) {
        const long long k = a.h_req_k[q0 + j];
        c[j] = (int)std::max<long long>(1, std::min<long long>(k, K > 0 ? C * k / K : 1));
        used += c[j];
      }
      while (used > C) {
        int jm = -1;
        for (int j = 0; j < R; j++)
          if (c[j] > 1 && (jm < 0 || c[j] > c[jm])) jm = j;
        if (jm < 0) break;
        c[jm]--;
        used--;
      }
      while (used < C) {
        int jm = -1;
        long long best = 0;
        for (int j = 0; j < R; j++) {
          const long long k = a.h_req_k[q0 + j];
          const long long rounds = (k + c[j] - 1) / c[j];
          if (c[j] < k && rounds > best) {
            best = rounds;
            jm = j;
          }
        }
        if (jm < 0) break;
        c[jm]++;
        used++;
      }
      std::vector<int32_t> &h = hreq.emplace_back(2 * (R + 1));
      h[0] = 0;
      h[R + 1] = 0;
      for (int j = 0; j < R; j++) {
        h[j + 1] = h[j] + a.h_req_k[q0 + j];
        h[R + 2 + j] = h[R + 1 + j] + c[j];
      }
      le = cudaMemcpyAsync(ws->req, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      if (le != cudaSuccess) break;
      CtaK kp = p;
      kp.src = a.src + soff;
      kp.nsrc = h[R];
      kp.nreq = R;
      kp.req = ws->req;
      launch(kp, used, ws->req + R + 1, a.req_bc + q0);
      soff += h[R];
      q0 = q1;
    }
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
  // the launched CTAs left their state cleared; CTAs not launched kept theirs
  ws->clean = was_clean || launched_max == ws->ncta;
  if (acc) {
    acc->seconds += ms * 1e-3;
    acc->sources += p.nsrc + 3ll * p.ntri;
    acc->sigma_overflow_sources += (int64_t)hs[4];
    acc->reached_vertices += (int64_t)hs[0];
    acc->reached_arcs += (int64_t)hs[1];
    acc->levels += (int64_t)hs[2];
    if ((int32_t)hs[3] > acc->max_depth) acc->max_depth = (int32_t)hs[3];
    acc->kernel_launches += sssp ? nlaunch : 2 * nlaunch;
    if (acc->tile_width == 0) acc->tile_width = 1;
  }
  return BC_OK;
}

}  // namespace bcl

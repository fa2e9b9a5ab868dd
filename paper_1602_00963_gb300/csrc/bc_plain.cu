// Per-source path: one BFS per source, run by a persistent cooperative kernel that
// loops over the sources of the call and, per source, over BFS levels.
//
// Forward (shortest-path counting, Alg. 2 / Alg. 3, Sec. 3.2):
//   * top-down levels use active-edge parallelism (Sec. 3.1): the frontier's adjacency
//     lists are treated as one concatenated edge array; each warp takes an equal,
//     contiguous slice and maps edge -> owning frontier vertex by a search in the
//     exclusive degree prefix CD.  CD is not recomputed per level: every append to the
//     queue Q reserves its slot and its edge offset with one packed 64-bit atomicAdd,
//     so CD is produced in Q order as the frontier is built, and the backward sweep
//     reuses it (the scan / search reuse of Sec. 3.1).  A warp keeps a window of 128
//     CD entries in shared memory and has four 32-edge steps in flight at once.
//   * Alg. 3 tests d[w] and adds sigma in one parallel loop, which can drop a term when
//     a thread reads d[w] before another thread has set it.  Here the discovering
//     compare-and-swap returns the previous depth, and a thread adds sigma exactly when
//     that value is -1 (it discovered w) or the current level (w was discovered at this
//     level), so every parent edge contributes once.
//   * bottom-up levels (direction switch): each unvisited vertex sums sigma over all its
//     neighbours in the frontier bitmap (all parents at level d-1, no early exit, so
//     sigma stays exact).
//   * sigma is kept modulo 2^64 with a sticky overflow bit; vertices whose count
//     overflows also get an extended-range value (double mantissa, int exponent).
// Backward (dependency accumulation, Alg. 4 / Alg. 5, successor checking):
//   for depth = D-1 .. 1, every edge (w, v) of the depth-level vertices w with
//   d[v] = d[w] + 1 adds sigma[w] * r[v] = sigma[w] / sigma[v] * (1 + delta[v] + omega[v])
//   to acc[w]; then delta[w] = acc[w] (updateDep), BC[w] += (omega[s] + 1) * delta[w]
//   (Eq. 3 / Eq. 4) and r[w] = (1 + delta[w] + omega[w]) / sigma[w].  Each term lies in
//   [0, n] and is added as a 128-bit fixed-point integer (64 fraction bits; warp-segmented
//   sums, one pair of 64-bit integer atomics per segment): integer sums do not depend on
//   the order of the additions, so the result repeats bit for bit from run to run.
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "bc_internal.h"

namespace bcl {

namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int U = 4;             // 32-edge steps in flight per warp
constexpr int WIN = 32 * U;      // owner window (queue entries) per warp
constexpr unsigned kFound = 1u, kOvf = 2u;

struct WarpWin {
  int cd[WIN + 1];  // CD of window entries (INT_MAX past the range), then the next CD
  int v[WIN];       // vertex of each entry
  int bias[WIN];    // row_ptr[v] - CD: col position of edge e is e + bias
  int ex[WIN];      // extended-range exponent of the owner (backward, EXT only)
  double sg[WIN];   // sigma of the owner (backward; EXT: its mantissa)
};
constexpr size_t kSmemBytes = sizeof(WarpWin) * kWarps;

struct PK {
  int32_t n;
  int64_t nnz;
  int32_t max_degree;
  const int32_t *__restrict__ rp;
  const int32_t *__restrict__ ci;
  const int32_t *__restrict__ omega;
  const int32_t *__restrict__ src;
  int32_t nsrc;
  double *bc;
  int leaf_term;
  int32_t *depth, *Q, *CD, *lvl_off, *lvl_eoff;
  unsigned long long *sig;
  uint32_t *ovf, *vis, *front;
  unsigned long long *acc;  // [2n]: per vertex the low and high word of a 64.64 fixed-point sum
  double *r, *xm;
  int32_t *xe;
  PlainCtl *ctl;
  int32_t *out_depth;
  unsigned long long *out_sigma;
  uint8_t *out_ovf;
  float alpha, beta;
  uint64_t limit_ns;
  unsigned long long *trace;  // optional phase trace: (phase << 56 | level << 32, time) pairs
  int trace_cap;
  int no_cd_reuse;            // backward: rescan CD per level (ablation)
};

// Grid barrier; with tracing on, CTA 0 stamps the time at which every CTA has finished
// the phase (so consecutive stamps give each phase's duration, slowest CTA included).
__device__ __forceinline__ bool phase_sync(const PK &p, GridSync *gs, int phase, int level) {
  bool ok = grid_sync(gs, p.limit_ns);
  if (p.trace && blockIdx.x == 0 && threadIdx.x == 0) {
    int i = p.ctl->trace_n++;
    if (i < p.trace_cap) {
      p.trace[2 * i] = ((unsigned long long)phase << 56) | ((unsigned long long)(unsigned)level << 24);
      p.trace[2 * i + 1] = globaltimer_ns();
    }
  }
  return ok;
}

// Extended-range sigma: value = m * 2^e.
struct XS {
  double m;
  int e;
};

__device__ __forceinline__ XS xs_from_u64(unsigned long long s) {
  XS x;
  x.m = frexp((double)s, &x.e);
  return x;
}
__device__ __forceinline__ void xs_add(XS &a, XS b) {
  if (b.m == 0.0) return;
  if (a.m == 0.0) { a = b; return; }
  if (b.e > a.e) {
    a.m = ldexp(a.m, a.e - b.e) + b.m;
    a.e = b.e;
  } else {
    a.m += ldexp(b.m, b.e - a.e);
  }
}
__device__ __forceinline__ XS xs_norm(XS a) {
  int de;
  a.m = frexp(a.m, &de);
  a.e += de;
  return a;
}
__device__ __forceinline__ XS get_xs(const PK &p, int v) {
  if (test_bit(p.ovf, v)) {
    XS x;
    x.m = p.xm[v];
    x.e = p.xe[v];
    return x;
  }
  return xs_from_u64(p.sig[v]);
}

// Largest i in [lo, hi) with CD[i] <= x (CD non-decreasing on [lo, hi), CD[lo] <= x).
__device__ __forceinline__ int warp_find_owner(const int32_t *CD, int lo, int hi, int x) {
  const int lane = lane_id();
  while (hi - lo > 32) {
    int stride = (hi - lo + 31) / 32;
    int pos = lo + lane * stride;
    bool ok = pos < hi && CD[pos] <= x;
    unsigned b = __ballot_sync(BC_FULL, ok);
    int k = 31 - __clz(b);
    lo = lo + k * stride;
    hi = min(lo + stride, hi);
  }
  int pos = lo + lane;
  bool ok = pos < hi && CD[pos] <= x;
  unsigned b = __ballot_sync(BC_FULL, ok);
  return lo + (31 - __clz(b));
}

// Warp-aggregated append of up to U flagged vertices per lane to Q (and their degree
// prefix to CD) with one packed atomicAdd per warp.
__device__ __forceinline__ void warp_append_u(const PK &p, const int (&w)[U], const bool (&isnew)[U]) {
  int cnt = 0, dsum = 0;
  int dg[U];
#pragma unroll
  for (int k = 0; k < U; k++) {
    dg[k] = isnew[k] ? (p.rp[w[k] + 1] - p.rp[w[k]]) : 0;
    cnt += isnew[k];
    dsum += dg[k];
  }
  if (__ballot_sync(BC_FULL, cnt > 0) == 0) return;
  int ctot, dtot;
  int cpre = warp_excl_scan(cnt, &ctot);
  int dpre = warp_excl_scan(dsum, &dtot);
  unsigned long long base = 0;
  if (lane_id() == 0) base = atomicAdd(&p.ctl->qpack, pack_qe((unsigned)ctot, (unsigned)dtot));
  base = __shfl_sync(BC_FULL, base, 0);
  int pos = (int)(base >> 32) + cpre;
  int eo = (int)(base & 0xffffffffull) + dpre;
#pragma unroll
  for (int k = 0; k < U; k++) {
    if (isnew[k]) {
      p.Q[pos] = w[k];
      p.CD[pos] = eo;
      pos++;
      eo += dg[k];
    }
  }
}

template <bool EXT, bool BWD>
__device__ __forceinline__ void fill_window(const PK &p, WarpWin &W, int base, int q1, int E1) {
  const int lane = lane_id();
  int vv[U], cc[U];
#pragma unroll
  for (int k = 0; k < U; k++) {
    int idx = base + lane + 32 * k;
    bool in = idx < q1;
    cc[k] = in ? p.CD[idx] : INT_MAX;
    vv[k] = in ? p.Q[idx] : -1;
  }
#pragma unroll
  for (int k = 0; k < U; k++) {
    int j = lane + 32 * k;
    W.cd[j] = cc[k];
    W.v[j] = vv[k];
    W.bias[j] = vv[k] >= 0 ? p.rp[vv[k]] - cc[k] : 0;
    if (BWD) {
      if (EXT) {
        const XS x = vv[k] >= 0 ? get_xs(p, vv[k]) : XS{0.0, 0};
        W.ex[j] = x.e;
        W.sg[j] = x.m;
      } else {
        W.sg[j] = vv[k] >= 0 ? (double)p.sig[vv[k]] : 0.0;
      }
    }
  }
  if (lane == 0) W.cd[WIN] = (base + WIN < q1) ? p.CD[base + WIN] : E1;
  __syncwarp();
}

__device__ __forceinline__ int win_owner(const WarpWin &W, int e) {
  int j = 0;
#pragma unroll
  for (int s = WIN / 2; s >= 1; s >>= 1)
    if (W.cd[j + s] <= e) j += s;
  return j;
}

// Iterate the warp's slice of the edge range [E0, E1) of queue range [q0, q1), U x 32
// edges at a time.  body(e0, ee) is called once per window with the window filled.
template <bool EXT, bool BWD, typename F>
__device__ __forceinline__ void edge_windows(const PK &p, WarpWin &W, int q0, int q1, int E0,
                                             int E1, int gwarp, int nwarps, F &&body) {
  long long E = (long long)E1 - E0;
  if (E <= 0) return;
  long long per = (E + nwarps - 1) / nwarps;
  per = (per + 31) & ~31ll;
  long long ebl = (long long)E0 + (long long)gwarp * per;
  if (ebl >= E1) return;
  const int eb = (int)ebl;
  const int ee = (int)min(ebl + per, (long long)E1);
  int base = warp_find_owner(p.CD, q0, q1, eb);
  for (int e0 = eb; e0 < ee; e0 += WIN) {
    fill_window<EXT, BWD>(p, W, base, q1, E1);
    body(e0, ee);
    // next window starts at the owner of edge e0 + WIN
    int jl = win_owner(W, e0 + WIN - 1);
    int nb = base + jl + ((e0 + WIN >= W.cd[jl + 1]) ? 1 : 0);
    __syncwarp();
    base = nb;
  }
}

__device__ void expand_topdown(const PK &p, WarpWin &W, int level, int q0, int q1, int E0,
                               int E1, int gwarp, int nwarps, bool fast) {
  const int lane = lane_id();
  edge_windows<false, false>(p, W, q0, q1, E0, E1, gwarp, nwarps, [&](int e0, int ee) {
    int w[U], v[U];
    bool isnew[U], dag[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      int e = e0 + lane + 32 * k;
      int j = win_owner(W, e);
      v[k] = W.v[j];
      w[k] = e < ee ? p.ci[e + W.bias[j]] : -1;
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      isnew[k] = false;
      dag[k] = false;
      if (w[k] >= 0 && !test_bit(p.vis, w[k])) {
        int old = atomicCAS(p.depth + w[k], -1, level);
        isnew[k] = old < 0;
        dag[k] = isnew[k] || old == level;
      }
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      if (dag[k]) {
        unsigned long long sv = p.sig[v[k]];
        if (fast) {
          atomicAdd(p.sig + w[k], sv);
        } else {
          unsigned long long old = atomicAdd(p.sig + w[k], sv);
          if (old + sv < old || test_bit(p.ovf, v[k])) {
            set_bit_atomic(p.ovf, w[k]);
            p.ctl->level_ovf[level & 1] = 1;
            p.ctl->src_ovf = 1;
          }
        }
      }
    }
    warp_append_u(p, w, isnew);
  });
}

__device__ void sweep_bottomup(const PK &p, int level, int gwarp, int nwarps,
                               unsigned long long (*s_sig)[32], unsigned (*s_flag)[32]) {
  const int lane = lane_id();
  const int wl = threadIdx.x >> 5;
  for (int g = gwarp; g * 32 < p.n; g += nwarps) {
    int u = g * 32 + lane;
    bool act = u < p.n && !test_bit(p.vis, u);
    int st = 0, c = 0;
    if (act) {
      st = p.rp[u];
      c = p.rp[u + 1] - st;
    }
    int tot;
    int ex = warp_excl_scan(c, &tot);
    if (tot == 0) continue;
    s_sig[wl][lane] = 0ull;
    s_flag[wl][lane] = 0u;
    __syncwarp();
    int bias = st - ex;
    for (int e0 = 0; e0 < tot; e0 += WIN) {
      int pn[U], jj[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        int my = e0 + lane + 32 * k;
        jj[k] = warp_owner(ex, my);
        int b = __shfl_sync(BC_FULL, bias, jj[k]);
        pn[k] = my < tot ? p.ci[my + b] : -1;
      }
      bool fr[U];
#pragma unroll
      for (int k = 0; k < U; k++) fr[k] = pn[k] >= 0 && test_bit(p.front, pn[k]);
#pragma unroll
      for (int k = 0; k < U; k++) {
        if (fr[k]) {
          unsigned long long sv = p.sig[pn[k]];
          unsigned long long old = atomicAdd(&s_sig[wl][jj[k]], sv);
          unsigned fl = kFound;
          if (old + sv < old || test_bit(p.ovf, pn[k])) fl |= kOvf;
          atomicOr(&s_flag[wl][jj[k]], fl);
        }
      }
    }
    __syncwarp();
    unsigned f = s_flag[wl][lane];
    bool isnew = act && (f & kFound);
    int wv[U] = {u};
    bool nv[U] = {isnew};
    if (isnew) {
      p.depth[u] = level;
      p.sig[u] = s_sig[wl][lane];
      if (f & kOvf) {
        set_bit_atomic(p.ovf, u);
        p.ctl->level_ovf[level & 1] = 1;
        p.ctl->src_ovf = 1;
      }
    }
    warp_append_u(p, wv, nv);
    __syncwarp();
  }
}

// Extended-range sigma of an overflowed vertex: sum over its parents (d = level-1).
__device__ void ext_sigma(const PK &p, int w, int level) {
  XS a;
  a.m = 0.0;
  a.e = 0;
  for (int e = p.rp[w]; e < p.rp[w + 1]; e++) {
    int x = p.ci[e];
    if (p.depth[x] == level - 1) xs_add(a, get_xs(p, x));
  }
  a = xs_norm(a);
  p.xm[w] = a.m;
  p.xe[w] = a.e;
}

// A term t in [0, 2^63) as a 128-bit fixed-point integer with 64 fraction bits (hi: integer
// part, lo: fraction), truncated below 2^-64; integer operations on the IEEE-754 fields.
__device__ __forceinline__ void fx_from(double t, unsigned long long &hi, unsigned long long &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(t);
  const int ex = (int)((b >> 52) & 0x7ffull);
  hi = lo = 0ull;
  if (ex == 0 || (b >> 63)) return;  // zero (or below 2^-1022: far below 2^-64)
  const unsigned long long m = (b & 0x000fffffffffffffull) | (1ull << 52);  // t = m 2^(ex - 1075)
  const int sh = ex - 1075 + 64;                                           // fixed = m 2^sh
  if (sh >= 64) {
    hi = m << (sh - 64);
  } else if (sh > 0) {
    hi = m >> (64 - sh);
    lo = m << sh;
  } else if (sh > -64) {
    lo = m >> (-sh);
  }
}

template <bool EXT>
__device__ void accumulate_level(const PK &p, WarpWin &W, int d, int q0, int q1, int E0, int E1,
                                 int gwarp, int nwarps) {
  const int lane = lane_id();
  edge_windows<EXT, true>(p, W, q0, q1, E0, E1, gwarp, nwarps, [&](int e0, int ee) {
    int own[U], nb[U], ew[U];
    double sw[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      int e = e0 + lane + 32 * k;
      int j = win_owner(W, e);
      bool valid = e < ee;
      own[k] = valid ? W.v[j] : -1;
      ew[k] = EXT ? W.ex[j] : 0;
      sw[k] = W.sg[j];
      nb[k] = valid ? p.ci[e + W.bias[j]] : -1;
    }
    int dv[U];
#pragma unroll
    for (int k = 0; k < U; k++) dv[k] = nb[k] >= 0 ? p.depth[nb[k]] : -9;
    double val[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      val[k] = 0.0;
      if (dv[k] == d + 1) {
        val[k] = p.r[nb[k]];
        if (EXT) val[k] = ldexp(val[k], ew[k] - p.xe[nb[k]]);
        val[k] *= sw[k];  // sigma[w] / sigma[v] * (1 + delta[v] + omega[v])
      }
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      unsigned long long hi, lo;
      fx_from(val[k], hi, lo);
      const int o = own[k];
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const unsigned long long yl = __shfl_down_sync(BC_FULL, lo, s);
        const unsigned long long yh = __shfl_down_sync(BC_FULL, hi, s);
        const int oo = __shfl_down_sync(BC_FULL, o, s);
        if (lane + s < 32 && oo == o) {
          const unsigned long long l2 = lo + yl;
          hi += yh + (l2 < lo ? 1ull : 0ull);
          lo = l2;
        }
      }
      const int prev = __shfl_up_sync(BC_FULL, o, 1);
      const bool head = (lane == 0) || (prev != o);
      if (head && o >= 0 && (hi | lo)) {
        unsigned long long *a = p.acc + 2 * (size_t)o;
        const unsigned long long old = lo ? atomicAdd(a, lo) : 0ull;
        const unsigned long long c = (lo && old + lo < old) ? 1ull : 0ull;  // the low word wrapped
        if (hi + c) atomicAdd(a + 1, hi + c);
      }
    }
  });
}

template <bool EXT>
__device__ void finalize_level(const PK &p, int q0, int q1, double ws, int gtid, int nthr) {
  for (int i = q0 + gtid; i < q1; i += nthr) {
    int w = p.Q[i];
    unsigned long long *a = p.acc + 2 * (size_t)w;
    const unsigned long long lo = a[0], hi = a[1];
    if (lo | hi) {
      a[0] = 0ull;
      a[1] = 0ull;
    }
    const double delta = (double)hi + (double)lo * 0x1p-64;
    double om = p.omega ? (double)p.omega[w] : 0.0;
    double sg;
    if (EXT) {
      XS x = get_xs(p, w);
      sg = x.m;
      p.xe[w] = x.e;
    } else {
      sg = (double)p.sig[w];
    }
    if (lo | hi) p.bc[w] += ws * delta;
    p.r[w] = (1.0 + delta + om) / sg;
  }
}

// Exclusive prefix of x over the CTA's threads in thread order; *total = the CTA's sum.
// Contains barriers: every thread of the CTA calls it.
__device__ __forceinline__ int cta_excl_scan(int x, int *total, int *s_warp) {
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  int wt;
  const int pre = warp_excl_scan(x, &wt);
  if (lane == 0) s_warp[wid] = wt;
  __syncthreads();
  if (wid == 0) {
    const int v = lane < kWarps ? s_warp[lane] : 0;
    int t;
    const int vp = warp_excl_scan(v, &t);
    if (lane < kWarps) s_warp[lane] = vp;
    if (lane == 0) s_warp[kWarps] = t;
  }
  __syncthreads();
  const int r = s_warp[wid] + pre;
  *total = s_warp[kWarps];
  __syncthreads();  // s_warp is reused by the next call
  return r;
}

// Sec. 3.1 without its reuse (the ablation BC_NO_CD_REUSE): before the backward sweep reads
// the degree prefix CD of level d's entries Q[q0, q1), it is scanned again instead of taken
// from the forward appends.  CTAs sum the degrees of equal chunks of the level, then each
// scans its chunk starting from E0 plus the sums of the CTAs before it.  The values equal
// the stored ones (the appends lay entries and their edge offsets out in queue order), so
// only the time differs (and the order of the backward's atomic additions).  Two grid
// barriers.
__device__ bool rescan_level(const PK &p, GridSync *gs, int d, int q0, int q1, int E0) {
  __shared__ int s_warp[kWarps + 1];
  __shared__ int s_base;
  const int nb = gridDim.x, b = blockIdx.x;
  const long long len = (long long)q1 - q0;
  const int c0 = q0 + (int)(len * b / nb), c1 = q0 + (int)(len * (b + 1) / nb);
  int part = 0;
  for (int i = c0 + (int)threadIdx.x; i < c1; i += kThreads) {
    const int v = p.Q[i];
    part += p.rp[v + 1] - p.rp[v];
  }
  int tot;
  (void)cta_excl_scan(part, &tot, s_warp);
  if (threadIdx.x == 0) p.ctl->scan_blk[b] = tot;
  if (!phase_sync(p, gs, 8, d)) return false;
  if (threadIdx.x < 32) {
    int acc = 0;
    for (int j = (int)threadIdx.x; j < b; j += 32) acc += ld_volatile_i32(&p.ctl->scan_blk[j]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(BC_FULL, acc, m);
    if (threadIdx.x == 0) s_base = E0 + acc;
  }
  __syncthreads();
  int base = s_base;
  for (int i0 = c0; i0 < c1; i0 += kThreads) {  // c0, c1 are uniform over the CTA
    const int i = i0 + (int)threadIdx.x;
    int dg = 0;
    if (i < c1) {
      const int v = p.Q[i];
      dg = p.rp[v + 1] - p.rp[v];
    }
    int t;
    const int pre = cta_excl_scan(dg, &t, s_warp);
    if (i < c1) p.CD[i] = base + pre;
    base += t;
  }
  return phase_sync(p, gs, 9, d);
}

__global__ void __launch_bounds__(kThreads, 1) plain_kernel(PK p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_sig[kWarps][32];
  __shared__ unsigned s_flag[kWarps][32];
  __shared__ unsigned long long s_ns, s_max;
  WarpWin &W = ((WarpWin *)smem)[threadIdx.x >> 5];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int gwarp = gtid >> 5;
  const int nwarps = nthr >> 5;
  PlainCtl *ctl = p.ctl;
  GridSync *gs = &ctl->bar;
  const bool sssp = p.out_depth != nullptr;

  for (int si = 0; si < p.nsrc; ++si) {
    const int s = p.src[si];
    if (gtid == 0) {
      int ds = p.rp[s + 1] - p.rp[s];
      p.depth[s] = 0;
      p.sig[s] = 1ull;
      p.Q[0] = s;
      p.CD[0] = 0;
      p.lvl_off[0] = 0;
      p.lvl_off[1] = 1;
      p.lvl_eoff[0] = 0;
      p.lvl_eoff[1] = ds;
      ctl->qpack = pack_qe(1u, (unsigned)ds);
      ctl->ns = 1ull + (p.omega ? (unsigned long long)p.omega[s] : 0ull);
      ctl->src_ovf = 0;
      ctl->level_ovf[0] = 0;
      ctl->level_ovf[1] = 0;
      ctl->sigmax[0] = 1ull;
      ctl->sigmax[1] = 0ull;
      set_bit_atomic(p.vis, s);
      set_bit_atomic(p.front, s);
    }
    if (!phase_sync(p, gs, 0, 0)) return;

    // ---------------------------------------------------------------- forward
    int level = 1;
    bool bu = false;
    while (true) {
      const int q0 = p.lvl_off[level - 1], q1 = p.lvl_off[level];
      const int nf = q1 - q0;
      if (nf == 0) break;
      const int E0 = p.lvl_eoff[level - 1], E1 = p.lvl_eoff[level];
      const double mf = (double)(E1 - E0);
      const double mu = (double)(p.nnz - E1);
      if (!bu) {
        if (mf > (double)p.alpha * mu) bu = true;
      } else {
        if ((double)nf * (double)p.beta < (double)p.n && mf < (double)p.alpha * mu) bu = false;
      }
      if (bu) {
        sweep_bottomup(p, level, gwarp, nwarps, s_sig, s_flag);
      } else {
        // no 64-bit carry is possible this level if max sigma * max degree < 2^64
        const bool fast = *(volatile int *)&ctl->src_ovf == 0 &&
                          (double)*(volatile unsigned long long *)&ctl->sigmax[(level - 1) & 1] *
                                  (double)p.max_degree < 1.8e19;
        expand_topdown(p, W, level, q0, q1, E0, E1, gwarp, nwarps, fast);
      }
      if (!phase_sync(p, gs, bu ? 2 : 1, level)) return;

      // post: level offsets, bitmaps, component size, level max sigma, extended sigma
      const unsigned long long pk = *(volatile unsigned long long *)&ctl->qpack;
      const int q2 = (int)(pk >> 32);
      const bool lvl_ovf = *(volatile int *)&ctl->level_ovf[level & 1] != 0;
      if (threadIdx.x == 0) {
        s_ns = 0ull;
        s_max = 0ull;
      }
      __syncthreads();
      unsigned long long nsl = 0, mx = 0;
      for (int i = q1 + gtid; i < q2; i += nthr) {
        int w = p.Q[i];
        set_bit_atomic(p.vis, w);
        set_bit_atomic(p.front, w);
        nsl += 1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull);
        unsigned long long sw = p.sig[w];
        mx = sw > mx ? sw : mx;
        if (lvl_ovf && test_bit(p.ovf, w)) ext_sigma(p, w, level);
      }
      for (int i = q0 + gtid; i < q1; i += nthr) clear_bit_atomic(p.front, p.Q[i]);
      if (nsl) atomicAdd(&s_ns, nsl);
      if (mx) atomicMax(&s_max, mx);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (s_ns) atomicAdd(&ctl->ns, s_ns);
        if (s_max) atomicMax(&ctl->sigmax[level & 1], s_max);
      }
      if (gtid == 0) {
        p.lvl_off[level + 1] = q2;
        p.lvl_eoff[level + 1] = (int)(pk & 0xffffffffull);
        ctl->level_ovf[(level + 1) & 1] = 0;
        ctl->sigmax[(level + 1) & 1] = 0ull;
      }
      if (!phase_sync(p, gs, 3, level)) return;
      level++;
    }
    const int D = level - 2;                 // deepest non-empty level
    const int qtot = p.lvl_off[level - 1];   // reached vertices

    if (sssp) {
      for (int v = gtid; v < p.n; v += nthr) {
        p.out_depth[v] = p.depth[v];
        p.out_sigma[v] = p.sig[v];
        p.out_ovf[v] = test_bit(p.ovf, v) ? 1 : 0;
      }
      // every vertex is exported before any is reset below
      if (!phase_sync(p, gs, 4, 0)) return;
    } else {
      // -------------------------------------------------------------- backward
      const bool ext = *(volatile int *)&ctl->src_ovf != 0;
      const double ws = p.omega ? (double)p.omega[s] + 1.0 : 1.0;
      if (D >= 1) {
        if (ext)
          finalize_level<true>(p, p.lvl_off[D], p.lvl_off[D + 1], ws, gtid, nthr);
        else
          finalize_level<false>(p, p.lvl_off[D], p.lvl_off[D + 1], ws, gtid, nthr);
        if (!phase_sync(p, gs, 4, D)) return;
        for (int d = D - 1; d >= 1; --d) {
          const int q0 = p.lvl_off[d], q1 = p.lvl_off[d + 1];
          const int E0 = p.lvl_eoff[d], E1 = p.lvl_eoff[d + 1];
          if (p.no_cd_reuse && !rescan_level(p, gs, d, q0, q1, E0)) return;
          if (ext)
            accumulate_level<true>(p, W, d, q0, q1, E0, E1, gwarp, nwarps);
          else
            accumulate_level<false>(p, W, d, q0, q1, E0, E1, gwarp, nwarps);
          if (!phase_sync(p, gs, 5, d)) return;
          if (ext)
            finalize_level<true>(p, q0, q1, ws, gtid, nthr);
          else
            finalize_level<false>(p, q0, q1, ws, gtid, nthr);
          if (!phase_sync(p, gs, 6, d)) return;
        }
      }
      if (gtid == 0 && p.leaf_term && p.omega && p.omega[s] > 0) {
        double om = (double)p.omega[s];
        double ns = (double)*(volatile unsigned long long *)&ctl->ns;
        p.bc[s] += om * (2.0 * ns - om - 3.0);
      }
    }
    if (gtid == 0) {
      if (*(volatile int *)&ctl->src_ovf) ctl->ovf_sources++;
      ctl->levels += level - 1;
      ctl->reached += qtot;
      ctl->reached_arcs += p.lvl_eoff[level - 1];
      if (D > ctl->max_depth) ctl->max_depth = D;
    }
    // reset the state of the reached vertices for the next source
    for (int i = gtid; i < qtot; i += nthr) {
      int w = p.Q[i];
      p.depth[w] = -1;
      p.sig[w] = 0ull;
      p.vis[w >> 5] = 0u;
      p.front[w >> 5] = 0u;
      p.ovf[w >> 5] = 0u;
    }
    if (!phase_sync(p, gs, 7, 0)) return;
  }
}

// The dynamic shared-memory size of plain_kernel is an attribute of the function on one
// device: it is set on each device before that device's first launch.
std::mutex g_setup_mu;
bool g_setup_done[128];

bc_status plain_setup(int *blocks_per_sm) {
  int dev = 0;
  BC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(BC_EINVAL, "per-source kernel: device index out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_setup_done[dev]) {
    BC_CUDA_TRY(cudaFuncSetAttribute(plain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes));
    int b = 0;
    BC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, plain_kernel, kThreads, kSmemBytes));
    if (b < 1) return fail(BC_ECUDA, "per-source kernel does not fit on an SM");
    g_setup_done[dev] = true;
  }
  *blocks_per_sm = 1;  // one CTA of 1024 threads per SM
  return BC_OK;
}

}  // namespace

int64_t plain_bytes(int32_t n) {
  int64_t N = n + 2, nw = (n + 31) / 32 + 1;
  return N * (4 * 5 + 8 * 6) + nw * 4 * 3 + (int64_t)sizeof(PlainCtl) + 4096;
}

void plain_free(Ctx *ctx, PlainWS *ws) {
  if (!ws->ctl) return;
  void *ptrs[] = {ws->depth, ws->Q, ws->CD, ws->lvl_off, ws->lvl_eoff, ws->sig, ws->ovf,
                  ws->vis, ws->front, ws->acc, ws->r, ws->xm, ws->xe, ws->ctl};
  for (void *q : ptrs) cudaFree(q);
  ctx->mem.release(nullptr, ws->bytes);
  *ws = PlainWS();
}

static bc_status plain_reset(PlainWS *ws, cudaStream_t st) {
  size_t N = (size_t)ws->n + 2, nw = (size_t)(ws->n + 31) / 32 + 1;
  BC_CUDA_TRY(cudaMemsetAsync(ws->depth, 0xff, N * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->sig, 0, N * 8, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->ovf, 0, nw * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->vis, 0, nw * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->front, 0, nw * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->acc, 0, N * 16, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->xe, 0, N * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(PlainCtl), st));
  return BC_OK;
}

bc_status plain_ensure(Ctx *ctx, PlainWS *ws, int32_t n) {
  if (ws->ctl && ws->n == n) return BC_OK;
  plain_free(ctx, ws);
  size_t N = (size_t)n + 2, nw = (size_t)(n + 31) / 32 + 1;
  size_t total = (size_t)plain_bytes(n);
  bc_status s = ctx->mem.alloc(nullptr, total);
  if (s) return s;
  cudaError_t e = cudaSuccess;
#define PA(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void **)&ws->ptr, (bytes));
  PA(depth, N * 4) PA(Q, N * 4) PA(CD, N * 4) PA(lvl_off, N * 4) PA(lvl_eoff, N * 4)
  PA(sig, N * 8) PA(ovf, nw * 4) PA(vis, nw * 4) PA(front, nw * 4) PA(acc, N * 16)
  PA(r, N * 8) PA(xm, N * 8) PA(xe, N * 4) PA(ctl, sizeof(PlainCtl))
#undef PA
  ws->n = n;
  ws->bytes = total;
  if (e != cudaSuccess) {
    cudaGetLastError();
    plain_free(ctx, ws);
    return fail(BC_ENOMEM, std::string("device allocation for the per-source workspace failed: ") +
                               cudaGetErrorString(e));
  }
  s = plain_reset(ws, 0);
  if (s) return s;
  BC_CUDA_TRY(cudaStreamSynchronize(0));
  return BC_OK;
}

// Launch the per-source kernel on a workspace whose arrays the caller has already laid
// out (and cleared: depth -1; sigma, bitmaps, acc, exponents and the control block 0).
// Allocates nothing and creates no events; waits for the kernel and reads its error word
// into *dev_err.
bc_status plain_run_view(const PlainWS &ws, const PlainArgs &a, int num_sms, uint64_t limit_ns,
                         cudaStream_t st, int *dev_err) {
  *dev_err = 0;
  if (a.nsrc <= 0) return BC_OK;
  int bps = 0;
  bc_status s = plain_setup(&bps);
  if (s) return s;
  PK p;
  memset(&p, 0, sizeof(p));
  p.n = a.g->n;
  p.nnz = a.g->nnz;
  p.max_degree = a.max_degree;
  p.rp = a.g->rp;
  p.ci = a.g->ci;
  p.omega = a.omega;
  p.src = a.src;
  p.nsrc = a.nsrc;
  p.bc = a.bc;
  p.leaf_term = a.leaf_term ? 1 : 0;
  p.depth = ws.depth;
  p.Q = ws.Q;
  p.CD = ws.CD;
  p.lvl_off = ws.lvl_off;
  p.lvl_eoff = ws.lvl_eoff;
  p.sig = ws.sig;
  p.ovf = ws.ovf;
  p.vis = ws.vis;
  p.front = ws.front;
  p.acc = ws.acc;
  p.r = ws.r;
  p.xm = ws.xm;
  p.xe = ws.xe;
  p.ctl = ws.ctl;
  p.alpha = a.alpha;
  p.beta = a.beta;
  p.limit_ns = limit_ns;
  void *args[] = {&p};
  cudaError_t le = cudaLaunchCooperativeKernel((void *)plain_kernel, dim3(num_sms * bps),
                                               dim3(kThreads), args, kSmemBytes, st);
  if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(plain_kernel)");
  int err = 0;
  BC_CUDA_TRY(cudaMemcpyAsync(&err, &ws.ctl->bar.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  *dev_err = err;
  return BC_OK;
}

bc_status plain_run(Ctx *ctx, PlainWS *ws, const PlainArgs &a, cudaStream_t st, bc_stats *acc) {
  if (a.nsrc <= 0) return BC_OK;
  int bps = 0;
  {
    const bc_status s = plain_setup(&bps);
    if (s) return s;
  }
  PK p;
  p.n = a.g->n;
  p.nnz = a.g->nnz;
  p.max_degree = a.max_degree;
  p.rp = a.g->rp;
  p.ci = a.g->ci;
  p.omega = a.omega;
  p.src = a.src;
  p.nsrc = a.nsrc;
  p.bc = a.bc;
  p.leaf_term = a.leaf_term ? 1 : 0;
  p.depth = ws->depth;
  p.Q = ws->Q;
  p.CD = ws->CD;
  p.lvl_off = ws->lvl_off;
  p.lvl_eoff = ws->lvl_eoff;
  p.sig = ws->sig;
  p.ovf = ws->ovf;
  p.vis = ws->vis;
  p.front = ws->front;
  p.acc = ws->acc;
  p.r = ws->r;
  p.xm = ws->xm;
  p.xe = ws->xe;
  p.ctl = ws->ctl;
  p.out_depth = a.out_depth;
  p.out_sigma = a.out_sigma;
  p.out_ovf = a.out_ovf;
  p.alpha = a.alpha;
  p.beta = a.beta;
  p.limit_ns = ctx->wait_limit_ns;
  p.trace = nullptr;
  p.trace_cap = 0;
  p.no_cd_reuse = a.no_cd_reuse ? 1 : 0;
  if (a.no_cd_reuse && ctx->num_sms * bps > kPlainScanBlocks)
    return fail(BC_EINVAL, "BC_NO_CD_REUSE: more CTAs than the rescan supports");
  static const char *trace_file = getenv("BC_TRACE_FILE");
  if (trace_file) {
    p.trace_cap = 1 << 20;
    if (cudaMalloc(&p.trace, (size_t)p.trace_cap * 16) != cudaSuccess) {
      cudaGetLastError();
      p.trace = nullptr;
      p.trace_cap = 0;
    }
  }
  dim3 grid(ctx->num_sms * bps), block(kThreads);
  void *args[] = {&p};
  BC_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(PlainCtl), st));
  cudaEvent_t e0, e1;
  BC_CUDA_TRY(cudaEventCreate(&e0));
  BC_CUDA_TRY(cudaEventCreate(&e1));
  BC_CUDA_TRY(cudaEventRecord(e0, st));
  cudaError_t le =
      cudaLaunchCooperativeKernel((void *)plain_kernel, grid, block, args, kSmemBytes, st);
  if (le != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(le, "cudaLaunchCooperativeKernel(plain_kernel)");
  }
  BC_CUDA_TRY(cudaEventRecord(e1, st));
  PlainCtl h;
  BC_CUDA_TRY(cudaMemcpyAsync(&h, ws->ctl, sizeof(PlainCtl), cudaMemcpyDeviceToHost, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (p.trace) {
    int cnt = h.trace_n < p.trace_cap ? h.trace_n : p.trace_cap;
    std::vector<unsigned long long> t((size_t)cnt * 2);
    cudaMemcpy(t.data(), p.trace, (size_t)cnt * 16, cudaMemcpyDeviceToHost);
    cudaFree(p.trace);
    if (FILE *f = fopen(trace_file, "a")) {
      for (int i = 0; i < cnt; i++)
        fprintf(f, "%d,%d,%llu\n", (int)(t[2 * i] >> 56), (int)((t[2 * i] >> 24) & 0xffffffffull),
                t[2 * i + 1]);
      fclose(f);
    }
  }
  if (h.bar.err != 0) {
    bc_status r = plain_reset(ws, st);
    cudaStreamSynchronize(st);
    if (r) return r;
    if (h.bar.err == BCD_TIMEOUT)
      return fail(BC_ETIMEDOUT, "per-source kernel: a grid barrier wait passed its limit");
    return fail(BC_ECUDA, "per-source kernel reported device error " + std::to_string(h.bar.err));
  }
  if (acc) {
    acc->seconds += ms * 1e-3;
    acc->sources += a.nsrc;
    acc->sigma_overflow_sources += h.ovf_sources;
    acc->levels += h.levels;
    acc->kernel_launches += 1;
    acc->reached_vertices += h.reached;
    acc->reached_arcs += h.reached_arcs;
    if (h.max_depth > acc->max_depth) acc->max_depth = h.max_depth;
    if (acc->tile_width == 0) acc->tile_width = 1;
  }
  return BC_OK;
}

}  // namespace bcl

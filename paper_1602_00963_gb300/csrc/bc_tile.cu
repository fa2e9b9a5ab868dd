// Multi-source tile path: T = 32 * G sources per launch (G = 1, 2, 4, 8).
//
// The method is Brandes' (Alg. 1) with the level-synchronous forward sweep of Alg. 2 /
// Alg. 3 and the successor-checking backward sweep of Alg. 4 / Alg. 5, run for T sources
// at once.  Per vertex the tile keeps T-bit masks (one 32-bit word per group of 32
// sources): visited, the frontier of a level (three rotating buffers, reused as the
// dense level masks of the backward sweep) and sigma overflow; per (vertex, source) it
// keeps sigma mod 2^64 and r = (1 + delta + omega) / sigma, laid out [n][T] so that the
// 32 sources of a group are 32 consecutive words read by the 32 lanes of a warp.
//
// Forward level l:
//   * top-down (small frontiers): a marking pass over the edges of the active vertices
//     A_{l-1} flags every neighbour w with F[p] & ~vis[w] != 0 as a candidate;
//   * bottom-up (large frontiers): every vertex not yet visited by all sources is a
//     candidate;
//   * pull: each candidate w sums, lane by lane, sigma over all neighbours p whose frontier
//     mask has the lane's bit (all parents at level l-1, no early exit, so sigma is
//     exact), sets its new mask and is appended to A_l.  No sigma atomics are needed.
// Backward level d (Alg. 5 with updateDep): each entry (w, M_w) of A_d sums r[v] over the
// neighbours v whose level-(d+1) mask shares bits with M_w; then delta = sigma * sum,
// BC[w] += sum over lanes of (omega[s]+1) * delta (fixed lane order) and r[w] = (1 +
// omega[w]) / sigma + sum.  r and its sums are float-float pairs (bc_ff.cuh): FP64 is slow
// on this GPU, and only the per-vertex BC update uses it.
//
// Work mapping (active-edge parallelism, Sec. 3.1): every list that is walked (active
// vertices, candidates, all vertices) carries an exclusive degree prefix, produced by the
// packed (count, edges) append counter or built once per graph.  A warp takes ranges of
// the concatenated adjacency (a static first range, then guided claims), snapped to
// list-entry starts so each entry belongs to one warp, and maps edge -> entry by a search
// in the prefix.  Lanes are edges for the frontier-mask tests; a hit of at most two
// sources is loaded by its own lane, denser hits are gathered as sigma / r rows by the
// source lanes.  Levels whose entries average at most two sources and 16 edges (high-
// diameter graphs) run one entry per lane instead.  High-degree vertices are cut into
// chunks of p.hub_chunk edges at fixed offsets (forward candidates of degree >= p.hub,
// backward entries of degree >= p.hub_chunk), each a warp work item taken from a counter
// as soon as a warp's walk is done; the warp finishing a vertex's last chunk adds the
// chunks' partial sums in chunk order and commits.
// Warp-level work is numbered across CTAs first.  σ, depth and the masks are exact.  Every
// floating-point sum has a fixed order: an entry walked warp-wide adds its hits in edge
// order (wherever the warps' run-time range claims put the 32-edge steps), the lane-per-
// entry mode walks an entry's edges in order, work items split an adjacency at fixed
// offsets and their partials are summed in chunk order, and BC takes one update per
// (vertex, level) in level order.  So r and BC repeat bit for bit from run to run.
//
// sigma beyond 2^64: a tile first runs with r computed from sigma mod 2^64; if any count
// overflowed, the tile is rerun (before any BC update) in extended mode, where each
// overflowed (vertex, source) also carries sigma as a double mantissa and int exponent.
//
// Three ways to run the level loop over the same phase bodies: a persistent cooperative
// kernel with bounded grid barriers (loop_mode 0), one launch per phase (1), and the
// per-phase launches of kLevelsPerChunk levels captured once as a CUDA graph and
// replayed until the level loop ends (2).
#include <climits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bc_ff.cuh"
#include "bc_internal.h"
#include "bc_scan.cuh"

namespace bcl {

namespace {

constexpr int kHubDefault = 512;        // forward: candidates of this degree or more are split
                                        // into warp work items (below)
constexpr int kHubChunkDefault = 256;   // backward: entries of this degree or more are split
                                        // into warp work items of this many edges
constexpr int kLevelsPerChunk = 8;  // levels per launched chunk / captured graph
constexpr int BCD_NEEDEXT = 4;      // device code: rerun the tile in extended mode

template <int G>
struct TPB {  // threads per CTA (one CTA per SM): 256-wide tiles keep more state per lane
  static constexpr int value = G >= 8 ? 768 : 1024;
};
// hits whose row gathers are in flight together: one for tiles of 128 sources or more, whose
// rows already issue G / 2 vector loads per lane (more rows in flight there spill registers
// at 64 per thread: 2.5 KB per thread at T = 128 with four rows, 0.4 KB with one, and the
// tile runs 23 % faster)
template <int G>
struct HB {
  static constexpr int value = G >= 4 ? 1 : (G >= 2 ? 4 : 8);
};

struct TileCtl {
  GridSync bar;
  unsigned long long apack[3];  // per-level append counter of A: count << 32 | edges (slot l % 3)
  unsigned long long cpack[3];  // per-level candidates C: count << 32 | edges (slot l % 3)
  unsigned long long chpk[3];   // per-level hub candidates: count << 32 | chunks (slot l % 3)
  int hecnt;                    // hub entries listed in HE
  int hubq[3];                  // forward hub work counter (slot l % 3)
  int bhubq[3];                 // backward hub work counter (slot d % 3)
  unsigned long long wq[3];     // forward pull walk: edges claimed (slot l % 3)
  unsigned long long bq[3];     // backward walk: edges claimed (slot d % 3)
  int ovf_any;                  // some sigma of this tile passed 2^64
  unsigned ovf_lanes[8];        // lanes (sources) with an overflowed sigma
  // launched / graph mode registers
  int level, mode, pmode, done, lmax, dlevel;  // pmode: the previous level's direction
  int a_pp, a_lo, a_hi, ecnt;
  long long levels;
  int trace_n;
  unsigned long long reached;       // (vertex, source) pairs reached
  unsigned long long reached_arcs;  // their adjacency entries
  unsigned long long ns[256];   // Eq. 3 component size per lane (leaf term)
};

}  // namespace

struct TileWS {
  int n = 0, T = 0, G = 0;
  int64_t capA = 0;
  bool ext_arrays = false;
  bool ext_sticky = false;  // this graph needed extended sigma before: start tiles in it
  uint32_t *vis = nullptr, *F = nullptr, *ovf = nullptr, *cand = nullptr;
  unsigned long long *sig = nullptr;
  float2 *r = nullptr;  // float-float r values
  double *xm = nullptr;
  int32_t *xe = nullptr;
  int32_t *A = nullptr, *ACD = nullptr, *ARP = nullptr;
  uint32_t *AM = nullptr;
  int32_t *Aoff = nullptr;
  unsigned long long *Lbits = nullptr;
  int32_t *HE = nullptr, *HEoff = nullptr;  // hub work items (A positions), per-level offsets
  int32_t *HEk = nullptr, *Hdone = nullptr;  // item's chunk number; chunks done per hub entry
  float2 *Hpart = nullptr;                   // per-item partial sums (one level's items)
  uint32_t *FPm = nullptr;                   // forward items: masks and overflow bits
  double *FPx = nullptr;                     // forward items, extended range
  int32_t *FPe = nullptr;
  int64_t hpart_items = 0, hpart_ext_items = 0;
  size_t bytes_hpart = 0, bytes_hpart_ext = 0;
  int32_t *C = nullptr, *CPD = nullptr, *CRP = nullptr, *Ch = nullptr, *ChP = nullptr;
  int32_t *Fdone = nullptr;  // forward: finished chunks per split candidate
  float2 *wsrc = nullptr;
  TileCtl *ctl = nullptr;
  size_t bytes_main = 0, bytes_ext = 0, bytes_A = 0;
  // per-graph lists: hubs (degree >= hub) and the bottom-up walk list (others, deg > 0)
  const int32_t *lists_for = nullptr;
  int lists_hub = 0, lists_chunk = 0;  // hub degree and chunk the lists were built for
  int32_t *hubs = nullptr, *Lbu = nullptr, *PDbu = nullptr, *RPbu = nullptr, *HPbu = nullptr;
  int nhubs = 0, nbu = 0, Ebu = 0, nhub_items = 0;
  size_t bytes_lists = 0;
};

namespace {

struct TK {
  int n;
  long long nnz;
  int nsrc;
  const int32_t *__restrict__ rp;
  const int32_t *__restrict__ ci;
  const int32_t *__restrict__ omega;
  const int32_t *__restrict__ src;
  double *bc;
  int leaf_term;
  uint32_t *vis, *F, *ovf, *cand;
  unsigned long long *sig;
  float2 *r;  // r = (1 + delta + omega) / sigma per (vertex, source), float-float
  double *xm;
  int32_t *xe;
  int32_t *A, *ACD, *ARP;  // active list: vertex, level-relative edge prefix, row_ptr of the vertex
  uint32_t *AM;
  long long capA;
  int32_t *Aoff;
  unsigned long long *Lbits;  // per level l: total number of sources over the entries of A_l
  int32_t *HE, *HEoff;
  int32_t *HEk, *Hdone;  // backward hub items: chunk number; finished chunks of the entry
  float2 *Hpart;         // [items of a level][T] partial r sums of hub chunks
  unsigned long long *FPs;  // forward items: [items][T] partial sigma sums (shares Hpart)
  uint32_t *FPm;            // forward items: [items][2G] new-level masks, overflow bits
  double *FPx;              // forward items, extended range: [items][T] mantissas
  int32_t *FPe;             //   and exponents
  int32_t *Fdone;           // forward: finished chunks per split candidate (list position)
  const int32_t *HPbu;      // bottom-up: exclusive prefix of the hubs' chunk counts
  int nhub_items;           // bottom-up: items of all hubs
  int32_t *C, *CPD, *CRP, *Ch, *ChP;
  const int32_t *hubs, *Lbu, *PDbu, *RPbu;
  int nhubs, nbu, Ebu;
  float2 *wsrc;  // per source: omega(s) + 1, float-float
  TileCtl *ctl;
  uint32_t unused[8];
  float alpha;  // top-down -> bottom-up when the frontier's edges exceed alpha * nnz
  float beta;   // > 0: stay bottom-up while the frontier's edges exceed nnz / beta
  int hub;        // degree from which a vertex is processed by whole CTAs / chunked
  int hub_chunk;  // edges of a hub per backward work item
  uint64_t limit_ns;
  int nreq;                       // > 0: lanes route BC to per-request buffers (serving)
  const uint8_t *lane_req;        // [T] request slot of each lane
  double *const *req_bc;          // [nreq] device BC buffers
  unsigned long long *trace;  // optional phase trace: (phase << 56 | level << 24, time) pairs
  int trace_cap;
};

// Grid barrier; with tracing on, CTA 0 stamps the time at which every CTA has finished
// the phase.
__device__ __forceinline__ bool tsync(const TK &p, GridSync *gs, int phase, int level) {
  const bool ok = grid_sync(gs, p.limit_ns);
  if (p.trace && blockIdx.x == 0 && threadIdx.x == 0) {
    const int i = p.ctl->trace_n++;
    if (i < p.trace_cap) {
      p.trace[2 * i] = ((unsigned long long)phase << 56) | ((unsigned long long)(unsigned)level << 24);
      p.trace[2 * i + 1] = globaltimer_ns();
    }
  }
  return ok;
}

template <int G>
__device__ __forceinline__ uint32_t *Fbuf(const TK &p, int l) {
  return p.F + (size_t)(l % 3) * (size_t)p.n * G;
}
__device__ __forceinline__ unsigned long long vload64(const unsigned long long *a) {
  return *(const volatile unsigned long long *)a;
}
__device__ __forceinline__ int vdeg(const TK &p, int v) { return p.rp[v + 1] - p.rp[v]; }
// Warp index for warp-level work, interleaved across CTAs (warp i of every CTA before warp
// i + 1 of any), so that a level with few work units still spreads over all SMs.
__device__ __forceinline__ int warp_rank() { return (int)((threadIdx.x >> 5) * gridDim.x + blockIdx.x); }
// Position of source t = 32 g + lane in vertex v's row of a per-(vertex, source) array
// ([n][T]: sigma, r, the extended-range arrays): a lane's G sources are adjacent, so a lane
// reads all of its sources of a row with vector loads.
template <int G>
__device__ __forceinline__ size_t sidx(long long v, int g, int lane) {
  return (size_t)v * (32 * G) + (size_t)lane * G + g;
}
template <int G>
__device__ __forceinline__ size_t sidx(long long v, int t) {
  return sidx<G>(v, t >> 5, t & 31);
}

// A lane's G adjacent values of a row (a = row + lane * G), in 16-byte vector loads.
template <int G>
__device__ __forceinline__ void load_lane(const unsigned long long *a, unsigned long long (&out)[G]) {
  if constexpr (G == 1) {
    out[0] = a[0];
  } else {
#pragma unroll
    for (int q = 0; q < G / 2; q++) {
      const ulonglong2 x = ((const ulonglong2 *)a)[q];
      out[2 * q] = x.x;
      out[2 * q + 1] = x.y;
    }
  }
}
template <int G>
__device__ __forceinline__ void load_lane(const float2 *a, float2 (&out)[G]) {
  if constexpr (G == 1) {
    out[0] = a[0];
  } else {
#pragma unroll
    for (int q = 0; q < G / 2; q++) {
      const float4 x = ((const float4 *)a)[q];
      out[2 * q] = make_float2(x.x, x.y);
      out[2 * q + 1] = make_float2(x.z, x.w);
    }
  }
}

// Ask L2 for the 128-byte lines of a [32][G] row of 8-byte values (lane-major) that hold the
// sources of mask m.  Dense hits gather their rows a few at a time, later in the step; lines
// requested here are then on their way while the rows before them are summed.
template <int G>
__device__ __forceinline__ void prefetch_row(const void *row, const uint32_t (&m)[G]) {
  constexpr int L = 16 / G;  // lanes per line
  uint32_t u = 0u;
#pragma unroll
  for (int g = 0; g < G; g++) u |= m[g];
#pragma unroll
  for (int k = 0; k < 2 * G; k++)
    if ((u >> (k * L)) & ((1u << L) - 1u))
      asm volatile("prefetch.global.L2 [%0];" ::"l"((const char *)row + 128 * k));
}

// Row v of a [n][G] mask array in one or two vector loads (rows are 4G-byte aligned).
template <int G>
__device__ __forceinline__ void load_row(const uint32_t *a, long long v, uint32_t (&out)[G]) {
  const uint32_t *r = a + (size_t)v * G;
  if constexpr (G == 1) {
    out[0] = r[0];
  } else if constexpr (G == 2) {
    const uint2 x = *(const uint2 *)r;
    out[0] = x.x;
    out[1] = x.y;
  } else {
#pragma unroll
    for (int q = 0; q < G / 4; q++) {
      const uint4 x = ((const uint4 *)r)[q];
      out[4 * q] = x.x;
      out[4 * q + 1] = x.y;
      out[4 * q + 2] = x.z;
      out[4 * q + 3] = x.w;
    }
  }
}

// Warp-aggregated append of the flagged lanes' vertices to A with its packed counter.
__device__ __forceinline__ void append_A(const TK &p, unsigned long long *ctr, int base_off,
                                         bool flag, int v) {
  unsigned m = __ballot_sync(BC_FULL, flag);
  if (!m) return;
  const int r0 = flag ? p.rp[v] : 0;
  int deg = flag ? p.rp[v + 1] - r0 : 0;
  int tot;
  int pre = warp_excl_scan(deg, &tot);
  unsigned long long b = 0;
  int leader = __ffs(m) - 1;
  if ((int)lane_id() == leader) b = atomicAdd(ctr, pack_qe(__popc(m), (unsigned)tot));
  b = __shfl_sync(BC_FULL, b, leader);
  if (flag) {
    long long pos = (long long)base_off + (long long)(b >> 32) + __popc(m & lanemask_lt());
    if (pos < p.capA) {
      p.A[pos] = v;
      p.ACD[pos] = (int)(b & 0xffffffffull) + pre;
      p.ARP[pos] = r0;
      if (deg >= p.hub_chunk) {  // listed for the backward sweep too, one warp item per chunk
        const int nch = (deg + p.hub_chunk - 1) / p.hub_chunk;
        const int hp = atomicAdd(&p.ctl->hecnt, nch);
        if ((long long)hp + nch <= p.capA) {
          for (int c = 0; c < nch; c++) {
            p.HE[hp + c] = (int)pos;
            p.HEk[hp + c] = c;
          }
          p.Hdone[hp] = 0;
        } else {
          atomicCAS(&p.ctl->bar.err, 0, BCD_CAPACITY);
        }
      }
    } else {
      atomicCAS(&p.ctl->bar.err, 0, BCD_CAPACITY);
    }
  }
}

// Per-warp buffer of committed vertices: one atomic per 32 appends.
struct AppendBuf {
  int v;  // lane i holds the i-th pending vertex
  int n;  // pending count (uniform)
};
__device__ __forceinline__ void abuf_push(const TK &p, AppendBuf &b, int w,
                                          unsigned long long *ctr, int base_off) {
  if ((int)lane_id() == b.n) b.v = w;
  if (++b.n == 32) {
    append_A(p, ctr, base_off, true, b.v);
    b.n = 0;
  }
}
__device__ __forceinline__ void abuf_flush(const TK &p, AppendBuf &b, unsigned long long *ctr,
                                           int base_off) {
  append_A(p, ctr, base_off, (int)lane_id() < b.n, b.v);
  b.n = 0;
}

// ------------------------------------------------------------------ extended sigma
__device__ __forceinline__ XS sig_xs(const TK &p, size_t idx, bool o) {
  if (o) {
    XS x;
    x.m = p.xm[idx];
    x.e = p.xe[idx];
    return x;
  }
  return xs_u64(p.sig[idx]);
}

// ------------------------------------------------------------------ the edge walk
// Largest i in [lo, hi) with PD[i] <= x (PD non-decreasing, PD[lo] <= x).
__device__ __forceinline__ int find_owner(const int32_t *PD, int lo, int hi, int x) {
  const int lane = lane_id();
  while (hi - lo > 32) {
    int stride = (hi - lo + 31) / 32;
    int pos = lo + lane * stride;
    unsigned b = __ballot_sync(BC_FULL, pos < hi && PD[pos] <= x);
    lo = lo + (31 - __clz(b)) * stride;
    hi = min(lo + stride, hi);
  }
  int pos = lo + lane;
  unsigned b = __ballot_sync(BC_FULL, pos < hi && PD[pos] <= x);
  return lo + (31 - __clz(b));
}

// Walk the adjacency of list entries [i_lo, i_hi) (entry i: vertex L[i], whose row starts
// at RP[i] = row_ptr[L[i]] and whose edges start at the level-relative prefix PD[i]; E edges
// in all), restricted to the entries that start inside the edge range [eb, ee): ranges are
// snapped to entry starts, so each entry is walked by exactly one warp.  With SKIP_HUBS,
// entries of degree >= skip_deg are jumped over (an entry's degree is the difference of
// consecutive prefixes, already in registers).  f(valid, k, w, col) is called once per
// 32-edge step (lane = edge) with the warp converged: k = entry, w = its vertex, col =
// position of the edge in col_idx.  A step's window of 32 entries is one round of
// independent loads (PD, L, RP).
template <bool SKIP_HUBS, typename F>
__device__ __forceinline__ void walk_range(const TK &p, const int32_t *L, const int32_t *PD,
                                           const int32_t *RP, int i_lo, int i_hi, int E, int eb, int ee,
                                           int skip_deg, F &&f) {
  const int lane = lane_id();
  int i0 = find_owner(PD, i_lo, i_hi, eb);
  if (PD[i0] < eb) i0++;
  if (i0 >= i_hi || PD[i0] >= ee) return;
  const int i1 = (ee >= E) ? i_hi : find_owner(PD, i0, i_hi, ee - 1) + 1;
  const int e_end = (i1 < i_hi) ? PD[i1] : E;
  int base = i0, e = PD[i0];
  while (e < e_end) {
    const int idx = base + lane;
    const bool in = idx < i1;
    const int cd = in ? PD[idx] : INT_MAX;
    const int vv = in ? L[idx] : 0;
    const int bias = in ? RP[idx] - cd : 0;
    const int cd_after = (base + 32 < i1) ? PD[base + 32] : e_end;
    // prefix of the next entry (its edges' start), so degree = nx - cd
    int nx = __shfl_down_sync(BC_FULL, cd, 1);
    if (lane == 31) nx = cd_after;
    if (idx + 1 >= i1) nx = e_end;
    const unsigned hubm = SKIP_HUBS ? __ballot_sync(BC_FULL, in && nx - cd >= skip_deg) : 0u;
    if (SKIP_HUBS && (hubm & 1u)) {  // the step would start inside a hub: jump over it
      e = __shfl_sync(BC_FULL, nx, 0);
      base++;
      continue;
    }
    const int my = e + lane;
    const int j = warp_owner(cd, my);
    const int w = __shfl_sync(BC_FULL, vv, j);
    const int col = my + __shfl_sync(BC_FULL, bias, j);
    bool valid = my < e_end;
    if (SKIP_HUBS) valid = valid && !((hubm >> j) & 1u);
    f(valid, base + j, w, col);
    const int j31 = __shfl_sync(BC_FULL, j, 31);
    int nxt = __shfl_sync(BC_FULL, cd, min(j31 + 1, 31));
    if (j31 == 31) nxt = cd_after;
    const int nb = base + j31 + ((e + 32 >= nxt) ? 1 : 0);
    e += 32;
    base = nb;
  }
}

// The walk over all E edges: each warp first takes a static chunk (number gwarp), then
// claims further ranges from a shared edge counter, guided: a claim takes about half the
// remaining edges' per-warp share, between 32 and kChunk, so that ranges shrink towards
// the end of the level and warps finish together.  The next range is claimed before the
// current one is walked, hiding the atomic's latency.
constexpr int kChunk = 1024;

template <bool SKIP_HUBS, typename F>
__device__ __forceinline__ void walk(const TK &p, const int32_t *L, const int32_t *PD, const int32_t *RP,
                                     int i_lo, int i_hi, int E, int gwarp, int nwarps, unsigned long long *ctr,
                                     int skip_deg, F &&f) {
  if (E <= 0 || i_hi <= i_lo) return;
  long long ch = ((long long)E / (4ll * nwarps) + 31) & ~31ll;
  ch = ch < 32 ? 32 : (ch > kChunk ? kChunk : ch);
  const long long base0 = ch * nwarps;  // edges of the static first chunks
  long long eb = (long long)gwarp * ch;
  long long ee = min(eb + ch, (long long)E);
  while (eb < E) {
    long long nb = E, ne = E;
    if (base0 < E) {
      long long off = 0, sz = 0;
      if (lane_id() == 0) {
        const long long left = (long long)E - base0 - (long long)*(volatile unsigned long long *)ctr;
        if (left > 0) {
          sz = ((left / (2ll * nwarps)) + 31) & ~31ll;
          sz = sz < 32 ? 32 : (sz > kChunk ? kChunk : sz);
          off = (long long)atomicAdd(ctr, (unsigned long long)sz);
        } else {
          off = (long long)E;  // nothing left
        }
      }
      off = __shfl_sync(BC_FULL, off, 0);
      sz = __shfl_sync(BC_FULL, sz, 0);
      nb = min(base0 + off, (long long)E);
      ne = min(nb + sz, (long long)E);
    }
    walk_range<SKIP_HUBS>(p, L, PD, RP, i_lo, i_hi, E, (int)eb, (int)ee, skip_deg, f);
    eb = nb;
    ee = ne;
  }
}

// ------------------------------------------------------------------ forward pull
template <int G, bool EXT>
struct PullAcc {
  unsigned long long s[G];
  uint32_t o;   // per-lane overflow bits, bit g
  uint32_t cy;  // 64-bit mode: carries out of this lane's additions (any group)
  uint32_t newm[G];
  XS x[EXT ? G : 1];
};

// s += v with the carry out of bit 63 counted in cy (one carry-chained pair of adds).
__device__ __forceinline__ void add_carry(unsigned long long &s, uint32_t &cy, unsigned long long v) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(s), "+r"(cy) : "l"(v));
}

// Sparse forward terms in 64-bit mode on tiles of up to 128 sources: per warp, one 64-bit
// accumulator per source in shared memory.  A sparse hit's lane adds its (source, sigma)
// pairs with shared atomics (integer sums, so their order does not matter) and the owner's
// lanes fold the accumulators in before committing, leaving them zero.
template <int G>
__device__ __forceinline__ unsigned long long *sparse_acc() {
  __shared__ unsigned long long s_acc[G <= 4 ? 32 * 32 * G : 1];
  return s_acc + (size_t)(threadIdx.x >> 5) * (32 * G);
}
template <int G>
__device__ __forceinline__ void sparse_acc_clear() {
  if constexpr (G <= 4) {
    unsigned long long *a = sparse_acc<G>() - (size_t)(threadIdx.x >> 5) * (32 * G);
    for (int i = threadIdx.x; i < 32 * 32 * G; i += blockDim.x) a[i] = 0ull;
    __syncthreads();
  }
}

template <int G, bool EXT>
__device__ __forceinline__ void pull_init(PullAcc<G, EXT> &a) {
  a.o = 0u;
  a.cy = 0u;
#pragma unroll
  for (int g = 0; g < G; g++) {
    a.s[g] = 0ull;
    a.newm[g] = 0u;
    if (EXT) {
      a.x[g].m = 0.0;
      a.x[g].e = 0;
    }
  }
}

// Add the sigma row of frontier vertex pn (lane masks m) to the accumulator.
template <int G, bool EXT>
__device__ __forceinline__ void pull_hit(const TK &p, int pn, const uint32_t (&m)[G],
                                         PullAcc<G, EXT> &a) {
  const int lane = lane_id();
#pragma unroll
  for (int g = 0; g < G; g++) {
    a.newm[g] |= m[g];
    if ((m[g] >> lane) & 1u) {
      const size_t idx = sidx<G>(pn, g, lane);
      const unsigned long long sv = p.sig[idx];
      const unsigned long long old = a.s[g];
      a.s[g] = old + sv;
      // 64-bit mode: an overflowed parent has already flagged the tile for the extended
      // rerun, so only this addition's carry is checked
      const bool po = EXT && ((p.ovf[(size_t)pn * G + g] >> lane) & 1u);
      if (a.s[g] < old || po) a.o |= 1u << g;
      if (EXT) {
        XS y;
        if (po) {
          y.m = p.xm[idx];
          y.e = p.xe[idx];
        } else {
          y = xs_u64(sv);
        }
        xs_add(a.x[g], y);
      }
    }
  }
}

// Store the pulled sigma of w for the lanes that reached it at this level and set its
// vis / F / ovf words (lane g writes word g).  Returns whether any lane reached w.
template <int G, bool EXT>
__device__ __forceinline__ bool pull_commit(const TK &p, int w, int level, const PullAcc<G, EXT> &a,
                                            const uint32_t (&visw)[G], bool leaf,
                                            unsigned long long (&nsacc)[G]) {
  const int lane = lane_id();
  bool any = false;
  uint32_t *Fn = Fbuf<G>(p, level);
#pragma unroll
  for (int g = 0; g < G; g++) {
    const uint32_t m = a.newm[g];
    if (!m) continue;
    any = true;
    const bool mine = (m >> lane) & 1u;
    const bool og = ((a.o >> g) & 1u) || (!EXT && a.cy != 0u);
    const size_t idx = sidx<G>(w, g, lane);
    if (mine) {
      p.sig[idx] = a.s[g];
      if (EXT && og) {
        XS x = xs_norm(a.x[g]);
        p.xm[idx] = x.m;
        p.xe[idx] = x.e;
      }
      if (leaf) nsacc[g] += 1ull + (unsigned long long)p.omega[w];
    }
    const unsigned ob = __ballot_sync(BC_FULL, mine && og);
    if (lane == g) {
      p.vis[(size_t)w * G + g] = visw[g] | m;
      Fn[(size_t)w * G + g] = m;
      if (ob) {
        p.ovf[(size_t)w * G + g] |= ob;
        p.ctl->ovf_any = 1;
        atomicOr(&p.ctl->ovf_lanes[g], ob);
      }
    }
  }
  return any;
}

template <int G>
__device__ __forceinline__ bool load_vis(const TK &p, int w, uint32_t (&visw)[G]) {
  bool full = true;
  load_row<G>(p.vis, w, visw);
#pragma unroll
  for (int g = 0; g < G; g++) full &= visw[g] == 0xffffffffu;
  return full;
}

// Up to two set bits of a lane's G-word source mask (source 32 g + bit; -1 where absent).
// Returns the number of set bits.
template <int G>
__device__ __forceinline__ int two_bits(const uint32_t (&b)[G], int &t0, int &t1) {
  int n = 0;
  t0 = t1 = -1;
#pragma unroll
  for (int g = 0; g < G; g++) {
    uint32_t x = b[g];
    n += __popc(x);
    if (x && t0 < 0) {
      t0 = 32 * g + __ffs(x) - 1;
      x &= x - 1;
    }
    if (x && t1 < 0) t1 = 32 * g + __ffs(x) - 1;
  }
  return n;
}

// A hit of at most kSparse sources (typical of high-diameter graphs, where the sources
// of a tile rarely share a level) is loaded by its own edge lane, so all such hits of a
// 32-edge step are in flight together; the owner's lanes then take them by shuffles.
constexpr int kSparse = 2;

// One sparse forward term: source t gets sigma s (overflow flag po, extended value x).
template <int G, bool EXT>
__device__ __forceinline__ void pull_sparse_add(PullAcc<G, EXT> &a, int t, unsigned long long s, bool po,
                                                XS x) {
  const int lane = lane_id();
#pragma unroll
  for (int g = 0; g < G; g++) {
    if ((t >> 5) != g) continue;
    a.newm[g] |= 1u << (t & 31);
    if (lane == (t & 31)) {
      const unsigned long long old = a.s[g];
      a.s[g] = old + s;
      if (a.s[g] < old || po) a.o |= 1u << g;
      if (EXT) xs_add(a.x[g], x);
    }
  }
}

// One forward edge per lane: frontier neighbour pj and the sources bm it brings to the
// owner; hits of at most kSparse sources carry their own sigma values.
template <int G, bool EXT>
struct FwdHit {
  int pj;
  uint32_t bm[G];
  bool hit, sp;
  int t0, t1;
  unsigned long long s0, s1;
  bool o0, o1;
  XS x0, x1;
};

template <int G, bool EXT>
__device__ __forceinline__ void fwd_hit_load(const TK &p, FwdHit<G, EXT> &h) {
  h.t0 = h.t1 = -1;
  h.sp = h.hit && two_bits<G>(h.bm, h.t0, h.t1) <= kSparse;
  h.s0 = h.s1 = 0ull;
  h.o0 = h.o1 = false;
  h.x0.m = h.x1.m = 0.0;
  h.x0.e = h.x1.e = 0;
  if (!h.sp) return;
  const size_t i0 = sidx<G>(h.pj, h.t0);
  h.s0 = p.sig[i0];
  h.o0 = EXT && ((p.ovf[(size_t)h.pj * G + (h.t0 >> 5)] >> (h.t0 & 31)) & 1u);
  const size_t i1 = sidx<G>(h.pj, (h.t1 >= 0 ? h.t1 : h.t0));
  if (h.t1 >= 0) {
    h.s1 = p.sig[i1];
    h.o1 = EXT && ((p.ovf[(size_t)h.pj * G + (h.t1 >> 5)] >> (h.t1 & 31)) & 1u);
  }
  if (EXT) {
    if (h.o0) {
      h.x0.m = p.xm[i0];
      h.x0.e = p.xe[i0];
    } else {
      h.x0 = xs_u64(h.s0);
    }
    if (h.t1 >= 0) {
      if (h.o1) {
        h.x1.m = p.xm[i1];
        h.x1.e = p.xe[i1];
      } else {
        h.x1 = xs_u64(h.s1);
      }
    }
  }
}

// Add the hits of lanes hs (sparse) and hd (the others), all of one owner, to a: sparse
// terms by shuffles, the others by sigma-row gathers (HB<G> rows in flight together).
// Integer sums do not depend on their order; the extended-range sums (EXT) are floating
// point, so there every hit is taken in lane (edge) order, sparse or not.
template <int G, bool EXT>
__device__ __forceinline__ void fwd_sparse_take(const FwdHit<G, EXT> &h, int jj, PullAcc<G, EXT> &a) {
  const int u0 = __shfl_sync(BC_FULL, h.t0, jj), u1 = __shfl_sync(BC_FULL, h.t1, jj);
  XS y0, y1;
  y0.m = y1.m = 0.0;
  y0.e = y1.e = 0;
  if (EXT) {
    y0.m = __shfl_sync(BC_FULL, h.x0.m, jj);
    y0.e = __shfl_sync(BC_FULL, h.x0.e, jj);
  }
  pull_sparse_add<G, EXT>(a, u0, __shfl_sync(BC_FULL, h.s0, jj), __shfl_sync(BC_FULL, h.o0, jj), y0);
  if (u1 >= 0) {
    if (EXT) {
      y1.m = __shfl_sync(BC_FULL, h.x1.m, jj);
      y1.e = __shfl_sync(BC_FULL, h.x1.e, jj);
    }
    pull_sparse_add<G, EXT>(a, u1, __shfl_sync(BC_FULL, h.s1, jj), __shfl_sync(BC_FULL, h.o1, jj), y1);
  }
}

template <int G, bool EXT>
__device__ __forceinline__ void fwd_hits_add(const TK &p, const FwdHit<G, EXT> &h, unsigned hs, unsigned hd,
                                             PullAcc<G, EXT> &a) {
  const int lane = lane_id();
  if (EXT) {
    unsigned hm = hs | hd;
    while (hm) {
      const int jj = __ffs(hm) - 1;
      hm &= hm - 1;
      if ((hs >> jj) & 1u) {
        fwd_sparse_take<G, EXT>(h, jj, a);
      } else {
        uint32_t m[G];
#pragma unroll
        for (int g = 0; g < G; g++) m[g] = __shfl_sync(BC_FULL, h.bm[g], jj);
        pull_hit<G, EXT>(p, __shfl_sync(BC_FULL, h.pj, jj), m, a);
      }
    }
    return;
  }
  if constexpr (G <= 4) {  // each sparse lane adds its pairs to the warp's accumulators
    if (hs) {
      unsigned long long *sa = sparse_acc<G>();
      bool carry = false;
      uint32_t nb[G];
#pragma unroll
      for (int g = 0; g < G; g++) nb[g] = 0u;
      if ((hs >> lane) & 1u) {
        unsigned long long old = atomicAdd(&sa[h.t0], h.s0);
        carry = old + h.s0 < old;
        if (h.t1 >= 0) {
          old = atomicAdd(&sa[h.t1], h.s1);
          carry = carry || old + h.s1 < old;
        }
#pragma unroll
        for (int g = 0; g < G; g++) {
          if ((h.t0 >> 5) == g) nb[g] |= 1u << (h.t0 & 31);
          if (h.t1 >= 0 && (h.t1 >> 5) == g) nb[g] |= 1u << (h.t1 & 31);
        }
      }
#pragma unroll
      for (int g = 0; g < G; g++) a.newm[g] |= __reduce_or_sync(BC_FULL, nb[g]);
      if (__ballot_sync(BC_FULL, carry)) a.cy |= 1u;
    }
  } else {
    while (hs) {
      const int jj = __ffs(hs) - 1;
      hs &= hs - 1;
      fwd_sparse_take<G, EXT>(h, jj, a);
    }
  }
  // 64-bit mode (EXT is handled above): an overflowed parent has already flagged the tile
  // for the extended rerun, so only the additions' carries are checked
  while (hd) {
    unsigned long long sv[HB<G>::value][G];
    uint32_t mq[HB<G>::value][G];
#pragma unroll
    for (int q = 0; q < HB<G>::value; q++) {
      const int jq = hd ? __ffs(hd) - 1 : -1;
      if (hd) hd &= hd - 1;
      const int pn = __shfl_sync(BC_FULL, h.pj, jq < 0 ? 0 : jq);
      bool mine = false;
#pragma unroll
      for (int g = 0; g < G; g++) {
        const uint32_t m = __shfl_sync(BC_FULL, h.bm[g], jq < 0 ? 0 : jq);
        mq[q][g] = jq < 0 ? 0u : m;
        mine |= (mq[q][g] >> lane) & 1u;
      }
      if (mine) {  // the lane's G values of the row in vector loads
        load_lane<G>(p.sig + sidx<G>(pn, 0, lane), sv[q]);
#pragma unroll
        for (int g = 0; g < G; g++)
          if (!((mq[q][g] >> lane) & 1u)) sv[q][g] = 0ull;
      } else {
#pragma unroll
        for (int g = 0; g < G; g++) sv[q][g] = 0ull;
      }
    }
#pragma unroll
    for (int q = 0; q < HB<G>::value; q++) {
#pragma unroll
      for (int g = 0; g < G; g++) {
        a.newm[g] |= mq[q][g];
        add_carry(a.s[g], a.cy, sv[q][g]);
      }
    }
  }
}

// 64-bit mode, tiles of up to 128 sources: fold the warp's shared sparse accumulators of the
// current owner into a and clear them (before every commit of a pulled vertex).
template <int G, bool EXT>
__device__ __forceinline__ void sparse_fold(PullAcc<G, EXT> &a) {
  if constexpr (!EXT && G <= 4) {
    unsigned long long *sa = sparse_acc<G>();
    const int lane = lane_id();
    __syncwarp();
#pragma unroll
    for (int g = 0; g < G; g++) {
      const unsigned long long v = sa[32 * g + lane];
      if (v) {
        add_carry(a.s[g], a.cy, v);
        sa[32 * g + lane] = 0ull;
      }
    }
    __syncwarp();
  }
}

// Forward pull over the walk of list L: lanes test the edges' frontier masks against their
// owner's unvisited mask; then, owner by owner, the sparse hits (loaded by their lanes)
// and the other hits (sigma rows gathered by the source lanes) are summed, each set in
// edge order.
template <int G, bool EXT>
__device__ void pull_walk(const TK &p, int level, const int32_t *L, const int32_t *PD, const int32_t *RP, int n_list,
                          int E, int gwarp, int nwarps, AppendBuf &ab, unsigned long long *ap,
                          int a_base, bool leaf, unsigned long long (&nsacc)[G]) {
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  int cur = -1;
  uint32_t visc[G];
  PullAcc<G, EXT> a;
  pull_init(a);
#pragma unroll
  for (int g = 0; g < G; g++) visc[g] = 0u;
  walk<false>(p, L, PD, RP, 0, n_list, E, gwarp, nwarps, &p.ctl->wq[level % 3], 0,
              [&](bool valid, int k, int w, int col) {
    uint32_t vw[G];
    FwdHit<G, EXT> h;
#pragma unroll
    for (int g = 0; g < G; g++) {
      vw[g] = 0xffffffffu;
      h.bm[g] = 0u;
    }
    bool full = true;
    // the owner's visited row and the edge's neighbour are independent loads
    const int pj = valid ? p.ci[col] : -1;
    if (valid) full = load_vis<G>(p, w, vw);
    h.pj = -1;
    h.hit = false;
    if (valid && !full) {
      h.pj = pj;
      load_row<G>(Fp, h.pj, h.bm);
#pragma unroll
      for (int g = 0; g < G; g++) {
        h.bm[g] &= ~vw[g];
        h.hit |= h.bm[g] != 0u;
      }
    }
    fwd_hit_load<G, EXT>(p, h);
    const unsigned vm = __ballot_sync(BC_FULL, valid);
    const unsigned sps = __ballot_sync(BC_FULL, h.sp);
    const unsigned dns = __ballot_sync(BC_FULL, h.hit && !h.sp);
    if (!(sps | dns)) return;
    const int k_lo = __shfl_sync(BC_FULL, k, __ffs(sps | dns) - 1);
    const int k_hi = __shfl_sync(BC_FULL, k, 31 - __clz(sps | dns));
    for (int kk = k_lo; kk <= k_hi; kk++) {
      const unsigned lanes_k = __ballot_sync(BC_FULL, valid && k == kk) & vm;
      const unsigned hs = sps & lanes_k, hd = dns & lanes_k;
      if (!(hs | hd)) continue;
      const int jl = __ffs(hs | hd) - 1;
      const int wk = __shfl_sync(BC_FULL, w, jl);
      if (wk != cur) {
        sparse_fold<G, EXT>(a);
        if (G >= 8 && cur >= 0) load_row<G>(p.vis, cur, visc);  // reloaded (registers bind at T = 256)
        if (cur >= 0 && pull_commit<G, EXT>(p, cur, level, a, visc, leaf, nsacc))
          abuf_push(p, ab, cur, ap, a_base);
        cur = wk;
#pragma unroll
        for (int g = 0; g < G; g++) visc[g] = G >= 8 ? 0u : __shfl_sync(BC_FULL, vw[g], jl);
        pull_init(a);
      }
      fwd_hits_add<G, EXT>(p, h, hs, hd, a);
    }
  });
  sparse_fold<G, EXT>(a);
  if (G >= 8 && cur >= 0) load_row<G>(p.vis, cur, visc);
  if (cur >= 0 && pull_commit<G, EXT>(p, cur, level, a, visc, leaf, nsacc))
    abuf_push(p, ab, cur, ap, a_base);
}

// Forward work item i of level l's split candidates (degree >= p.hub; list L with the
// exclusive prefix IP of their chunk counts, nl entries; one item per chunk of p.hub_chunk
// edges at fixed offsets from the vertex's first edge): one warp sums, per source lane,
// sigma over the chunk's parents.  A single-chunk vertex is committed at once; otherwise the
// chunk's sums, new-level masks and overflow bits go to the level's partial buffers and the
// warp finishing the vertex's last chunk adds them up in chunk order (a fixed order, so the
// extended-range sums repeat bit for bit) and commits.
template <int G, bool EXT>
__device__ void fwd_warp_item(const TK &p, int level, const int32_t *L, const int32_t *IP, int nl, int i,
                              unsigned long long *ap, int a_base, bool leaf, unsigned long long (&nsacc)[G]) {
  const int lane = lane_id();
  const int k = find_owner(IP, 0, nl, i);
  const int c = i - IP[k];
  const int w = L[k];
  uint32_t visw[G];
  if (load_vis<G>(p, w, visw)) return;  // reached by every source: none of w's items commits
  const int r0 = p.rp[w], r1 = p.rp[w + 1];
  const int nch = (r1 - r0 + p.hub_chunk - 1) / p.hub_chunk;
  const int e0 = r0 + c * p.hub_chunk, e1 = min(r1, e0 + p.hub_chunk);
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  PullAcc<G, EXT> a;
  pull_init(a);
  for (int base = e0; base < e1; base += 32) {
    const int jdx = base + lane;
    FwdHit<G, EXT> h;
    h.pj = jdx < e1 ? p.ci[jdx] : -1;
    h.hit = false;
    if (h.pj >= 0) {
      load_row<G>(Fp, h.pj, h.bm);
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) h.bm[g] = 0u;
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
      h.bm[g] &= ~visw[g];
      h.hit |= h.bm[g] != 0u;
    }
    fwd_hit_load<G, EXT>(p, h);
    fwd_hits_add<G, EXT>(p, h, __ballot_sync(BC_FULL, h.sp), __ballot_sync(BC_FULL, h.hit && !h.sp), a);
  }
  sparse_fold<G, EXT>(a);
  if (nch > 1) {
    unsigned long long *ps = p.FPs + (size_t)i * (32 * G);
    uint32_t *pm = p.FPm + (size_t)i * (2 * G);
#pragma unroll
    for (int g = 0; g < G; g++) {
      __stcg(&ps[32 * g + lane], a.s[g]);
      const unsigned ob = __ballot_sync(BC_FULL, ((a.o >> g) & 1u) || (!EXT && a.cy != 0u));
      if (lane == 0) {
        __stcg(&pm[g], a.newm[g]);
        __stcg(&pm[G + g], ob);
      }
      if (EXT) {
        __stcg(&p.FPx[(size_t)i * (32 * G) + 32 * g + lane], a.x[g].m);
        __stcg(&p.FPe[(size_t)i * (32 * G) + 32 * g + lane], a.x[g].e);
      }
    }
    __threadfence();
    int last = 0;
    if (lane == 0) last = atomicAdd(&p.Fdone[k], 1) == nch - 1;
    if (!__shfl_sync(BC_FULL, last, 0)) return;
    __threadfence();
    pull_init(a);
    for (int cc = 0; cc < nch; cc++) {
      const size_t it = (size_t)(i - c + cc);
#pragma unroll
      for (int g = 0; g < G; g++) {
        const unsigned long long v = __ldcg(&p.FPs[it * (32 * G) + 32 * g + lane]);
        const unsigned long long old = a.s[g];
        a.s[g] = old + v;
        const uint32_t ob = __ldcg(&p.FPm[it * (2 * G) + G + g]);
        if (a.s[g] < old || ((ob >> lane) & 1u)) a.o |= 1u << g;
        a.newm[g] |= __ldcg(&p.FPm[it * (2 * G) + g]);
        if (EXT) {
          XS y;
          y.m = __ldcg(&p.FPx[it * (32 * G) + 32 * g + lane]);
          y.e = __ldcg(&p.FPe[it * (32 * G) + 32 * g + lane]);
          xs_add(a.x[g], y);
        }
      }
    }
    if (lane == 0) p.Fdone[k] = 0;  // clean for the next level
  }
  const bool any = pull_commit<G, EXT>(p, w, level, a, visw, leaf, nsacc);
  append_A(p, ap, a_base, any && lane == 0, w);
}

// ------------------------------------------------------------------ lane-per-entry mode
// On high-diameter graphs the sources of a tile rarely share a level, so most entries
// carry one source and a few edges; walked warp-wide, each such entry costs a warp-serial
// sequence of its own.  Levels whose entries average at most two sources and 16 edges are
// instead run one entry per lane: the lane walks the entry's adjacency alone (four edges
// per round, their loads in flight together), keeping the sums of two sources at a time in
// registers (one pass per pair).  Entries with more than kLaneSrc sources or kLaneDeg
// edges fall back to the warp-wide path, one at a time; hubs stay with whole CTAs.  Each
// (entry, source) sum runs in edge order.
constexpr int kLaneDeg = 64;
constexpr int kLaneSrc = 8;  // sources per lane-mode entry (in passes of two)

__device__ __forceinline__ bool lane_level(unsigned long long bits, long long entries, long long edges) {
  return entries > 0 && bits <= 2ull * (unsigned long long)entries && edges <= 16ll * entries;
}

template <bool EXT>
struct LaneSlot {
  int t;                  // source lane of the tile, -1 while free
  bool o;                 // sigma passed 2^64 (carry or an overflowed parent)
  unsigned long long s;   // sigma mod 2^64
  XS x;                   // extended sigma (EXT)
};

template <bool EXT>
__device__ __forceinline__ void slot_init(LaneSlot<EXT> &z) {
  z.t = -1;
  z.o = false;
  z.s = 0ull;
  z.x.m = 0.0;
  z.x.e = 0;
}

template <bool EXT>
__device__ __forceinline__ void slot_add(LaneSlot<EXT> &z, int t, unsigned long long v, bool po, const XS &x) {
  z.t = t;
  const unsigned long long old = z.s;
  z.s = old + v;
  z.o = z.o || z.s < old || po;
  if (EXT) xs_add(z.x, x);
}

// Sum sigma over the parents of candidate w (frontier neighbours, per unvisited source)
// for the first two sources met; the other sources that reach w are collected in more.
template <int G, bool EXT>
__device__ __forceinline__ void lane_pull(const TK &p, const uint32_t *Fp, int w, const uint32_t (&vw)[G],
                                          LaneSlot<EXT> &a, LaneSlot<EXT> &b, uint32_t (&more)[G]) {
  const int e1 = p.rp[w + 1];
  for (int e = p.rp[w]; e < e1; e += 4) {
    int pj[4];
#pragma unroll
    for (int u = 0; u < 4; u++) pj[u] = e + u < e1 ? p.ci[e + u] : -1;
    uint32_t fm[4][G];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      if (pj[u] >= 0) {
        load_row<G>(Fp, pj[u], fm[u]);
#pragma unroll
        for (int g = 0; g < G; g++) fm[u][g] &= ~vw[g];
      } else {
#pragma unroll
        for (int g = 0; g < G; g++) fm[u][g] = 0u;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int g = 0; g < G; g++) {
        uint32_t m = fm[u][g];
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1;
          const int t = 32 * g + bit;
          const size_t idx = sidx<G>(pj[u], t);
          const unsigned long long v = p.sig[idx];
          const bool po = EXT && ((p.ovf[(size_t)pj[u] * G + g] >> bit) & 1u);
          XS x;
          x.m = 0.0;
          x.e = 0;
          if (EXT) {
            if (po) {
              x.m = p.xm[idx];
              x.e = p.xe[idx];
            } else {
              x = xs_u64(v);
            }
          }
          if (a.t < 0 || a.t == t) {
            slot_add<EXT>(a, t, v, po, x);
          } else if (b.t < 0 || b.t == t) {
            slot_add<EXT>(b, t, v, po, x);
          } else {
            more[g] |= 1u << bit;
          }
        }
      }
    }
  }
}

// Add sigma of the parents of w for the known sources of slots a and b (t >= 0 or -1).
template <int G, bool EXT>
__device__ __forceinline__ void lane_pull_pair(const TK &p, const uint32_t *Fp, int w, LaneSlot<EXT> &a,
                                               LaneSlot<EXT> &b) {
  const int e1 = p.rp[w + 1];
  const int ga = a.t >> 5, gb = b.t >= 0 ? b.t >> 5 : ga;
  for (int e = p.rp[w]; e < e1; e += 4) {
    int pj[4];
#pragma unroll
    for (int u = 0; u < 4; u++) pj[u] = e + u < e1 ? p.ci[e + u] : -1;
    uint32_t fa[4], fb[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      fa[u] = pj[u] >= 0 ? Fp[(size_t)pj[u] * G + ga] : 0u;
      fb[u] = (pj[u] >= 0 && b.t >= 0) ? (gb == ga ? fa[u] : Fp[(size_t)pj[u] * G + gb]) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int z = 0; z < 2; z++) {
        LaneSlot<EXT> &sl = z ? b : a;
        const uint32_t f = z ? fb[u] : fa[u];
        if (sl.t < 0 || !((f >> (sl.t & 31)) & 1u)) continue;
        const size_t idx = sidx<G>(pj[u], sl.t);
        const unsigned long long v = p.sig[idx];
        const bool po = EXT && ((p.ovf[(size_t)pj[u] * G + (sl.t >> 5)] >> (sl.t & 31)) & 1u);
        XS x;
        x.m = 0.0;
        x.e = 0;
        if (EXT) {
          if (po) {
            x.m = p.xm[idx];
            x.e = p.xe[idx];
          } else {
            x = xs_u64(v);
          }
        }
        slot_add<EXT>(sl, sl.t, v, po, x);
      }
    }
  }
}

// Store one slot of a lane-mode candidate: sigma (and its extended form) and the slot's
// bit in the new-level and overflow masks.
template <int G, bool EXT>
__device__ __forceinline__ void lane_store_slot(const TK &p, int w, const LaneSlot<EXT> &z, uint32_t (&nm)[G],
                                                uint32_t (&om)[G], bool leaf) {
  if (z.t < 0) return;
  const size_t idx = sidx<G>(w, z.t);
  p.sig[idx] = z.s;
  if (EXT && z.o) {
    const XS x = xs_norm(z.x);
    p.xm[idx] = x.m;
    p.xe[idx] = x.e;
  }
#pragma unroll
  for (int g = 0; g < G; g++) {
    if ((z.t >> 5) != g) continue;
    nm[g] |= 1u << (z.t & 31);
    if (z.o) om[g] |= 1u << (z.t & 31);
  }
  if (leaf) atomicAdd(&p.ctl->ns[z.t], 1ull + (unsigned long long)p.omega[w]);
}

// Warp-wide pull of one candidate (sigma rows gathered by the source lanes).  Returns
// whether any source reached w.
template <int G, bool EXT>
__device__ bool warp_pull_one(const TK &p, int level, int w, const uint32_t (&visc)[G], bool leaf,
                              unsigned long long (&nsacc)[G]) {
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  PullAcc<G, EXT> a;
  pull_init(a);
  const int e1 = p.rp[w + 1];
  for (int base = p.rp[w]; base < e1; base += 32) {
    const int e = base + lane_id();
    const int pj = e < e1 ? p.ci[e] : -1;
    uint32_t fm[G];
    bool hit = false;
    if (pj >= 0) {
      load_row<G>(Fp, pj, fm);
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) fm[g] = 0u;
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
      fm[g] &= ~visc[g];
      hit |= fm[g] != 0u;
    }
    unsigned hits = __ballot_sync(BC_FULL, hit);
    while (hits) {
      const int jj = __ffs(hits) - 1;
      hits &= hits - 1;
      uint32_t m[G];
#pragma unroll
      for (int g = 0; g < G; g++) m[g] = __shfl_sync(BC_FULL, fm[g], jj);
      pull_hit<G, EXT>(p, __shfl_sync(BC_FULL, pj, jj), m, a);
    }
  }
  return pull_commit<G, EXT>(p, w, level, a, visc, leaf, nsacc);
}

// Lane-mode pull over the candidates C[0, nc): warps take 32 consecutive candidates.
template <int G, bool EXT>
__device__ void pull_lanes(const TK &p, int level, int nc, int gwarp, int nwarps, unsigned long long *ap,
                           int a_base, bool leaf, unsigned long long (&nsacc)[G]) {
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  uint32_t *Fn = Fbuf<G>(p, level);
  const int lane = lane_id();
  for (int base = gwarp * 32; base < nc; base += nwarps * 32) {
    const int i = base + lane;
    const bool in = i < nc;
    const int w = in ? p.C[i] : 0;
    uint32_t vw[G];
    bool full = true;
    if (in) full = load_vis<G>(p, w, vw);
    const bool small = in && !full && vdeg(p, w) <= kLaneDeg;
    LaneSlot<EXT> a, b;
    slot_init<EXT>(a);
    slot_init<EXT>(b);
    uint32_t more[G];
    int nmore = 0;
#pragma unroll
    for (int g = 0; g < G; g++) more[g] = 0u;
    if (small) {
      lane_pull<G, EXT>(p, Fp, w, vw, a, b, more);
#pragma unroll
      for (int g = 0; g < G; g++) nmore += __popc(more[g]);
    }
    const bool ok = small && nmore <= kLaneSrc - 2;
    const bool fb = in && !full && !ok;
    const bool got = ok && a.t >= 0;
    uint32_t nm[G], om[G];
#pragma unroll
    for (int g = 0; g < G; g++) nm[g] = om[g] = 0u;
    if (got) {
      lane_store_slot<G, EXT>(p, w, a, nm, om, leaf);
      lane_store_slot<G, EXT>(p, w, b, nm, om, leaf);
      for (;;) {  // the other sources, two per pass
        int t0, t1;
        if (two_bits<G>(more, t0, t1) == 0) break;
#pragma unroll
        for (int g = 0; g < G; g++) {
          if ((t0 >> 5) == g) more[g] &= ~(1u << (t0 & 31));
          if (t1 >= 0 && (t1 >> 5) == g) more[g] &= ~(1u << (t1 & 31));
        }
        slot_init<EXT>(a);
        slot_init<EXT>(b);
        a.t = t0;
        b.t = t1;
        lane_pull_pair<G, EXT>(p, Fp, w, a, b);
        lane_store_slot<G, EXT>(p, w, a, nm, om, leaf);
        lane_store_slot<G, EXT>(p, w, b, nm, om, leaf);
      }
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (!nm[g]) continue;
        p.vis[(size_t)w * G + g] = vw[g] | nm[g];
        Fn[(size_t)w * G + g] = nm[g];
        if (om[g]) p.ovf[(size_t)w * G + g] |= om[g];
      }
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
      const uint32_t ob = __reduce_or_sync(BC_FULL, om[g]);
      if (lane == 0 && ob) {
        p.ctl->ovf_any = 1;
        atomicOr(&p.ctl->ovf_lanes[g], ob);
      }
    }
    append_A(p, ap, a_base, got, w);
    unsigned fbm = __ballot_sync(BC_FULL, fb);
    while (fbm) {
      const int j = __ffs(fbm) - 1;
      fbm &= fbm - 1;
      const int wf = __shfl_sync(BC_FULL, w, j);
      uint32_t visc[G];
#pragma unroll
      for (int g = 0; g < G; g++) visc[g] = __shfl_sync(BC_FULL, vw[g], j);
      const bool any = warp_pull_one<G, EXT>(p, level, wf, visc, leaf, nsacc);
      append_A(p, ap, a_base, any && lane == 0, wf);
    }
  }
}

// ------------------------------------------------------------------ forward phases
template <int G>
__device__ void phase_init_vis(const TK &p, int gtid, int nthr) {
  for (long long i = gtid; i < (long long)p.n * G; i += nthr) p.vis[i] = p.unused[i % G];
}

// The tile's sources become A_0 (distinct vertices with at least one edge; a repeated
// source sets several lanes of one vertex).  Single thread.
template <int G>
__device__ void init_sources(const TK &p) {
  unsigned cnt = 0, edges = 0;
  uint32_t *F0 = Fbuf<G>(p, 0);
  for (int t = 0; t < p.nsrc; t++) {
    const int s = p.src[t];
    const int g = t >> 5;
    const uint32_t bit = 1u << (t & 31);
    const int ds = vdeg(p, s);
    bool first = true;
    for (int h = 0; h < G; h++) first &= (p.vis[(size_t)s * G + h] & ~p.unused[h]) == 0u;
    p.vis[(size_t)s * G + g] |= bit;
    p.sig[sidx<G>(s, t)] = 1ull;
    if (ds > 0) {
      F0[(size_t)s * G + g] |= bit;
      if (first) {
        p.A[cnt] = s;
        p.ACD[cnt] = (int)edges;
        p.ARP[cnt] = p.rp[s];
        cnt++;
        edges += (unsigned)ds;
      }
    }
    if (p.leaf_term && p.omega) p.ctl->ns[t] = 1ull + (unsigned long long)p.omega[s];
  }
  p.ctl->apack[0] = pack_qe(cnt, edges);
  p.ctl->apack[1] = p.ctl->apack[2] = 0ull;
  p.ctl->cpack[0] = p.ctl->cpack[1] = p.ctl->cpack[2] = 0ull;
  p.ctl->chpk[0] = p.ctl->chpk[1] = p.ctl->chpk[2] = 0ull;
  p.Aoff[0] = 0;
  p.Lbits[0] = 0ull;
  p.HEoff[0] = 0;
  p.HEoff[1] = 0;
  p.Aoff[1] = (int)cnt;
}

// Masks of A_{l-1} into AM; clear F of A_{l-2}.
template <int G>
__device__ void phase_keep(const TK &p, int level, int a_pp, int a0, int a1, int gtid, int nthr) {
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  unsigned long long rv = 0, ra = 0;
  for (long long i = (long long)a0 * G + gtid; i < (long long)a1 * G; i += nthr) {
    const int w = p.A[i / G];
    const uint32_t m = Fp[(size_t)w * G + (i % G)];
    p.AM[i] = m;
    rv += __popc(m);
    ra += (unsigned long long)__popc(m) * (unsigned long long)vdeg(p, w);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    rv += __shfl_xor_sync(BC_FULL, rv, o);
    ra += __shfl_xor_sync(BC_FULL, ra, o);
  }
  if ((threadIdx.x & 31) == 0 && rv) {
    atomicAdd(&p.ctl->reached, rv);
    atomicAdd(&p.ctl->reached_arcs, ra);
    atomicAdd(&p.Lbits[level - 1], rv);
  }
  if (level >= 2) {
    uint32_t *Fc = Fbuf<G>(p, level - 2);
    for (long long i = (long long)a_pp * G + gtid; i < (long long)a0 * G; i += nthr)
      Fc[(size_t)p.A[i / G] * G + (i % G)] = 0u;
  }
}

// Top-down marking of the candidates of level l: edges of A_{l-1} (unsnapped equal
// slices; an edge's owner is found in the prefix ACD).  Each new candidate is appended to
// C with its degree prefix, or to Ch if it is a hub.
template <int G>
__device__ void phase_mark(const TK &p, int level, int a0, int a1, int E1, int gwarp, int nwarps) {
  const int lane = lane_id();
  if (E1 <= 0) return;
  const long long per = (((long long)E1 + nwarps - 1) / nwarps + 31) & ~31ll;
  const long long eb = (long long)gwarp * per;
  if (eb >= E1) return;
  const int ee = (int)min(eb + per, (long long)E1);
  const uint32_t *Fp = Fbuf<G>(p, level - 1);
  int base = find_owner(p.ACD, a0, a1, (int)eb);
  unsigned long long *cp = &p.ctl->cpack[level % 3];
  unsigned long long *chp = &p.ctl->chpk[level % 3];
  for (int e = (int)eb; e < ee; e += 32) {
    const int idx = base + lane;
    const bool in = idx < a1;
    const int cdj = in ? p.ACD[idx] : INT_MAX;
    const int vj = in ? p.A[idx] : 0;
    const int bias = in ? p.ARP[idx] - cdj : 0;
    const int cd_after = (base + 32 < a1) ? p.ACD[base + 32] : E1;
    const int my = e + lane;
    const int j = warp_owner(cdj, my);
    const int v = __shfl_sync(BC_FULL, vj, j);
    const int col = my + __shfl_sync(BC_FULL, bias, j);
    bool isc = false;
    int w = 0;
    if (my < ee) {
      w = p.ci[col];
      bool hit = false;
      uint32_t fv[G], vv[G];
      load_row<G>(Fp, v, fv);
      load_row<G>(p.vis, w, vv);
#pragma unroll
      for (int g = 0; g < G; g++) hit |= (fv[g] & ~vv[g]) != 0u;
      if (hit) {
        const uint32_t bit = 1u << (w & 31);
        isc = !(atomicOr(p.cand + (w >> 5), bit) & bit);
      }
    }
    const int rw = isc ? p.rp[w] : 0;
    const int dw = isc ? p.rp[w + 1] - rw : 0;
    const bool hub = isc && dw >= p.hub;
    const bool nrm = isc && !hub;
    const unsigned mn = __ballot_sync(BC_FULL, nrm), mh = __ballot_sync(BC_FULL, hub);
    if (mn) {
      int tot;
      const int pre = warp_excl_scan(nrm ? dw : 0, &tot);
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(cp, pack_qe(__popc(mn), (unsigned)tot));
      b = __shfl_sync(BC_FULL, b, 0);
      if (nrm) {
        const int pos = (int)(b >> 32) + __popc(mn & lanemask_lt());
        p.C[pos] = w;
        p.CPD[pos] = (int)(b & 0xffffffffull) + pre;
        p.CRP[pos] = rw;
      }
    }
    if (mh) {  // split candidates, with the exclusive prefix of their chunk counts
      const int nchk = hub ? (dw + p.hub_chunk - 1) / p.hub_chunk : 0;
      int tot;
      const int pre = warp_excl_scan(nchk, &tot);
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(chp, pack_qe(__popc(mh), (unsigned)tot));
      b = __shfl_sync(BC_FULL, b, 0);
      if (hub) {
        const int pos = (int)(b >> 32) + __popc(mh & lanemask_lt());
        p.Ch[pos] = w;
        p.ChP[pos] = (int)(b & 0xffffffffull) + pre;
      }
    }
    const int j31 = __shfl_sync(BC_FULL, j, 31);
    int nxt = __shfl_sync(BC_FULL, cdj, min(j31 + 1, 31));
    if (j31 == 31) nxt = cd_after;
    base += j31 + ((e + 32 >= nxt) ? 1 : 0);
  }
}

// Bottom-up level following another bottom-up level: the non-hub vertices that some source
// has not reached yet (of the per-graph list Lbu), appended to C with their degree prefix,
// so that the pull walks only them (late bottom-up levels: most vertices are reached by
// every source, and their edges would be walked for nothing).
template <int G>
__device__ void phase_compact(const TK &p, int level, int gwarp, int nwarps) {
  const int lane = lane_id();
  unsigned long long *cp = &p.ctl->cpack[level % 3];
  for (int b = gwarp * 32; b < p.nbu; b += nwarps * 32) {
    const int i = b + lane;
    bool keep = false;
    int w = 0, rw = 0, dw = 0;
    if (i < p.nbu) {
      w = p.Lbu[i];
      uint32_t vv[G];
      keep = !load_vis<G>(p, w, vv);
      if (keep) {
        rw = p.RPbu[i];
        dw = p.rp[w + 1] - rw;
      }
    }
    const unsigned mk = __ballot_sync(BC_FULL, keep);
    if (!mk) continue;
    int tot;
    const int pre = warp_excl_scan(keep ? dw : 0, &tot);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cp, pack_qe(__popc(mk), (unsigned)tot));
    base = __shfl_sync(BC_FULL, base, 0);
    if (keep) {
      const int pos = (int)(base >> 32) + __popc(mk & lanemask_lt());
      p.C[pos] = w;
      p.CPD[pos] = (int)(base & 0xffffffffull) + pre;
      p.CRP[pos] = rw;
    }
  }
}

// Pull of level l: hubs (Ch, or every hub in bottom-up mode) by whole CTAs, then the walk
// over C (top-down) or over every non-hub vertex (bottom-up).  Reached vertices go to A_l.
template <int G, bool EXT>
__device__ void phase_pull(const TK &p, int level, bool bu, bool compacted, int a_lo, int a_base, int gwarp,
                           int nwarps) {
  const int lane = lane_id();
  const bool leaf = p.leaf_term && p.omega;
  unsigned long long nsacc[G];
#pragma unroll
  for (int g = 0; g < G; g++) nsacc[g] = 0ull;
  unsigned long long *ap = &p.ctl->apack[level % 3];
  const unsigned long long chk = vload64(&p.ctl->chpk[level % 3]);
  const int nh = bu ? p.nhubs : (int)(chk >> 32);
  const int nitems = bu ? p.nhub_items : (int)(chk & 0xffffffffull);
  const int32_t *hl = bu ? p.hubs : p.Ch;
  const int32_t *hp = bu ? p.HPbu : p.ChP;
  AppendBuf ab;
  ab.v = 0;
  ab.n = 0;
  if (bu) {  // every non-hub vertex, or those some source has not reached (phase_compact)
    const int32_t *L = p.Lbu, *PD = p.PDbu, *RP = p.RPbu;
    int nl = p.nbu, el = p.Ebu;
    if (compacted) {
      const unsigned long long cpk = vload64(&p.ctl->cpack[level % 3]);
      L = p.C;
      PD = p.CPD;
      RP = p.CRP;
      nl = (int)(cpk >> 32);
      el = (int)(cpk & 0xffffffffull);
    }
    pull_walk<G, EXT>(p, level, L, PD, RP, nl, el, gwarp, nwarps, ab, ap, a_base, leaf, nsacc);
  } else {
    const unsigned long long cpk = vload64(&p.ctl->cpack[level % 3]);
    const int nc = (int)(cpk >> 32);
    const int ec = (int)(cpk & 0xffffffffull);
    // lane mode: A_{l-1} (entries a_lo .. a_base) carries <= 2 sources per entry on average
    // and the candidates have few edges
    if (lane_level(vload64(&p.Lbits[level - 1]), a_base - a_lo, (long long)ec) && ec <= 16ll * nc)
      pull_lanes<G, EXT>(p, level, nc, gwarp, nwarps, ap, a_base, leaf, nsacc);
    else
      pull_walk<G, EXT>(p, level, p.C, p.CPD, p.CRP, nc, ec, gwarp, nwarps, ab, ap, a_base, leaf, nsacc);
    // clear the candidate bits of this level (C and Ch)
    for (int i = gwarp * 32 + lane; i < nc; i += nwarps * 32) {
      const int w = p.C[i];
      atomicAnd(p.cand + (w >> 5), ~(1u << (w & 31)));
    }
    for (int i = gwarp * 32 + lane; i < nh; i += nwarps * 32) {
      const int w = p.Ch[i];
      atomicAnd(p.cand + (w >> 5), ~(1u << (w & 31)));
    }
  }
  abuf_flush(p, ab, ap, a_base);
  // work items of the split candidates, one per warp from a counter, taken by each warp as
  // soon as its walk is done (balances the few, very large adjacency lists)
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&p.ctl->hubq[level % 3], 1);
    i = __shfl_sync(BC_FULL, i, 0);
    if (i >= nitems) break;
    fwd_warp_item<G, EXT>(p, level, hl, hp, nh, i, ap, a_base, leaf, nsacc);
  }
  if (leaf) {
#pragma unroll
    for (int g = 0; g < G; g++)
      if (nsacc[g]) atomicAdd(&p.ctl->ns[32 * g + lane], nsacc[g]);
  }
}

// ------------------------------------------------------------------ backward phases
// r of the deepest level's (vertex, source) pairs: delta = 0 there.
template <int G, bool EXT>
__device__ void phase_bwd_deep(const TK &p, int a0, int a1, int gtid, int nthr) {
  for (long long i = (long long)a0 * 32 * G + gtid; i < (long long)a1 * 32 * G; i += nthr) {
    const int k = (int)(i / (32 * G)), t = (int)(i % (32 * G)), g = t >> 5, ln = t & 31;
    const uint32_t m = p.AM[(size_t)k * G + g];
    if (!((m >> ln) & 1u)) continue;
    const int w = p.A[k];
    const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
    const size_t idx = sidx<G>(w, t);
    float2 sg;
    if (EXT) {
      const bool o = (p.ovf[(size_t)w * G + g] >> ln) & 1u;
      const XS x = sig_xs(p, idx, o);
      sg = ff_mant(x.m);
      if (!o) p.xe[idx] = x.e;
    } else {
      sg = ff_u64(p.sig[idx]);
    }
    p.r[idx] = ff_mul(om1, ff_rcp(sg));
  }
}

// Tiles of 128 sources or more (64-bit mode) load the owner's sigma and BC at its commit
// instead of holding them in registers through the walk (registers bind there).
template <int G, bool EXT>
struct LateOwner {
  static constexpr bool value = !EXT && G >= 4;
};

template <int G, bool EXT>
struct BwdOwner {
  uint32_t mw[G];
  float2 sg[EXT ? G : 1];                  // extended range: sigma's mantissa, float-float
  unsigned long long sr[(EXT || LateOwner<G, EXT>::value) ? 1 : G];  // 64-bit mode: sigma
  int ew[EXT ? G : 1];
  float2 acc[G];   // sum of the successors' r: hits gathered as rows
  float2 accs[G];  // the same for sparse hits (at most two sources), folded in by bwd_fold
  double bcw;      // BC[w], loaded when the owner starts (only this entry updates it this level)
};

// acc = accs + acc (a fixed order), accs = 0: the owner's full sum of the successors' r
template <int G, bool EXT>
__device__ __forceinline__ void bwd_fold(BwdOwner<G, EXT> &o) {
#pragma unroll
  for (int g = 0; g < G; g++) {
    float2 t = o.accs[g];
    ff_add(t, o.acc[g]);
    o.acc[g] = t;
    o.accs[g] = make_float2(0.0f, 0.0f);
  }
}

template <int G, bool EXT>
__device__ __forceinline__ void bwd_start(const TK &p, int w, const uint32_t (&mw)[G], BwdOwner<G, EXT> &o) {
  const int lane = lane_id();
  if constexpr (!LateOwner<G, EXT>::value) o.bcw = p.nreq == 0 ? p.bc[w] : 0.0;
  bool mine = false;
#pragma unroll
  for (int g = 0; g < G; g++) {
    o.mw[g] = mw[g];
    o.acc[g] = make_float2(0.0f, 0.0f);
    o.accs[g] = make_float2(0.0f, 0.0f);
    mine |= (mw[g] >> lane) & 1u;
  }
  if constexpr (LateOwner<G, EXT>::value) {
    return;
  } else if constexpr (!EXT) {  // the lane's sigma values in vector loads, used only at commit
    if (mine) {
      load_lane<G>(p.sig + sidx<G>(w, 0, lane), o.sr);
    } else {
#pragma unroll
      for (int g = 0; g < (EXT ? 1 : G); g++) o.sr[g] = 1ull;
    }
    return;
  }
#pragma unroll
  for (int g = 0; g < (EXT ? G : 1); g++) {
    o.sg[g] = make_float2(1.0f, 0.0f);
    o.ew[g] = 0;
    if ((o.mw[g] >> lane) & 1u) {
      const size_t idx = sidx<G>(w, g, lane);
      const bool ov = (p.ovf[(size_t)w * G + g] >> lane) & 1u;
      const XS x = sig_xs(p, idx, ov);
      o.sg[g] = ff_mant(x.m);
      o.ew[g] = x.e;
    }
  }
}

// The same for entry k of the active list (vertex and masks loaded here).
template <int G, bool EXT>
__device__ __forceinline__ void bwd_start_k(const TK &p, int k, BwdOwner<G, EXT> &o) {
  uint32_t mw[G];
  load_row<G>(p.AM, k, mw);
  bwd_start<G, EXT>(p, p.A[k], mw, o);
}

template <int G, bool EXT>
__device__ __forceinline__ void bwd_hit(const TK &p, int v, const uint32_t (&m)[G], BwdOwner<G, EXT> &o) {
  const int lane = lane_id();
#pragma unroll
  for (int g = 0; g < G; g++) {
    if ((m[g] >> lane) & 1u) {
      const size_t idx = sidx<G>(v, g, lane);
      float2 x = p.r[idx];
      if (EXT) x = ff_scale(x, o.ew[g] - p.xe[idx]);
      ff_add(o.acc[g], x);
    }
  }
}

template <int G, bool EXT>
__device__ __forceinline__ void bwd_commit(const TK &p, int w, BwdOwner<G, EXT> &o) {
  const int lane = lane_id();
  bwd_fold<G, EXT>(o);
  const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
  float2 contrib = make_float2(0.0f, 0.0f);
  float2 dl[G];
  unsigned long long sl[LateOwner<G, EXT>::value ? G : 1];
  if constexpr (LateOwner<G, EXT>::value) {
    o.bcw = p.nreq == 0 ? p.bc[w] : 0.0;
    bool mine = false;
#pragma unroll
    for (int g = 0; g < G; g++) mine |= (o.mw[g] >> lane) & 1u;
    if (mine) {
      load_lane<G>(p.sig + sidx<G>(w, 0, lane), sl);
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) sl[g] = 1ull;
    }
  }
#pragma unroll
  for (int g = 0; g < G; g++) {
    dl[g] = make_float2(0.0f, 0.0f);
    if ((o.mw[g] >> lane) & 1u) {
      const size_t idx = sidx<G>(w, g, lane);
      float2 sg;
      if constexpr (EXT)
        sg = o.sg[g];
      else if constexpr (LateOwner<G, EXT>::value)
        sg = ff_u64(sl[g]);
      else
        sg = ff_u64(o.sr[g]);
      // delta = sigma * sum r(succ);  r = (1 + delta + omega) / sigma = (1 + omega) / sigma + sum
      dl[g] = ff_mul(p.wsrc[32 * g + lane], ff_mul(sg, o.acc[g]));
      ff_add(contrib, dl[g]);
      float2 r = ff_mul(om1, ff_rcp(sg));
      ff_add(r, o.acc[g]);
      p.r[idx] = r;
      if (EXT) p.xe[idx] = o.ew[g];
    }
  }
  if (p.nreq == 0) {
    unsigned act = 0u;
#pragma unroll
    for (int g = 0; g < G; g++) act |= o.mw[g];
    if (__popc(act) == 1) {  // one lane holds the whole sum
      if (lane == __ffs(act) - 1 && !ff_zero(contrib)) p.bc[w] = o.bcw + ff_to(contrib);
      return;
    }
    if (!__ballot_sync(BC_FULL, !ff_zero(contrib))) return;  // no successor: delta = 0
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) ff_add(contrib, ff_shfl_xor(contrib, m));
    if (lane == 0 && !ff_zero(contrib)) p.bc[w] = o.bcw + ff_to(contrib);
    return;
  }
  // lanes belong to different requests (serving): one fixed-order sum per request
  for (int q = 0; q < p.nreq; q++) {
    float2 c = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int g = 0; g < G; g++)
      if (((o.mw[g] >> lane) & 1u) && p.lane_req[32 * g + lane] == q) ff_add(c, dl[g]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) ff_add(c, ff_shfl_xor(c, m));
    if (lane == 0 && !ff_zero(c)) p.req_bc[q][w] += ff_to(c);
  }
}

// One backward edge per lane: successor v and the owner's sources bm whose level-(d+1)
// mask it shares; hits of at most kSparse sources carry their own r values.
template <int G, bool EXT>
struct BwdHit {
  int v;
  uint32_t bm[G];
  bool hit, sp;
  int t0, t1;
  float2 r0, r1;
  int e0, e1;
};

template <int G, bool EXT>
__device__ __forceinline__ void bwd_hit_load(const TK &p, BwdHit<G, EXT> &h) {
  h.t0 = h.t1 = -1;
  h.sp = h.hit && two_bits<G>(h.bm, h.t0, h.t1) <= kSparse;
  h.r0 = h.r1 = make_float2(0.0f, 0.0f);
  h.e0 = h.e1 = 0;
  if (!h.sp) return;
  const size_t i0 = sidx<G>(h.v, h.t0);
  h.r0 = p.r[i0];
  if (EXT) h.e0 = p.xe[i0];
  if (h.t1 >= 0) {
    const size_t i1 = sidx<G>(h.v, h.t1);
    h.r1 = p.r[i1];
    if (EXT) h.e1 = p.xe[i1];
  }
}

// Add the hits of lanes hs (sparse) and hd (the others), all of one owner: sparse terms by
// shuffles into o.accs, the others by r-row gathers into o.acc (HB<G> rows in flight
// together).  Whether a hit is sparse depends on its mask alone, and each of the two sums
// takes its terms in lane (edge) order, step after step, so both are the same fold of the
// owner's edges wherever the walk's 32-edge steps fall: the sums repeat bit for bit.
template <int G, bool EXT>
__device__ __forceinline__ void bwd_hits_add(const TK &p, const BwdHit<G, EXT> &h, unsigned hs, unsigned hd,
                                             BwdOwner<G, EXT> &o) {
  const int lane = lane_id();
  while (hs) {
    const int jj = __ffs(hs) - 1;
    hs &= hs - 1;
#pragma unroll
    for (int z = 0; z < 2; z++) {
      const int t = __shfl_sync(BC_FULL, z ? h.t1 : h.t0, jj);
      const float2 x = ff_shfl(z ? h.r1 : h.r0, jj);
      const int xe = EXT ? __shfl_sync(BC_FULL, z ? h.e1 : h.e0, jj) : 0;
#pragma unroll
      for (int g = 0; g < G; g++)
        if (t >= 0 && (t >> 5) == g && lane == (t & 31)) ff_add(o.accs[g], EXT ? ff_scale(x, o.ew[g] - xe) : x);
    }
  }
  if (EXT) {
    while (hd) {
      const int jj = __ffs(hd) - 1;
      hd &= hd - 1;
      uint32_t m[G];
#pragma unroll
      for (int g = 0; g < G; g++) m[g] = __shfl_sync(BC_FULL, h.bm[g], jj);
      bwd_hit<G, EXT>(p, __shfl_sync(BC_FULL, h.v, jj), m, o);
    }
    return;
  }
  // up to HB<G>::value successors at a time: their r-row loads are in flight together
  if constexpr (G % 2 == 0) {  // the lane's sources in pairs, summed by packed additions
    if (!hd) return;
    FF2 acc2[G / 2];
#pragma unroll
    for (int j = 0; j < G / 2; j++) acc2[j] = ff2_pack(o.acc[2 * j], o.acc[2 * j + 1]);
    while (hd) {
      FF2 xq[HB<G>::value][G / 2];
      uint32_t mq[HB<G>::value][G];
#pragma unroll
      for (int q = 0; q < HB<G>::value; q++) {
        const int jj = hd ? __ffs(hd) - 1 : -1;
        if (hd) hd &= hd - 1;
        const int vq = __shfl_sync(BC_FULL, h.v, jj < 0 ? 0 : jj);
        bool mine = false;
#pragma unroll
        for (int g = 0; g < G; g++) {
          const uint32_t m = __shfl_sync(BC_FULL, h.bm[g], jj < 0 ? 0 : jj);
          mq[q][g] = jj < 0 ? 0u : m;
          mine |= (mq[q][g] >> lane) & 1u;
        }
        const float4 *row = (const float4 *)(p.r + sidx<G>(vq, 0, lane));
#pragma unroll
        for (int j = 0; j < G / 2; j++) {
          float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if (mine) x = row[j];  // (hi, lo) of source 2j, then of 2j + 1
          if (!((mq[q][2 * j] >> lane) & 1u)) x.x = x.y = 0.0f;
          if (!((mq[q][2 * j + 1] >> lane) & 1u)) x.z = x.w = 0.0f;
          xq[q][j].hi = f2_pack(x.x, x.z);
          xq[q][j].lo = f2_pack(x.y, x.w);
        }
      }
#pragma unroll
      for (int q = 0; q < HB<G>::value; q++)
#pragma unroll
        for (int j = 0; j < G / 2; j++)
          if (mq[q][2 * j] | mq[q][2 * j + 1]) ff2_add(acc2[j], xq[q][j]);
    }
#pragma unroll
    for (int j = 0; j < G / 2; j++) ff2_unpack(acc2[j], o.acc[2 * j], o.acc[2 * j + 1]);
    return;
  }
  while (hd) {
    float2 xq[HB<G>::value][G];
    uint32_t mq[HB<G>::value][G];
#pragma unroll
    for (int q = 0; q < HB<G>::value; q++) {
      const int jj = hd ? __ffs(hd) - 1 : -1;
      if (hd) hd &= hd - 1;
      const int vq = __shfl_sync(BC_FULL, h.v, jj < 0 ? 0 : jj);
      bool mine = false;
#pragma unroll
      for (int g = 0; g < G; g++) {
        const uint32_t m = __shfl_sync(BC_FULL, h.bm[g], jj < 0 ? 0 : jj);
        mq[q][g] = jj < 0 ? 0u : m;
        mine |= (mq[q][g] >> lane) & 1u;
      }
      if (mine) {  // the lane's G values of the row in vector loads
        load_lane<G>(p.r + sidx<G>(vq, 0, lane), xq[q]);
#pragma unroll
        for (int g = 0; g < G; g++)
          if (!((mq[q][g] >> lane) & 1u)) xq[q][g] = make_float2(0.0f, 0.0f);
      } else {
#pragma unroll
        for (int g = 0; g < G; g++) xq[q][g] = make_float2(0.0f, 0.0f);
      }
    }
#pragma unroll
    for (int q = 0; q < HB<G>::value; q++)
#pragma unroll
      for (int g = 0; g < G; g++)
        if (mq[q][g]) ff_add(o.acc[g], xq[q][g]);
  }
}

// Backward walk over A_d (hubs skipped): every entry is committed once, in entry order,
// with the r values of its successors summed: first the sparse hits (loaded by their edge
// lanes), then the other hits (r rows gathered by the source lanes), each in edge order.
template <int G, bool EXT>
__device__ void bwd_walk(const TK &p, int a0, int a1, int E, const uint32_t *Dn, int gwarp,
                         int nwarps, unsigned long long *ctr) {
  int cur = -1, cur_w = -1;
  BwdOwner<G, EXT> o;
  walk<true>(p, p.A, p.ACD, p.ARP, a0, a1, E, gwarp, nwarps, ctr, p.hub_chunk,
             [&](bool valid, int k, int w, int col) {
    BwdHit<G, EXT> h;
    h.hit = false;
    h.v = -1;
    uint32_t am[G];  // the owner's level-d mask (each edge lane loads its owner's)
#pragma unroll
    for (int g = 0; g < G; g++) {
      h.bm[g] = 0u;
      am[g] = 0u;
    }
    if (valid) {
      h.v = p.ci[col];
      load_row<G>(Dn, h.v, h.bm);
      load_row<G>(p.AM, k, am);
#pragma unroll
      for (int g = 0; g < G; g++) {
        h.bm[g] &= am[g];
        h.hit |= h.bm[g] != 0u;
      }
    }
    bwd_hit_load<G, EXT>(p, h);
    if (h.hit && !h.sp) prefetch_row<G>(p.r + sidx<G>(h.v, 0, 0), h.bm);
    const unsigned vm = __ballot_sync(BC_FULL, valid);
    const unsigned sps = __ballot_sync(BC_FULL, h.sp);
    const unsigned dns = __ballot_sync(BC_FULL, h.hit && !h.sp);
    if (!vm) return;
    const int k_lo = __shfl_sync(BC_FULL, k, __ffs(vm) - 1);
    const int k_hi = __shfl_sync(BC_FULL, k, 31 - __clz(vm));
    for (int kk = k_lo; kk <= k_hi; kk++) {
      const unsigned lanes_k = __ballot_sync(BC_FULL, valid && k == kk);
      if (!lanes_k) continue;  // a hub entry inside the step
      if (kk != cur) {
        if (cur >= 0) bwd_commit<G, EXT>(p, cur_w, o);
        const int jl = __ffs(lanes_k) - 1;  // a lane of this owner: its vertex and masks
        uint32_t mw[G];
#pragma unroll
        for (int g = 0; g < G; g++) mw[g] = __shfl_sync(BC_FULL, am[g], jl);
        cur = kk;
        cur_w = __shfl_sync(BC_FULL, w, jl);
        bwd_start<G, EXT>(p, cur_w, mw, o);
      }
      bwd_hits_add<G, EXT>(p, h, sps & lanes_k, dns & lanes_k, o);
    }
  });
  if (cur >= 0) bwd_commit<G, EXT>(p, cur_w, o);
}

// Backward work item i of level d's split entries (degree >= hub_chunk; one item per chunk
// of hub_chunk edges, cut at fixed offsets from the entry's first edge): one warp sums the
// chunk's successor terms in edge order.  A single-chunk entry is committed at once; else
// each chunk's sum goes to the level's partial buffer and the warp finishing an entry's
// last chunk adds the partials in chunk order (fixed, whatever the finishing order) and
// commits.
template <int G, bool EXT>
__device__ void bwd_warp_item(const TK &p, int i, int h0, const uint32_t *Dn) {
  const int lane = lane_id();
  const int k = p.HE[i], c = p.HEk[i];
  const int w = p.A[k];
  const int nch = (vdeg(p, w) + p.hub_chunk - 1) / p.hub_chunk;
  BwdOwner<G, EXT> o;
  bwd_start_k<G, EXT>(p, k, o);
  const int e0 = p.rp[w] + c * p.hub_chunk, e1 = min(p.rp[w + 1], e0 + p.hub_chunk);
  // a pipeline over the 32-edge steps: neighbour ids two steps ahead, their masks one step
  // ahead (in flight while a step's hits are summed), and the dense rows of the next step
  // requested from L2 as soon as its masks are in
  int vn = e0 + lane < e1 ? p.ci[e0 + lane] : -1;
  uint32_t bn[G];
#pragma unroll
  for (int g = 0; g < G; g++) bn[g] = 0u;
  if (vn >= 0) load_row<G>(Dn, vn, bn);
  int vnn = e0 + 32 + lane < e1 ? p.ci[e0 + 32 + lane] : -1;
  for (int base = e0; base < e1; base += 32) {
    BwdHit<G, EXT> h;
    h.v = vn;
    h.hit = false;
#pragma unroll
    for (int g = 0; g < G; g++) {
      h.bm[g] = bn[g] & o.mw[g];
      h.hit |= h.bm[g] != 0u;
    }
    vn = vnn;
#pragma unroll
    for (int g = 0; g < G; g++) bn[g] = 0u;
    if (vn >= 0) load_row<G>(Dn, vn, bn);
    vnn = base + 64 + lane < e1 ? p.ci[base + 64 + lane] : -1;
    bwd_hit_load<G, EXT>(p, h);
    if (h.hit && !h.sp) prefetch_row<G>(p.r + sidx<G>(h.v, 0, 0), h.bm);
    bwd_hits_add<G, EXT>(p, h, __ballot_sync(BC_FULL, h.sp), __ballot_sync(BC_FULL, h.hit && !h.sp), o);
    if (vn >= 0) {  // the next step's dense rows
      uint32_t m[G];
      int nb = 0;
#pragma unroll
      for (int g = 0; g < G; g++) {
        m[g] = bn[g] & o.mw[g];
        nb += __popc(m[g]);
      }
      if (nb > kSparse) prefetch_row<G>(p.r + sidx<G>(vn, 0, 0), m);
    }
  }
  if (nch == 1) {
    bwd_commit<G, EXT>(p, w, o);
    return;
  }
  bwd_fold<G, EXT>(o);
  float2 *part = p.Hpart + (size_t)(i - h0) * (32 * G);
#pragma unroll
  for (int g = 0; g < G; g++)
    if (o.mw[g]) __stcg(&part[32 * g + lane], o.acc[g]);
  __threadfence();
  int last = 0;
  if (lane == 0) last = atomicAdd(&p.Hdone[i - c], 1) == nch - 1;
  if (__shfl_sync(BC_FULL, last, 0)) {
    __threadfence();
    const float2 *p0 = p.Hpart + (size_t)(i - c - h0) * (32 * G);
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (!o.mw[g]) continue;
      float2 sum = make_float2(0.0f, 0.0f);
      for (int cc = 0; cc < nch; cc++) ff_add(sum, __ldcg(&p0[(size_t)cc * (32 * G) + 32 * g + lane]));
      o.acc[g] = sum;
    }
    bwd_commit<G, EXT>(p, w, o);
  }
}

// One lane-mode backward pass of vertex w for sources t0 and t1 (>= 0, or -1): r of each
// successor summed in edge order, then delta and r of (w, t); the BC contribution is added
// to contrib (or, serving, to the sources' request buffers).
template <int G, bool EXT>
__device__ __forceinline__ void bwd_lane_pair(const TK &p, int w, int t0, int t1, const uint32_t *Dn,
                                              float2 &contrib) {
  float2 sg[2] = {make_float2(1.0f, 0.0f), make_float2(1.0f, 0.0f)};
  float2 acc[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
  int ew[2] = {0, 0};
  const int ts[2] = {t0, t1};
#pragma unroll
  for (int z = 0; z < 2; z++) {
    if (ts[z] < 0) continue;
    const size_t idx = sidx<G>(w, ts[z]);
    if (EXT) {
      const bool o = (p.ovf[(size_t)w * G + (ts[z] >> 5)] >> (ts[z] & 31)) & 1u;
      const XS x = sig_xs(p, idx, o);
      sg[z] = ff_mant(x.m);
      ew[z] = x.e;
    } else {
      sg[z] = ff_u64(p.sig[idx]);
    }
  }
  const int g0 = t0 >> 5, g1 = t1 >= 0 ? t1 >> 5 : g0;
  const int e1 = p.rp[w + 1];
  for (int e = p.rp[w]; e < e1; e += 4) {
    int v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = e + u < e1 ? p.ci[e + u] : -1;
    uint32_t d0[4], d1[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      d0[u] = v[u] >= 0 ? Dn[(size_t)v[u] * G + g0] : 0u;
      d1[u] = (v[u] >= 0 && t1 >= 0) ? (g1 == g0 ? d0[u] : Dn[(size_t)v[u] * G + g1]) : 0u;
    }
    float2 x[2][4];
    int xe[2][4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int z = 0; z < 2; z++) {
        const uint32_t dm = z ? d1[u] : d0[u];
        const bool h = ts[z] >= 0 && ((dm >> (ts[z] & 31)) & 1u);
        const size_t idx = sidx<G>(v[u], ts[z]);
        x[z][u] = h ? p.r[idx] : make_float2(0.0f, 0.0f);
        xe[z][u] = (EXT && h) ? p.xe[idx] : 0;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int z = 0; z < 2; z++) ff_add(acc[z], EXT ? ff_scale(x[z][u], ew[z] - xe[z][u]) : x[z][u]);
  }
  const float2 om1 = ff_u64(1ull + (p.omega ? (unsigned long long)p.omega[w] : 0ull));
#pragma unroll
  for (int z = 0; z < 2; z++) {
    if (ts[z] < 0) continue;
    const size_t idx = sidx<G>(w, ts[z]);
    const float2 dl = ff_mul(p.wsrc[ts[z]], ff_mul(sg[z], acc[z]));
    float2 r = ff_mul(om1, ff_rcp(sg[z]));
    ff_add(r, acc[z]);
    p.r[idx] = r;
    if (EXT) p.xe[idx] = ew[z];
    if (p.nreq == 0) {
      ff_add(contrib, dl);
    } else if (!ff_zero(dl)) {
      p.req_bc[p.lane_req[ts[z]]][w] += ff_to(dl);
    }
  }
}

// Lane-mode backward of entry (w, sources mw): passes over the adjacency for two sources
// at a time, then one BC update (sources in increasing order).
template <int G, bool EXT>
__device__ __forceinline__ void bwd_lane_entry(const TK &p, int w, const uint32_t (&mw)[G], const uint32_t *Dn) {
  uint32_t rem[G];
#pragma unroll
  for (int g = 0; g < G; g++) rem[g] = mw[g];
  float2 contrib = make_float2(0.0f, 0.0f);
  for (;;) {
    int t0, t1;
    if (two_bits<G>(rem, t0, t1) == 0) break;
#pragma unroll
    for (int g = 0; g < G; g++) {
      if ((t0 >> 5) == g) rem[g] &= ~(1u << (t0 & 31));
      if (t1 >= 0 && (t1 >> 5) == g) rem[g] &= ~(1u << (t1 & 31));
    }
    bwd_lane_pair<G, EXT>(p, w, t0, t1, Dn, contrib);
  }
  if (p.nreq == 0 && !ff_zero(contrib)) p.bc[w] += ff_to(contrib);
}

// Lane-mode backward over A_d [a0, a1): warps take 32 consecutive entries; hub entries are
// left to the CTAs, entries with more than kLaneSrc sources or kLaneDeg edges are walked
// warp-wide one at a time.
template <int G, bool EXT>
__device__ void bwd_lanes(const TK &p, int a0, int a1, const uint32_t *Dn, int gwarp, int nwarps) {
  const int lane = lane_id();
  for (int base = a0 + gwarp * 32; base < a1; base += nwarps * 32) {
    const int k = base + lane;
    const bool in = k < a1;
    const int w = in ? p.A[k] : 0;
    const int dg = in ? vdeg(p, w) : 0;
    uint32_t mw[G];
    if (in) {
      load_row<G>(p.AM, k, mw);
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) mw[g] = 0u;
    }
    int nb = 0;
#pragma unroll
    for (int g = 0; g < G; g++) nb += __popc(mw[g]);
    const bool hub = dg >= p.hub_chunk;  // split into warp items
    const bool lanep = in && !hub && dg <= kLaneDeg && nb >= 1 && nb <= kLaneSrc;
    const bool fb = in && !hub && !lanep;
    if (lanep) bwd_lane_entry<G, EXT>(p, w, mw, Dn);
    unsigned fbm = __ballot_sync(BC_FULL, fb);
    while (fbm) {
      const int j = __ffs(fbm) - 1;
      fbm &= fbm - 1;
      const int kf = __shfl_sync(BC_FULL, k, j), wf = __shfl_sync(BC_FULL, w, j);
      BwdOwner<G, EXT> o;
      bwd_start_k<G, EXT>(p, kf, o);
      const int e1 = p.rp[wf + 1];
      for (int eb = p.rp[wf]; eb < e1; eb += 32) {
        const int e = eb + lane;
        const int v = e < e1 ? p.ci[e] : -1;
        uint32_t dm[G];
        bool hit = false;
        if (v >= 0) {
          load_row<G>(Dn, v, dm);
        } else {
#pragma unroll
          for (int g = 0; g < G; g++) dm[g] = 0u;
        }
#pragma unroll
        for (int g = 0; g < G; g++) {
          dm[g] &= o.mw[g];
          hit |= dm[g] != 0u;
        }
        unsigned hits = __ballot_sync(BC_FULL, hit);
        while (hits) {
          const int jj = __ffs(hits) - 1;
          hits &= hits - 1;
          uint32_t m[G];
#pragma unroll
          for (int g = 0; g < G; g++) m[g] = __shfl_sync(BC_FULL, dm[g], jj);
          bwd_hit<G, EXT>(p, __shfl_sync(BC_FULL, v, jj), m, o);
        }
      }
      bwd_commit<G, EXT>(p, wf, o);
    }
  }
}

// Backward level d: hubs of A_d by whole CTAs, the rest by the walk; scatter A_d's masks
// into the level-d buffer (read at level d-1) and clear A_{d+2}'s masks.  Three distinct
// buffers, so one barrier per level suffices.
template <int G, bool EXT>
__device__ void phase_bwd_level(const TK &p, int d, int a0, int a1, int Ed, int c0, int c1, int gtid,
                                int nthr, int gwarp, int nwarps) {
  const uint32_t *Dn = Fbuf<G>(p, d + 1);
  uint32_t *Dd = Fbuf<G>(p, d);
  uint32_t *Dc = Fbuf<G>(p, d + 2);
  for (long long i = (long long)a0 * G + gtid; i < (long long)a1 * G; i += nthr)
    Dd[(size_t)p.A[i / G] * G + (i % G)] = p.AM[i];
  for (long long i = (long long)c0 * G + gtid; i < (long long)c1 * G; i += nthr)
    Dc[(size_t)p.A[i / G] * G + (i % G)] = 0u;
  if (lane_level(vload64(&p.Lbits[d]), a1 - a0, (long long)Ed))
    bwd_lanes<G, EXT>(p, a0, a1, Dn, gwarp, nwarps);
  else
    bwd_walk<G, EXT>(p, a0, a1, Ed, Dn, gwarp, nwarps, &p.ctl->bq[d % 3]);
  // work items of A_d's split entries (listed at append time, one per chunk), one per warp
  // from a counter, taken by each warp as soon as its walk is done
  const int h0 = p.HEoff[d], h1 = p.HEoff[d + 1];
  int *ctr = &p.ctl->bhubq[d % 3];
  for (;;) {
    int i = 0;
    if (lane_id() == 0) i = atomicAdd(ctr, 1);
    i = h0 + __shfl_sync(BC_FULL, i, 0);
    if (i >= h1) break;
    bwd_warp_item<G, EXT>(p, i, h0, Dn);
  }
}

__device__ void leaf_terms(const TK &p) {
  if (!(p.leaf_term && p.omega)) return;
  for (int t = 0; t < p.nsrc; t++) {
    const int s = p.src[t];
    const double om = (double)p.omega[s];
    if (om > 0.0) p.bc[s] += om * (2.0 * (double)p.ctl->ns[t] - om - 3.0);
  }
}

// edges of A_d: the level-relative prefix of its last entry plus that entry's degree
__device__ __forceinline__ int level_edges(const TK &p, int a0, int a1) {
  if (a1 <= a0) return 0;
  return p.ACD[a1 - 1] + vdeg(p, p.A[a1 - 1]);
}

// Direction of the next level from the frontier's edge count ecnt: top-down -> bottom-up
// when ecnt > alpha * nnz; with beta > 0, a bottom-up sweep stays bottom-up while ecnt >
// nnz / beta (hysteresis), else the alpha test decides every level.
__device__ __forceinline__ bool next_dir(const TK &p, bool bu, int ecnt) {
  if (bu && p.beta > 0.f) return (double)ecnt * (double)p.beta > (double)p.nnz;
  return (double)ecnt > (double)p.alpha * (double)p.nnz;
}

// ------------------------------------------------------------------ persistent kernel
template <int G, bool EXT>
__global__ void __launch_bounds__(TPB<G>::value, 1) tile_persistent(TK p, int fwd_only) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int gwarp = warp_rank(), nwarps = nthr >> 5;
  GridSync *gs = &p.ctl->bar;
  sparse_acc_clear<G>();
  phase_init_vis<G>(p, gtid, nthr);
  if (!tsync(p, gs, 0, 0)) return;
  if (gtid == 0) init_sources<G>(p);
  if (!tsync(p, gs, 0, 0)) return;
  int level = 1, a_pp = 0, a_lo = 0, a_hi, ecnt;
  {
    const unsigned long long pk = vload64(&p.ctl->apack[0]);
    a_hi = (int)(pk >> 32);
    ecnt = (int)(pk & 0xffffffffull);
  }
  bool bu = false;
  while (a_hi > a_lo) {
    const bool pbu = bu;
    bu = next_dir(p, bu, ecnt);
    const bool compact = bu && pbu;  // a second bottom-up level in a row
    phase_keep<G>(p, level, a_pp, a_lo, a_hi, gtid, nthr);
    if (!bu) {
      phase_mark<G>(p, level, a_lo, a_hi, ecnt, gwarp, nwarps);
      if (!tsync(p, gs, 1, level)) return;
    } else if (compact) {
      phase_compact<G>(p, level, gwarp, nwarps);
      if (!tsync(p, gs, 1, level)) return;
    }
    phase_pull<G, EXT>(p, level, bu, compact, a_lo, a_hi, gwarp, nwarps);
    if (gtid == 0) {
      p.Lbits[level] = 0ull;  // A_level's sources are counted at the next level
      p.ctl->apack[(level + 1) % 3] = 0ull;
      p.ctl->cpack[(level + 1) % 3] = 0ull;
      p.ctl->chpk[(level + 1) % 3] = 0ull;
      p.ctl->hubq[(level + 1) % 3] = 0;
      p.ctl->wq[(level + 1) % 3] = 0;
    }
    if (!tsync(p, gs, bu ? 3 : 2, level)) return;
    const unsigned long long pk = vload64(&p.ctl->apack[level % 3]);
    a_pp = a_lo;
    a_lo = a_hi;
    a_hi = a_lo + (int)(pk >> 32);
    ecnt = (int)(pk & 0xffffffffull);
    level++;
    if (gtid == 0) {
      p.Aoff[level] = a_hi;
      p.HEoff[level] = *(volatile int *)&p.ctl->hecnt;
    }
  }
  const int lmax = level - 2;
  if (gtid == 0) {
    p.ctl->lmax = lmax;
    p.ctl->levels += level - 1;
  }
  // 64-bit mode checks only carries, so the overflow flags are exact only in extended
  // mode: a tile that overflowed reruns there, also when only sigma is exported
  if (!EXT && *(volatile int *)&p.ctl->ovf_any) {
    if (gtid == 0) atomicCAS(&p.ctl->bar.err, 0, BCD_NEEDEXT);
    return;
  }
  if (fwd_only) return;
  if (!tsync(p, gs, 4, 0)) return;
  if (lmax >= 1) {
    phase_bwd_deep<G, EXT>(p, p.Aoff[lmax], p.Aoff[lmax + 1], gtid, nthr);
    if (!tsync(p, gs, 4, lmax)) return;
    for (int d = lmax - 1; d >= 1; --d) {
      int c0 = 0, c1 = 0;
      if (d + 2 <= lmax) {
        c0 = p.Aoff[d + 2];
        c1 = p.Aoff[d + 3];
      }
      const int a0 = p.Aoff[d], a1 = p.Aoff[d + 1];
      phase_bwd_level<G, EXT>(p, d, a0, a1, level_edges(p, a0, a1), c0, c1, gtid, nthr, gwarp,
                              nwarps);
      if (gtid == 0) {  // the slots of level d - 1
        p.ctl->bhubq[(d + 2) % 3] = 0;
        p.ctl->bq[(d + 2) % 3] = 0;
      }
      if (!tsync(p, gs, 5, d)) return;
    }
  }
  if (gtid == 0) leaf_terms(p);
}

// ------------------------------------------------------------------ launched kernels
template <int G>
__global__ void __launch_bounds__(TPB<G>::value) k_init_vis(TK p) {
  phase_init_vis<G>(p, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <int G>
__global__ void k_init_src(TK p) {
  init_sources<G>(p);
  TileCtl *c = p.ctl;
  const unsigned long long pk = c->apack[0];
  c->level = 1;
  c->a_pp = 0;
  c->a_lo = 0;
  c->a_hi = (int)(pk >> 32);
  c->ecnt = (int)(pk & 0xffffffffull);
  c->pmode = 0;
  c->mode = next_dir(p, false, c->ecnt);
  c->done = c->a_hi == 0;
  if (c->done) {
    c->lmax = 0;
    c->dlevel = 0;
  }
}

template <int G>
__global__ void __launch_bounds__(TPB<G>::value) k_fwd_mark(TK p) {
  const TileCtl *c = p.ctl;
  if (c->done || c->bar.err) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  phase_keep<G>(p, c->level, c->a_pp, c->a_lo, c->a_hi, gtid, nthr);
  if (!c->mode)
    phase_mark<G>(p, c->level, c->a_lo, c->a_hi, c->ecnt, warp_rank(), nthr >> 5);
  else if (c->pmode)
    phase_compact<G>(p, c->level, warp_rank(), nthr >> 5);
}

template <int G, bool EXT>
__global__ void __launch_bounds__(TPB<G>::value, 1) k_fwd_pull(TK p) {
  const TileCtl *c = p.ctl;
  if (c->done || c->bar.err) return;
  sparse_acc_clear<G>();
  const int nthr = gridDim.x * blockDim.x;
  phase_pull<G, EXT>(p, c->level, c->mode != 0, c->mode != 0 && c->pmode != 0, c->a_lo, c->a_hi, warp_rank(),
                     nthr >> 5);
}

__global__ void k_fwd_end(TK p) {
  TileCtl *c = p.ctl;
  if (c->done || c->bar.err) return;
  int level = c->level;
  const unsigned long long pk = c->apack[level % 3];
  p.Lbits[level] = 0ull;  // A_level's sources are counted at the next level
  c->apack[(level + 1) % 3] = 0ull;
  c->cpack[(level + 1) % 3] = 0ull;
  c->chpk[(level + 1) % 3] = 0ull;
  c->hubq[(level + 1) % 3] = 0;
  c->wq[(level + 1) % 3] = 0;
  c->a_pp = c->a_lo;
  c->a_lo = c->a_hi;
  c->a_hi = c->a_lo + (int)(pk >> 32);
  c->ecnt = (int)(pk & 0xffffffffull);
  level++;
  c->level = level;
  p.Aoff[level] = c->a_hi;
  p.HEoff[level] = c->hecnt;
  c->pmode = c->mode;
  c->mode = next_dir(p, c->mode != 0, c->ecnt);
  if ((long long)c->a_hi > p.capA) {  // appends past the active-list capacity were dropped
    atomicCAS(&c->bar.err, 0, BCD_CAPACITY);
    c->done = 1;
    return;
  }
  if (c->a_hi == c->a_lo) {
    c->done = 1;
    c->lmax = level - 2;
    c->levels += level - 1;
    c->dlevel = level - 3;  // first backward level (lmax - 1)
  }
}

template <int G, bool EXT>
__global__ void __launch_bounds__(TPB<G>::value) k_bwd_deep(TK p) {
  const TileCtl *c = p.ctl;
  if (c->lmax < 1 || c->bar.err) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  phase_bwd_deep<G, EXT>(p, p.Aoff[c->lmax], p.Aoff[c->lmax + 1], gtid, nthr);
}

template <int G, bool EXT>
__global__ void __launch_bounds__(TPB<G>::value, 1) k_bwd_level(TK p) {
  const TileCtl *c = p.ctl;
  const int d = c->dlevel, lmax = c->lmax;
  if (d < 1 || c->bar.err) return;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  int c0 = 0, c1 = 0;
  if (d + 2 <= lmax) {
    c0 = p.Aoff[d + 2];
    c1 = p.Aoff[d + 3];
  }
  const int a0 = p.Aoff[d], a1 = p.Aoff[d + 1];
  phase_bwd_level<G, EXT>(p, d, a0, a1, level_edges(p, a0, a1), c0, c1, gtid, nthr, warp_rank(),
                          nthr >> 5);
}

__global__ void k_bwd_step(TK p) {
  if (p.ctl->dlevel >= 1) {
    p.ctl->dlevel--;
    p.ctl->bhubq[p.ctl->dlevel % 3] = 0;
    p.ctl->bq[p.ctl->dlevel % 3] = 0;
  }
}

__global__ void k_leaf(TK p) {
  if (!p.ctl->bar.err) leaf_terms(p);
}

// Export depth / sigma / overflow of the tile's sources, source-major [k][n].
template <int G>
__global__ void k_export(TK p, int lmax, int32_t *depth, unsigned long long *sigma, uint8_t *ovf) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  for (int t = gtid; t < p.nsrc; t += nthr) {  // the sources themselves (also degree 0)
    const size_t o = (size_t)t * p.n + p.src[t];
    depth[o] = 0;
    if (sigma) sigma[o] = 1ull;
    if (ovf) ovf[o] = 0;
  }
  for (int l = 1; l <= lmax; l++) {
    const int a0 = p.Aoff[l], a1 = p.Aoff[l + 1];
    for (long long i = (long long)a0 * 32 * G + gtid; i < (long long)a1 * 32 * G; i += nthr) {
      const int k = (int)(i / (32 * G)), t = (int)(i % (32 * G));
      if (t >= p.nsrc) continue;
      const int w = p.A[k];
      const uint32_t m = p.AM[(size_t)k * G + (t >> 5)];
      if ((m >> (t & 31)) & 1u) {
        const size_t o = (size_t)t * p.n + w;
        depth[o] = l;
        if (sigma) sigma[o] = p.sig[sidx<G>(w, t)];
        if (ovf) ovf[o] = (p.ovf[(size_t)w * G + (t >> 5)] >> (t & 31)) & 1u;
      }
    }
  }
}

// Per-graph lists: hubs, and the bottom-up walk list (non-hub vertices with an edge).
__global__ void k_lists(int32_t n, const int32_t *rp, int hub, int32_t *hubs, int *nh, int32_t *flag) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int d = rp[v + 1] - rp[v];
    if (d >= hub) hubs[atomicAdd(nh, 1)] = v;
    flag[v] = (d > 0 && d < hub) ? 1 : 0;
  }
}
__global__ void k_lists_fill(int32_t n, const int32_t *rp, const int32_t *flag, const int32_t *pos,
                             int32_t *L, int32_t *RP, int32_t *degs) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (flag[v]) {
      L[pos[v]] = v;
      RP[pos[v]] = rp[v];
      degs[pos[v]] = rp[v + 1] - rp[v];
    }
}

// chunk count of each hub: its forward work items
__global__ void k_hub_chunks(const int32_t *hubs, int nh, const int32_t *rp, int chunk, int32_t *cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nh; k += gridDim.x * blockDim.x) {
    const int v = hubs[k];
    cnt[k] = (rp[v + 1] - rp[v] + chunk - 1) / chunk;
  }
}

__global__ void k_wsrc(const int32_t *src, int nsrc, const int32_t *omega, float2 *wsrc, int T) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T)
    wsrc[t] = t < nsrc ? ff_u64(1ull + (omega ? (unsigned long long)omega[src[t]] : 0ull)) : make_float2(0.0f, 0.0f);
}

// ------------------------------------------------------------------ host dispatch helpers
struct KPtrs {
  void *persistent, *pull, *mark, *init_vis, *init_src, *bdeep, *blevel, *exportk;
  int tpb;
};

template <int G, bool EXT>
KPtrs kptrs_t() {
  return KPtrs{(void *)tile_persistent<G, EXT>, (void *)k_fwd_pull<G, EXT>, (void *)k_fwd_mark<G>,
               (void *)k_init_vis<G>, (void *)k_init_src<G>, (void *)k_bwd_deep<G, EXT>,
               (void *)k_bwd_level<G, EXT>, (void *)k_export<G>, TPB<G>::value};
}

KPtrs kptrs(int G, bool ext) {
  switch (G) {
    case 1: return ext ? kptrs_t<1, true>() : kptrs_t<1, false>();
    case 2: return ext ? kptrs_t<2, true>() : kptrs_t<2, false>();
    case 4: return ext ? kptrs_t<4, true>() : kptrs_t<4, false>();
    default: return ext ? kptrs_t<8, true>() : kptrs_t<8, false>();
  }
}

}  // namespace

// ================================================================== host side
static void ws_release(Ctx *ctx, TileWS *ws, bool main, bool ext, bool A) {
  if (main && ws->Hpart) {
    cudaFree(ws->Hpart);
    cudaFree(ws->FPm);
    ctx->mem.release(nullptr, ws->bytes_hpart);
    ws->Hpart = nullptr;
    ws->FPm = nullptr;
    ws->hpart_items = 0;
    ws->bytes_hpart = 0;
  }
  if (main && ws->FPx) {
    cudaFree(ws->FPx);
    cudaFree(ws->FPe);
    ctx->mem.release(nullptr, ws->bytes_hpart_ext);
    ws->FPx = nullptr;
    ws->FPe = nullptr;
    ws->hpart_ext_items = 0;
    ws->bytes_hpart_ext = 0;
  }
  if (main && ws->ctl) {
    void *ptrs[] = {ws->vis, ws->F, ws->ovf, ws->cand, ws->sig, ws->r, ws->Aoff, ws->Lbits, ws->HEoff,
                    ws->C, ws->CPD, ws->CRP, ws->Ch, ws->ChP, ws->Fdone, ws->wsrc, ws->ctl};
    for (void *q : ptrs) cudaFree(q);
    ctx->mem.release(nullptr, ws->bytes_main);
    ws->vis = ws->F = ws->ovf = ws->cand = nullptr;
    ws->sig = nullptr;
    ws->r = nullptr;
    ws->Aoff = ws->HEoff = ws->C = ws->CPD = ws->CRP = ws->Ch = ws->ChP = ws->Fdone = nullptr;
    ws->Lbits = nullptr;
    ws->wsrc = nullptr;
    ws->ctl = nullptr;
    ws->bytes_main = 0;
  }
  if (ext && ws->ext_arrays) {
    cudaFree(ws->xm);
    cudaFree(ws->xe);
    ctx->mem.release(nullptr, ws->bytes_ext);
    ws->xm = nullptr;
    ws->xe = nullptr;
    ws->ext_arrays = false;
    ws->bytes_ext = 0;
  }
  if (A && ws->A) {
    cudaFree(ws->A);
    cudaFree(ws->ACD);
    cudaFree(ws->ARP);
    cudaFree(ws->AM);
    cudaFree(ws->HE);
    cudaFree(ws->HEk);
    cudaFree(ws->Hdone);
    ws->HE = ws->HEk = ws->Hdone = nullptr;
    ctx->mem.release(nullptr, ws->bytes_A);
    ws->A = ws->ACD = ws->ARP = nullptr;
    ws->AM = nullptr;
    ws->bytes_A = 0;
    ws->capA = 0;
  }
}

static void lists_release(Ctx *ctx, TileWS *ws) {
  if (!ws->hubs) return;
  cudaFree(ws->hubs);
  cudaFree(ws->Lbu);
  cudaFree(ws->PDbu);
  cudaFree(ws->RPbu);
  cudaFree(ws->HPbu);
  ctx->mem.release(nullptr, ws->bytes_lists);
  ws->hubs = ws->Lbu = ws->PDbu = ws->RPbu = ws->HPbu = nullptr;
  ws->lists_for = nullptr;
  ws->bytes_lists = 0;
}

void tile_free(Ctx *ctx, TileWS *ws) {
  if (!ws) return;
  ws_release(ctx, ws, true, true, true);
  lists_release(ctx, ws);
  delete ws;
}

#define TA(ptr, bytes)                                                                    \
  do {                                                                                    \
    const size_t b_ = (bytes);                                                            \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), b_ != 0 ? b_ : (size_t)16);     \
  } while (0)

static bc_status ws_main(Ctx *ctx, TileWS *ws, int n, int T, cudaStream_t st) {
  if (ws->ctl && ws->n == n && ws->T == T) return BC_OK;
  ws_release(ctx, ws, true, true, true);
  const int G = T / 32;
  const size_t N = (size_t)n, NG = N * G, NT = N * T;
  const size_t bytes = NG * 4 * 5 + NT * 16 + (N / 32 + 1) * 4 + (N + 3) * 4 + (N + 3) * 8 + N * 24 +
                       T * 8 + sizeof(TileCtl);
  bc_status s = ctx->mem.alloc(nullptr, bytes);
  if (s) return s;
  cudaError_t e = cudaSuccess;
  TA(ws->vis, NG * 4);
  TA(ws->F, NG * 4 * 3);
  TA(ws->ovf, NG * 4);
  TA(ws->cand, (N / 32 + 1) * 4);
  TA(ws->sig, NT * 8);
  TA(ws->r, NT * 8);
  TA(ws->Aoff, (N + 3) * 4);
  TA(ws->Lbits, (N + 3) * 8);
  TA(ws->HEoff, (N + 3) * 4);
  TA(ws->C, N * 4);
  TA(ws->CPD, N * 4);
  TA(ws->CRP, N * 4);
  TA(ws->Ch, N * 4);
  TA(ws->ChP, N * 4);
  TA(ws->Fdone, N * 4);
  TA(ws->wsrc, (size_t)T * 8);
  TA(ws->ctl, sizeof(TileCtl));
  ws->n = n;
  ws->T = T;
  ws->G = G;
  ws->bytes_main = bytes;
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws_release(ctx, ws, true, false, false);
    return fail(BC_ENOMEM, std::string("tile workspace allocation failed: ") + cudaGetErrorString(e));
  }
  // cleared before any launch on any stream uses it (a plain cudaMemset may still be
  // running when the host goes on, and callers' streams need not sync with its stream)
  BC_CUDA_TRY(cudaMemsetAsync(ws->cand, 0, (N / 32 + 1) * 4, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  return BC_OK;
}

static bc_status ws_ext(Ctx *ctx, TileWS *ws) {
  if (ws->ext_arrays) return BC_OK;
  const size_t NT = (size_t)ws->n * ws->T;
  bc_status s = ctx->mem.alloc(nullptr, NT * 12);
  if (s) return s;
  cudaError_t e = cudaSuccess;
  TA(ws->xm, NT * 8);
  TA(ws->xe, NT * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ws->xm) cudaFree(ws->xm);
    ws->xm = nullptr;
    ctx->mem.release(nullptr, NT * 12);
    return fail(BC_ENOMEM, "extended-sigma arrays allocation failed");
  }
  ws->ext_arrays = true;
  ws->bytes_ext = NT * 12;
  return BC_OK;
}

static bc_status ws_A(Ctx *ctx, TileWS *ws, int64_t cap) {
  if (ws->A && ws->capA >= cap) return BC_OK;
  ws_release(ctx, ws, false, false, true);
  const size_t bytes = (size_t)cap * (24 + 4 * ws->G);
  bc_status s = ctx->mem.alloc(nullptr, bytes);
  if (s) return s;
  cudaError_t e = cudaSuccess;
  TA(ws->A, (size_t)cap * 4);
  TA(ws->ACD, (size_t)cap * 4);
  TA(ws->ARP, (size_t)cap * 4);
  TA(ws->HE, (size_t)cap * 4);
  TA(ws->HEk, (size_t)cap * 4);
  TA(ws->Hdone, (size_t)cap * 4);
  TA(ws->AM, (size_t)cap * 4 * ws->G);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->mem.release(nullptr, bytes);
    void *ptrs[] = {ws->A, ws->ACD, ws->ARP, ws->HE, ws->HEk, ws->Hdone, ws->AM};
    for (void *q : ptrs)
      if (q) cudaFree(q);
    ws->A = ws->ACD = ws->ARP = ws->HE = ws->HEk = ws->Hdone = nullptr;
    ws->AM = nullptr;
    return fail(BC_ENOMEM, "tile active-list allocation failed");
  }
  ws->capA = cap;
  ws->bytes_A = bytes;
  return BC_OK;
}

// Partial sums of one level's work items (a level lists each vertex at most once).
static bc_status ws_hpart(Ctx *ctx, TileWS *ws, int64_t nnz, int hub, int hub_chunk, bool ext) {
  // forward: at most nnz / hub_chunk + nnz / hub items (the chunks, plus one partial chunk
  // per split candidate); backward: at most 2 nnz / hub_chunk
  const int64_t items = nnz / hub_chunk + nnz / (hub < hub_chunk ? hub : hub_chunk) + 16;
  if (!(ws->Hpart && ws->hpart_items >= items)) {
    if (ws->Hpart) {
      cudaFree(ws->Hpart);
      cudaFree(ws->FPm);
      ctx->mem.release(nullptr, ws->bytes_hpart);
      ws->Hpart = nullptr;
      ws->FPm = nullptr;
      ws->hpart_items = 0;
    }
    const size_t bytes = (size_t)items * ws->T * sizeof(float2) + (size_t)items * 2 * ws->G * 4;
    bc_status s = ctx->mem.alloc(nullptr, bytes);
    if (s) return s;
    cudaError_t e = cudaSuccess;
    TA(ws->Hpart, (size_t)items * ws->T * sizeof(float2));
    TA(ws->FPm, (size_t)items * 2 * ws->G * 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ws->Hpart) cudaFree(ws->Hpart);
      if (ws->FPm) cudaFree(ws->FPm);
      ws->Hpart = nullptr;
      ws->FPm = nullptr;
      ctx->mem.release(nullptr, bytes);
      return fail(BC_ENOMEM, "tile work-item partials allocation failed");
    }
    ws->hpart_items = items;
    ws->bytes_hpart = bytes;
  }
  if (ext && !(ws->FPx && ws->hpart_ext_items >= items)) {
    if (ws->FPx) {
      cudaFree(ws->FPx);
      cudaFree(ws->FPe);
      ctx->mem.release(nullptr, ws->bytes_hpart_ext);
      ws->FPx = nullptr;
      ws->FPe = nullptr;
      ws->hpart_ext_items = 0;
    }
    const size_t bytes = (size_t)items * ws->T * 12;
    bc_status s = ctx->mem.alloc(nullptr, bytes);
    if (s) return s;
    cudaError_t e = cudaSuccess;
    TA(ws->FPx, (size_t)items * ws->T * 8);
    TA(ws->FPe, (size_t)items * ws->T * 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ws->FPx) cudaFree(ws->FPx);
      if (ws->FPe) cudaFree(ws->FPe);
      ws->FPx = nullptr;
      ws->FPe = nullptr;
      ctx->mem.release(nullptr, bytes);
      return fail(BC_ENOMEM, "tile extended work-item partials allocation failed");
    }
    ws->hpart_ext_items = items;
    ws->bytes_hpart_ext = bytes;
  }
  return BC_OK;
}

static bc_status ws_lists(Ctx *ctx, TileWS *ws, const DeviceGraph *dg, int hub, int chunk, cudaStream_t st) {
  if (ws->hubs && ws->lists_for == dg->rp && ws->lists_hub == hub && ws->lists_chunk == chunk) return BC_OK;
  lists_release(ctx, ws);
  const size_t N = (size_t)dg->n;
  const size_t bytes = N * 4 * 5 + 20;
  bc_status s = ctx->mem.alloc(nullptr, bytes);
  if (s) return s;
  cudaError_t e = cudaSuccess;
  TA(ws->hubs, N * 4);
  TA(ws->Lbu, N * 4);
  TA(ws->PDbu, N * 4 + 4);
  TA(ws->RPbu, N * 4);
  TA(ws->HPbu, N * 4 + 4);
  int32_t *flag = nullptr, *pos = nullptr, *degs = nullptr;
  int *d_cnt = nullptr;
  void *scratch = nullptr;
  TA(flag, (N + 1) * 4);
  TA(pos, (N + 1) * 4);
  TA(degs, (N + 1) * 4);
  TA(d_cnt, 16);
  TA(scratch, scan_scratch_bytes((int64_t)N + 1));
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, (N + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(degs, 0, (N + 1) * 4, st);
  if (e == cudaSuccess) {
    k_lists<<<ctx->num_sms * 4, 256, 0, st>>>(dg->n, dg->rp, hub, ws->hubs, d_cnt, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_exclusive_i32(flag, pos, (int64_t)N + 1, scratch, st);
  if (e == cudaSuccess) {
    k_lists_fill<<<ctx->num_sms * 4, 256, 0, st>>>(dg->n, dg->rp, flag, pos, ws->Lbu, ws->RPbu, degs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h + 1, pos + N, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // degree prefix of the bottom-up list (degs[nbu] is 0, so PDbu[nbu] is the total)
  if (e == cudaSuccess) e = scan_exclusive_i32(degs, ws->PDbu, (int64_t)h[1] + 1, scratch, st);
  int ebu = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ebu, ws->PDbu + h[1], 4, cudaMemcpyDeviceToHost, st);
  // work items of the hubs (bottom-up levels): exclusive prefix of their chunk counts
  if (e == cudaSuccess) e = cudaMemsetAsync(degs, 0, ((size_t)h[0] + 1) * 4, st);
  if (e == cudaSuccess && h[0] > 0) {
    k_hub_chunks<<<ctx->num_sms, 256, 0, st>>>(ws->hubs, h[0], dg->rp, chunk, degs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_exclusive_i32(degs, ws->HPbu, (int64_t)h[0] + 1, scratch, st);
  int nitems = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nitems, ws->HPbu + h[0], 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (flag) cudaFree(flag);
  if (pos) cudaFree(pos);
  if (degs) cudaFree(degs);
  if (d_cnt) cudaFree(d_cnt);
  if (scratch) cudaFree(scratch);
  ws->bytes_lists = bytes;
  if (e != cudaSuccess) {
    lists_release(ctx, ws);
    return cuda_fail(e, "tile vertex lists");
  }
  ws->nhubs = h[0];
  ws->nbu = h[1];
  ws->Ebu = ebu;
  ws->nhub_items = nitems;
  ws->lists_for = dg->rp;
  ws->lists_hub = hub;
  ws->lists_chunk = chunk;
  return BC_OK;
}

static bc_status launch(void *f, dim3 grid, dim3 block, TK &p, size_t smem, cudaStream_t st) {
  void *args[] = {&p};
  const cudaError_t e = cudaLaunchKernel(f, grid, block, args, smem, st);
  return e == cudaSuccess ? BC_OK : cuda_fail(e, "cudaLaunchKernel (tile phase)");
}

static bc_status capture_chunk(cudaStream_t st, cudaGraphExec_t *out, const KPtrs &k, dim3 grid,
                               dim3 block, TK &p, bool fwd) {
  cudaGraph_t graph;
  BC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  bc_status s = BC_OK;
  for (int i = 0; i < kLevelsPerChunk && !s; i++) {
    if (fwd) {
      s = launch(k.mark, grid, block, p, 0, st);
      if (!s) s = launch(k.pull, grid, block, p, 0, st);
      if (!s) s = launch((void *)k_fwd_end, dim3(1), dim3(1), p, 0, st);
    } else {
      s = launch(k.blevel, grid, block, p, 0, st);
      if (!s) s = launch((void *)k_bwd_step, dim3(1), dim3(1), p, 0, st);
    }
  }
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (s) return s;
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
  return BC_OK;
}

// Run one tile (forward + backward) in loop mode `mode`; returns the device error code in
// *derr and the number of kernel launches in *launches.
static bc_status run_tile(Ctx *ctx, TileWS *ws, TK &p, int G, bool ext, int mode, bool fwd_only,
                          cudaStream_t st, int *derr, int64_t *launches, int *lmax_out) {
  const size_t N = (size_t)ws->n, NG = N * G;
  const KPtrs k = kptrs(G, ext);
  bc_status s = BC_OK;
  BC_CUDA_TRY(cudaMemsetAsync(ws->F, 0, NG * 4 * 3, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->ovf, 0, NG * 4, st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(TileCtl), st));
  BC_CUDA_TRY(cudaMemsetAsync(ws->Fdone, 0, N * 4, st));  // last-finisher counters (a failed tile may leave some set)
  const int nsm = ctx->num_sms;
  const dim3 grid(nsm), block(k.tpb);
  *launches = 0;
  *derr = 0;
  if (mode == 0) {
    int fo = fwd_only ? 1 : 0;
    void *args[] = {&p, &fo};
    const cudaError_t le = cudaLaunchCooperativeKernel(k.persistent, grid, block, args, 0, st);
    if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(tile)");
    *launches = 1;
  } else {
    s = launch(k.init_vis, grid, block, p, 0, st);
    if (!s) s = launch(k.init_src, dim3(1), dim3(1), p, 0, st);
    if (s) return s;
    *launches += 2;
    cudaGraphExec_t gexec = nullptr;
    if (mode == 2) {
      s = capture_chunk(st, &gexec, k, grid, block, p, true);
      if (s) return s;
    }
    int guard = 0;
    for (;;) {
      if (mode == 2) {
        const cudaError_t ce = cudaGraphLaunch(gexec, st);
        if (ce != cudaSuccess) {
          cudaGraphExecDestroy(gexec);
          return cuda_fail(ce, "cudaGraphLaunch");
        }
      } else {
        for (int i = 0; i < kLevelsPerChunk && !s; i++) {
          s = launch(k.mark, grid, block, p, 0, st);
          if (!s) s = launch(k.pull, grid, block, p, 0, st);
          if (!s) s = launch((void *)k_fwd_end, dim3(1), dim3(1), p, 0, st);
        }
        if (s) return s;
      }
      *launches += 3 * kLevelsPerChunk;
      int hd[2];
      BC_CUDA_TRY(cudaMemcpyAsync(hd, &p.ctl->bar.err, 4, cudaMemcpyDeviceToHost, st));
      BC_CUDA_TRY(cudaMemcpyAsync(hd + 1, &p.ctl->done, 4, cudaMemcpyDeviceToHost, st));
      BC_CUDA_TRY(cudaStreamSynchronize(st));
      if (hd[0]) {  // device error (capacity): stop, the caller retries or fails
        if (gexec) cudaGraphExecDestroy(gexec);
        *derr = hd[0];
        return BC_OK;
      }
      if (hd[1]) break;
      if (++guard > ws->n / kLevelsPerChunk + 4) {  // levels <= n
        if (gexec) cudaGraphExecDestroy(gexec);
        return fail(BC_ECUDA, "tile level loop did not terminate");
      }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    int hc[2];
    BC_CUDA_TRY(cudaMemcpyAsync(hc, &p.ctl->ovf_any, 4, cudaMemcpyDeviceToHost, st));
    BC_CUDA_TRY(cudaMemcpyAsync(hc + 1, &p.ctl->lmax, 4, cudaMemcpyDeviceToHost, st));
    BC_CUDA_TRY(cudaStreamSynchronize(st));
    *lmax_out = hc[1];
    if (!ext && hc[0]) {
      *derr = BCD_NEEDEXT;
      return BC_OK;
    }
    if (fwd_only) return BC_OK;
    const int lmax = hc[1];
    if (lmax >= 1) {
      s = launch(k.bdeep, grid, block, p, 0, st);
      if (s) return s;
      *launches += 1;
      const int nb = lmax - 1;  // backward levels lmax-1 .. 1
      if (mode == 2 && nb > 0) {
        s = capture_chunk(st, &gexec, k, grid, block, p, false);
        if (s) return s;
        for (int c = 0; c < (nb + kLevelsPerChunk - 1) / kLevelsPerChunk; c++) {
          const cudaError_t le = cudaGraphLaunch(gexec, st);
          if (le != cudaSuccess) {
            cudaGraphExecDestroy(gexec);
            return cuda_fail(le, "cudaGraphLaunch");
          }
          *launches += 2 * kLevelsPerChunk;
        }
        cudaGraphExecDestroy(gexec);
      } else {
        for (int i = 0; i < nb && !s; i++) {
          s = launch(k.blevel, grid, block, p, 0, st);
          if (!s) s = launch((void *)k_bwd_step, dim3(1), dim3(1), p, 0, st);
          *launches += 2;
        }
        if (s) return s;
      }
    }
    s = launch((void *)k_leaf, dim3(1), dim3(1), p, 0, st);
    if (s) return s;
    *launches += 1;
  }
  TileCtl h;
  BC_CUDA_TRY(cudaMemcpyAsync(&h, ws->ctl, sizeof(TileCtl), cudaMemcpyDeviceToHost, st));
  BC_CUDA_TRY(cudaStreamSynchronize(st));
  *derr = h.bar.err;
  *lmax_out = h.lmax;
  return BC_OK;
}

bc_status tile_run(Ctx *ctx, Graph *g, TileWS **wsp, const TileArgs &a, cudaStream_t st,
                   bc_stats *acc) {
  (void)g;
  if (a.nsrc <= 0) return BC_OK;
  if (a.T != 32 && a.T != 64 && a.T != 128 && a.T != 256)
    return fail(BC_EINVAL, "tile width must be 32, 64, 128 or 256");
  const DeviceGraph *dg = a.g;
  if (!*wsp) {
    *wsp = new (std::nothrow) TileWS();
    if (!*wsp) return fail(BC_ENOMEM, "host allocation failed");
  }
  TileWS *ws = *wsp;
  const int hub = a.hub > 0 ? a.hub : kHubDefault;
  const int hub_chunk = a.hub_chunk > 0 ? a.hub_chunk : kHubChunkDefault;
  if (hub_chunk < 256 || hub_chunk % 32 || hub < 64)
    return fail(BC_EINVAL, "tile path: hub chunk must be a multiple of 32 and >= 256, hub degree >= 64");
  bc_status s = ws_main(ctx, ws, dg->n, a.T, st);
  if (!s) s = ws_lists(ctx, ws, dg, hub, hub_chunk, st);
  if (!s) s = ws_hpart(ctx, ws, dg->nnz, hub, hub_chunk, false);
  if (s) return s;
  const int G = a.T / 32;
  if (!ws->A) {
    s = ws_A(ctx, ws, (int64_t)dg->n * 4 + 1024);
    if (s) return s;
  }
  cudaEvent_t e0, e1;
  BC_CUDA_TRY(cudaEventCreate(&e0));
  BC_CUDA_TRY(cudaEventCreate(&e1));
  float total_ms = 0.f;
  unsigned long long *trace_buf = nullptr;
  int64_t launches_total = 0, levels_total = 0, ovf_sources = 0, reached = 0, reached_arcs = 0;
  int maxd = 0;
  for (int t0 = 0; t0 < a.nsrc && !s; t0 += a.T) {
    const int nt = a.nsrc - t0 < a.T ? a.nsrc - t0 : a.T;
    bool ext = ws->ext_sticky;
    for (int attempt = 0; attempt < 24; attempt++) {
      if (ext) {
        s = ws_ext(ctx, ws);
        if (!s) s = ws_hpart(ctx, ws, dg->nnz, hub, hub_chunk, true);
        if (s) break;
      }
      TK p;
      memset(&p, 0, sizeof(p));
      p.n = dg->n;
      p.nnz = dg->nnz;
      p.nsrc = nt;
      p.rp = dg->rp;
      p.ci = dg->ci;
      p.omega = a.omega;
      p.src = a.src + t0;
      p.bc = a.bc;
      p.leaf_term = a.omega != nullptr;
      p.vis = ws->vis;
      p.F = ws->F;
      p.ovf = ws->ovf;
      p.cand = ws->cand;
      p.sig = ws->sig;
      p.r = ws->r;
      p.xm = ws->xm;
      p.xe = ws->xe;
      p.A = ws->A;
      p.ACD = ws->ACD;
      p.ARP = ws->ARP;
      p.AM = ws->AM;
      p.capA = ws->capA;
      p.Aoff = ws->Aoff;
      p.Lbits = ws->Lbits;
      p.HE = ws->HE;
      p.HEoff = ws->HEoff;
      p.HEk = ws->HEk;
      p.Hdone = ws->Hdone;
      p.Hpart = ws->Hpart;
      p.FPs = (unsigned long long *)ws->Hpart;
      p.FPm = ws->FPm;
      p.FPx = ws->FPx;
      p.FPe = ws->FPe;
      p.Fdone = ws->Fdone;
      p.HPbu = ws->HPbu;
      p.nhub_items = ws->nhub_items;
      p.C = ws->C;
      p.CPD = ws->CPD;
      p.CRP = ws->CRP;
      p.Ch = ws->Ch;
      p.ChP = ws->ChP;
      p.hubs = ws->hubs;
      p.Lbu = ws->Lbu;
      p.PDbu = ws->PDbu;
      p.RPbu = ws->RPbu;
      p.nhubs = ws->nhubs;
      p.nbu = ws->nbu;
      p.Ebu = ws->Ebu;
      p.wsrc = ws->wsrc;
      p.ctl = ws->ctl;
      for (int gi = 0; gi < 8; gi++) {
        uint32_t m = 0;
        for (int b = 0; b < 32; b++)
          if (gi * 32 + b >= nt) m |= 1u << b;
        p.unused[gi] = m;
      }
      p.alpha = a.alpha;
      p.beta = a.beta;
      p.hub = hub;
      p.hub_chunk = hub_chunk;
      p.nreq = a.nreq;
      p.lane_req = a.lane_req ? a.lane_req + t0 : nullptr;
      p.req_bc = a.req_bc;
      p.limit_ns = ctx->wait_limit_ns;
      static const char *trace_file = getenv("BC_TRACE_FILE");
      if (trace_file && !trace_buf) {
        if (cudaMalloc(&trace_buf, (size_t)(1 << 20) * 16) != cudaSuccess) {
          cudaGetLastError();
          trace_buf = nullptr;
        }
      }
      p.trace = trace_buf;
      p.trace_cap = trace_buf ? (1 << 20) : 0;
      k_wsrc<<<(a.T + 255) / 256, 256, 0, st>>>(p.src, nt, a.omega, ws->wsrc, a.T);
      BC_CUDA_TRY(cudaEventRecord(e0, st));
      int derr = 0, lmax = 0;
      int64_t launches = 0;
      const bool fwd_only = a.out_depth != nullptr;
      s = run_tile(ctx, ws, p, G, ext, a.loop_mode, fwd_only, st, &derr, &launches, &lmax);
      if (s) break;
      BC_CUDA_TRY(cudaEventRecord(e1, st));
      BC_CUDA_TRY(cudaEventSynchronize(e1));
      if (derr == BCD_CAPACITY) {
        BC_CUDA_TRY(cudaMemsetAsync(ws->cand, 0, ((size_t)ws->n / 32 + 1) * 4, st));
        s = ws_A(ctx, ws, ws->capA * 2);
        if (s) break;
        continue;
      }
      if (derr == BCD_NEEDEXT) {
        ext = true;
        ws->ext_sticky = true;
        continue;
      }
      if (derr == BCD_TIMEOUT) {
        cudaMemsetAsync(ws->cand, 0, ((size_t)ws->n / 32 + 1) * 4, st);
        cudaStreamSynchronize(st);
        s = fail(BC_ETIMEDOUT, "tile kernel: a grid barrier wait passed its limit");
        break;
      }
      if (derr != 0) {
        s = fail(BC_ECUDA, "tile kernel reported device error " + std::to_string(derr));
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      total_ms += ms;
      launches_total += launches + 1;  // + the per-tile weight kernel
      TileCtl h;
      BC_CUDA_TRY(cudaMemcpy(&h, ws->ctl, sizeof(TileCtl), cudaMemcpyDeviceToHost));
      if (trace_buf) {
        const int cnt = h.trace_n < (1 << 20) ? h.trace_n : (1 << 20);
        std::vector<unsigned long long> tv((size_t)cnt * 2);
        cudaMemcpy(tv.data(), trace_buf, (size_t)cnt * 16, cudaMemcpyDeviceToHost);
        if (FILE *f = fopen(getenv("BC_TRACE_FILE"), "a")) {
          for (int i = 0; i < cnt; i++)
            fprintf(f, "%d,%d,%llu\n", (int)(tv[2 * i] >> 56), (int)((tv[2 * i] >> 24) & 0xffffffffull),
                    tv[2 * i + 1]);
          fclose(f);
        }
      }
      levels_total += h.levels;
      reached += (int64_t)h.reached;
      reached_arcs += (int64_t)h.reached_arcs;
      for (int gi = 0; gi < G; gi++) ovf_sources += __builtin_popcount(h.ovf_lanes[gi]);
      if (lmax > maxd) maxd = lmax;
      if (fwd_only) {
        void *fx = kptrs(G, false).exportk;
        void *args[] = {&p, &lmax, (void *)&a.out_depth, (void *)&a.out_sigma, (void *)&a.out_ovf};
        BC_CUDA_TRY(cudaMemsetAsync(a.out_depth, 0xff, (size_t)nt * ws->n * 4, st));
        if (a.out_sigma) BC_CUDA_TRY(cudaMemsetAsync(a.out_sigma, 0, (size_t)nt * ws->n * 8, st));
        if (a.out_ovf) BC_CUDA_TRY(cudaMemsetAsync(a.out_ovf, 0, (size_t)nt * ws->n, st));
        BC_CUDA_TRY(cudaLaunchKernel(fx, dim3(ctx->num_sms * 4), dim3(256), args, 0, st));
        BC_CUDA_TRY(cudaStreamSynchronize(st));
      }
      break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (trace_buf) cudaFree(trace_buf);
  if (s) return s;
  if (acc) {
    acc->seconds += total_ms * 1e-3;
    acc->sources += a.nsrc;
    acc->kernel_launches += launches_total;
    acc->levels += levels_total;
    acc->sigma_overflow_sources += ovf_sources;
    acc->reached_vertices += reached;
    acc->reached_arcs += reached_arcs;
    if (maxd > acc->max_depth) acc->max_depth = maxd;
    acc->tile_width = a.T;
  }
  return BC_OK;
}

}  // namespace bcl

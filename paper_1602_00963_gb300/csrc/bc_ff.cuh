// Extended-range (mantissa, exponent) and float-float ("double-float") arithmetic for the
// sweeps (product code only).
//
// FP64 runs at a small fraction of the FP32 rate on GB300, so the backward sweeps keep
// r = (1 + delta + omega) / sigma and its sums as unevaluated pairs of floats (value
// hi + lo, about 48 significant bits): Knuth's two-sum for additions, FMA-exact products,
// one Newton step for reciprocals.  Sigma enters from its integer (or extended-range
// mantissa) bits; only per-vertex BC updates are done in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bc_common.cuh"

namespace bcl {

constexpr long long kFFMantBits = 0x000fffffffffffffll;

// ------------------------------------------------------------------ extended range
// Path counts beyond 2^64 (grids reach 2^1700) are carried as value = m * 2^e.  Every m
// here is +0 or a positive normal double, so scaling and normalising are integer
// operations on the IEEE-754 exponent field (no FP64 pipe).
struct XS {
  double m;
  int e;
};
__device__ __forceinline__ bool is_zero(double m) { return __double_as_longlong(m) == 0ll; }
// m * 2^k; results below the normal range become 0 (they join sums of terms >= 2^-1 of
// the same scale, where they are far below the FP64 rounding)
__device__ __forceinline__ double scale2(double m, int k) {
  const long long b = __double_as_longlong(m);
  if (b == 0ll) return 0.0;
  const int ne = (int)(b >> 52) + k;
  if (ne <= 0) return 0.0;
  return __longlong_as_double((b & kFFMantBits) | ((long long)ne << 52));
}
// sigma mod 2^64 (not overflowed) as m in [0.5, 1) and e; the mantissa keeps the top 53
// bits (truncated: relative error < 2^-52)
__device__ __forceinline__ XS xs_u64(unsigned long long s) {
  XS x;
  if (!s) {
    x.m = 0.0;
    x.e = 0;
    return x;
  }
  const int lz = __clzll((long long)s);
  const unsigned long long t = s << lz;
  x.m = __longlong_as_double((long long)((t >> 11) & (unsigned long long)kFFMantBits) | (1022ll << 52));
  x.e = 64 - lz;
  return x;
}
__device__ __forceinline__ void xs_add(XS &a, XS b) {
  if (is_zero(b.m)) return;
  if (is_zero(a.m)) {
    a = b;
    return;
  }
  if (b.e > a.e) {
    a.m = scale2(a.m, a.e - b.e) + b.m;
    a.e = b.e;
  } else {
    a.m += scale2(b.m, b.e - a.e);
  }
}
__device__ __forceinline__ XS xs_norm(XS a) {  // mantissa into [0.5, 1)
  const long long b = __double_as_longlong(a.m);
  if (b == 0ll) return a;
  a.e += (int)(b >> 52) - 1022;
  a.m = __longlong_as_double((b & kFFMantBits) | (1022ll << 52));
  return a;
}

// ------------------------------------------------------------------ float-float
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }  // k in [-126, 127]
__device__ __forceinline__ float2 ff_norm(float s, float e) {  // |s| >= |e| (or s == 0)
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}
__device__ __forceinline__ void ff_add(float2 &a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  a = ff_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float pr = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -pr);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return ff_norm(pr, e);
}
// 1 / a for a > 0: y = rcp(hi), then y + y (1 - a y) (1 - hi y is exact: hi y ~ 1)
__device__ __forceinline__ float2 ff_rcp(float2 a) {
  const float y = __frcp_rn(a.x);
  const float pr = __fmul_rn(a.x, y);
  float e = __fmaf_rn(a.x, y, -pr);
  e = __fmaf_rn(a.y, y, e);
  const float t = __fsub_rn(__fsub_rn(1.0f, pr), e);
  return ff_norm(y, __fmul_rn(y, t));
}
// a nonzero integer: its top 24 bits and the next 24 (the rest is truncated, < 2^-47)
__device__ __forceinline__ float2 ff_u64(unsigned long long s) {
  const int lz = __clzll((long long)s);
  const unsigned long long t = s << lz;
  const int e = 63 - lz;
  const float hi = __uint2float_rn((unsigned)(t >> 40)) * pow2f(e - 23);
  const float lo = __uint2float_rn((unsigned)(t >> 16) & 0xffffffu) * pow2f(e - 47);
  return ff_norm(hi, lo);
}
// an extended-range mantissa m in [0.5, 1)
__device__ __forceinline__ float2 ff_mant(double m) {
  const unsigned long long mant =
      ((unsigned long long)__double_as_longlong(m) & (unsigned long long)kFFMantBits) | (1ull << 52);
  const float2 a = ff_u64(mant);  // m = mant * 2^-53
  return make_float2(a.x * pow2f(-53), a.y * pow2f(-53));
}
// a * 2^k (k <= 0); parts below the normal float range become 0 (they join sums of terms
// of the same scale near 1, far below the rounding)
__device__ __forceinline__ float scale2f(float m, int k) {
  const int b = __float_as_int(m);
  const int ne = ((b >> 23) & 0xff) + k;
  if ((b & 0x7fffffff) == 0 || ne <= 0) return 0.0f;
  return __int_as_float((b & (int)0x807fffff) | (ne << 23));
}
__device__ __forceinline__ float2 ff_scale(float2 a, int k) { return make_float2(scale2f(a.x, k), scale2f(a.y, k)); }
__device__ __forceinline__ double ff_to(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ bool ff_zero(float2 a) { return a.x == 0.0f && a.y == 0.0f; }
__device__ __forceinline__ float2 ff_shfl(float2 a, int src) {
  return make_float2(__shfl_sync(BC_FULL, a.x, src), __shfl_sync(BC_FULL, a.y, src));
}
__device__ __forceinline__ float2 ff_shfl_xor(float2 a, int m) {
  return make_float2(__shfl_xor_sync(BC_FULL, a.x, m), __shfl_xor_sync(BC_FULL, a.y, m));
}

// ------------------------------------------------------------------ paired float-float
// Two float-float values (of two sources) in packed registers: hi = {hi_a, hi_b}, lo =
// {lo_a, lo_b}.  The packed f32x2 additions of sm_100 and later round each half as the scalar
// __fadd_rn / __fsub_rn do (round to nearest even, subnormals kept), so ff2_add computes on
// each half exactly the sequence of ff_add: results are bit for bit those of two ff_add calls,
// in half the instructions.
struct FF2 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ FF2 ff2_pack(float2 a, float2 b) {
  FF2 r;
  r.hi = f2_pack(a.x, b.x);
  r.lo = f2_pack(a.y, b.y);
  return r;
}
__device__ __forceinline__ void ff2_unpack(FF2 r, float2 &a, float2 &b) {
  f2_unpack(r.hi, a.x, b.x);
  f2_unpack(r.lo, a.y, b.y);
}
// ff_add on both halves (Knuth's two-sum of the high parts, then the renormalisation)
__device__ __forceinline__ void ff2_add(FF2 &a, FF2 b) {
  const unsigned long long s = f2_add(a.hi, b.hi);
  const unsigned long long bb = f2_sub(s, a.hi);
  const unsigned long long e = f2_add(f2_sub(a.hi, f2_sub(s, bb)), f2_sub(b.hi, bb));
  const unsigned long long t = f2_add(e, f2_add(a.lo, b.lo));
  const unsigned long long hi = f2_add(s, t);
  a.lo = f2_sub(t, f2_sub(hi, s));
  a.hi = hi;
}

}  // namespace bcl

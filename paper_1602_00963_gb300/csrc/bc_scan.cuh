// Device exclusive prefix sum of int32 arrays (three passes: per-block scan, scan of
// block totals, add-back).  Product code only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace bcl {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

inline size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)(nb + 1) * 4 + 64;
}

static __global__ void k_scan_tiles(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sum) {
  __shared__ int32_t s[kScanThreads];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t k = base + i;
    v[i] = k < n ? in[k] : 0;
    int32_t t = v[i];
    v[i] = run;
    run += t;
  }
  s[threadIdx.x] = run;
  __syncthreads();
  for (int d = 1; d < kScanThreads; d <<= 1) {
    int32_t y = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += y;
    __syncthreads();
  }
  int32_t off = threadIdx.x ? s[threadIdx.x - 1] : 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t k = base + i;
    if (k < n) out[k] = v[i] + off;
  }
  if (threadIdx.x == kScanThreads - 1) tile_sum[blockIdx.x] = s[threadIdx.x];
}

static __global__ void k_scan_sums(int32_t *tile_sum, int64_t nb) {
  // single block: sequential carry over chunks of blockDim.x
  __shared__ int32_t s[kScanThreads];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    int64_t k = c0 + threadIdx.x;
    int32_t x = k < nb ? tile_sum[k] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int d = 1; d < kScanThreads; d <<= 1) {
      int32_t y = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (k < nb) tile_sum[k] = carry + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += s[kScanThreads - 1];
    __syncthreads();
  }
}

static __global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_sum) {
  int64_t k = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int32_t add = tile_sum[blockIdx.x];
  for (int i = 0; i < kScanItems; i++, k += kScanThreads)
    if (k < n) out[k] += add;
}

inline cudaError_t scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, void *scratch,
                                      cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  int32_t *ts = (int32_t *)scratch;
  k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, ts);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(ts, nb);
  k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, ts);
  return cudaGetLastError();
}

}  // namespace bcl

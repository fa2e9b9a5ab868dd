// Device-side helpers shared by the library's kernels (product code only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define BC_FULL 0xffffffffu

// Device error codes written to the control block (mapped to bc_status on the host).
enum {
  BCD_OK = 0,
  BCD_TIMEOUT = 1,   // a bounded spin gave up
  BCD_CAPACITY = 2,  // a device buffer was too small (host retries with more room)
  BCD_BADARG = 3,
};

// Grid-wide barrier with a bounded spin.  All CTAs of a cooperative launch call it the
// same number of times.  Returns false (for every thread of the CTA) if this CTA gave
// up waiting or another CTA reported an error; callers then leave the kernel.
struct GridSync {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
  return *(const volatile int *)p;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_sync(GridSync *gs, uint64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned g = ld_acquire_u32(&gs->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&gs->count, 1u);
    if (arrived == gridDim.x - 1) {
      gs->count = 0;
      __threadfence();
      st_release_u32(&gs->gen, g + 1);
    } else {
      uint64_t t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&gs->gen) == g) {
        if ((spins++ & 63u) == 0 && globaltimer_ns() - t0 >= limit_ns) {
          atomicCAS(&gs->err, 0, BCD_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    if (ld_volatile_i32(&gs->err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive prefix sum over the warp (all 32 lanes participate).
__device__ __forceinline__ int warp_excl_scan(int x, int *total) {
  int incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(BC_FULL, incl, d);
    if ((int)lane_id() >= d) incl += y;
  }
  *total = __shfl_sync(BC_FULL, incl, 31);
  return incl - x;
}

// Largest j in [0, 32) with key_j <= e, where lane j holds key_j, keys are
// non-decreasing and key_0 <= e.
__device__ __forceinline__ int warp_owner(int key, int e) {
  int j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    int kc = __shfl_sync(BC_FULL, key, j + step);
    if (kc <= e) j += step;
  }
  return j;
}

__device__ __forceinline__ bool test_bit(const uint32_t *bits, int v) {
  return (bits[v >> 5] >> (v & 31)) & 1u;
}
__device__ __forceinline__ void set_bit_atomic(uint32_t *bits, int v) {
  atomicOr(bits + (v >> 5), 1u << (v & 31));
}
__device__ __forceinline__ void clear_bit_atomic(uint32_t *bits, int v) {
  atomicAnd(bits + (v >> 5), ~(1u << (v & 31)));
}

// Packed append counter: high 32 bits count queue entries, low 32 bits count their
// adjacency entries, so one 64-bit atomicAdd reserves queue slots and edge offsets in
// the same order and the edge offsets form an exclusive prefix sum over the queue.
__device__ __forceinline__ unsigned long long pack_qe(unsigned cnt, unsigned edges) {
  return ((unsigned long long)cnt << 32) | (unsigned long long)edges;
}

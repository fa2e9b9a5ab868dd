// bc_sources_noalloc: the per-source BC computation for callers that cannot allocate
// device memory.  Its working storage is one file-scope device array, so the call makes
// no cudaMalloc / cudaFree and allocates nothing through any library.
//
// Who needs it: code that runs while device allocation is off limits — inside a region
// whose memory is owned by another allocator (a framework's caching allocator or a fixed
// memory pool that must not fragment), in latency-critical loops where cudaMalloc's
// implicit device synchronisation is not acceptable, or in processes started with a
// hard device-memory quota.  They pass inputs and outputs they already own; everything
// else lives in the static scratch below.
//
// Limits and rules:
//   * n <= BC_NOALLOC_MAX_N; larger graphs are rejected with BC_EINVAL, and so are an odd
//     nnz and any source id outside [0, n) (checked on the device before the traversal;
//     the CSR itself is not validated).
//   * The scratch (about 4.2 MB) is part of the library image: every GPU on which the
//     library is loaded holds it until the process exits.
//   * All calls of a process share the one array.  The entry point clears what must start
//     cleared at the beginning of every call and holds a lock until the call's work is
//     complete, so one call runs at a time.  Each process gets its own copy of the array
//     (a module global lives in the process's own CUDA context).
//   * The CUDA runtime places the array on a device when it loads the library's device
//     code there (with lazy loading: at the latest during the first call on that device);
//     the calls themselves allocate nothing.
//   * The first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call before any
//     stream capture.
//   * A call waits for its own work: it synchronises the given stream (after the source
//     check and after the traversal) before it returns.
#include <cstring>
#include <mutex>

#include "bc_internal.h"

namespace bcl {
namespace {

constexpr int kMaxN = BC_NOALLOC_MAX_N;
constexpr size_t kN2 = (size_t)kMaxN + 2;
constexpr size_t kNW = (size_t)kMaxN / 32 + 1;

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the workspace arrays inside the scratch
constexpr size_t o_depth = 0;
constexpr size_t o_Q = o_depth + al256(kN2 * 4);
constexpr size_t o_CD = o_Q + al256(kN2 * 4);
constexpr size_t o_loff = o_CD + al256(kN2 * 4);
constexpr size_t o_leoff = o_loff + al256(kN2 * 4);
constexpr size_t o_sig = o_leoff + al256(kN2 * 4);
constexpr size_t o_acc = o_sig + al256(kN2 * 8);
constexpr size_t o_r = o_acc + al256(kN2 * 16);
constexpr size_t o_xm = o_r + al256(kN2 * 8);
constexpr size_t o_xe = o_xm + al256(kN2 * 8);
constexpr size_t o_ovf = o_xe + al256(kN2 * 4);
constexpr size_t o_vis = o_ovf + al256(kNW * 4);
constexpr size_t o_front = o_vis + al256(kNW * 4);
constexpr size_t o_ctl = o_front + al256(kNW * 4);
constexpr size_t o_chk = o_ctl + al256(sizeof(PlainCtl));  // source-range check word
constexpr size_t kScratchBytes = o_chk + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Clear the parts of the workspace that the kernel expects cleared: depth = -1; sigma,
// bitmaps, successor sums, exponents and the control block = 0.
__global__ void k_noalloc_clear(unsigned char *base, int n) {
  const size_t N = (size_t)n + 2, NW = (size_t)n / 32 + 1;
  int32_t *depth = (int32_t *)(base + o_depth);
  unsigned long long *sig = (unsigned long long *)(base + o_sig);
  unsigned long long *acc = (unsigned long long *)(base + o_acc);
  int32_t *xe = (int32_t *)(base + o_xe);
  uint32_t *ovf = (uint32_t *)(base + o_ovf), *vis = (uint32_t *)(base + o_vis),
           *front = (uint32_t *)(base + o_front);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    depth[i] = -1;
    sig[i] = 0ull;
    acc[2 * i] = 0ull;
    acc[2 * i + 1] = 0ull;
    xe[i] = 0;
    if (i < NW) {
      ovf[i] = 0u;
      vis[i] = 0u;
      front[i] = 0u;
    }
  }
  uint32_t *ctl = (uint32_t *)(base + o_ctl);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sizeof(PlainCtl) / 4;
       i += (size_t)gridDim.x * blockDim.x)
    ctl[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *(int *)(base + o_chk) = 0;
}

// Sets the check word when a source id lies outside [0, n): the per-source kernel indexes
// its state arrays with the ids, so none may run past them.
__global__ void k_noalloc_check(const int32_t *src, int32_t k, int32_t n, unsigned char *base) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    if (src[i] < 0 || src[i] >= n) atomicOr((int *)(base + o_chk), 1);
}

std::mutex g_mu;
unsigned char *g_addr[128];  // device address of g_scratch per device (set up once)

}  // namespace
}  // namespace bcl

using namespace bcl;

extern "C" bc_status bc_sources_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                        int64_t nnz, const int32_t *src, int32_t k, double *bc_out,
                                        void *cuda_stream) {
  if (n <= 0 || n > kMaxN)
    return fail(BC_EINVAL, "bc_sources_noalloc: n must be in [1, " + std::to_string(kMaxN) +
                               "] (the static scratch is sized for that many vertices)");
  if (nnz < 0 || nnz >= ((int64_t)1 << 31))
    return fail(BC_EINVAL, "bc_sources_noalloc: nnz must be in [0, 2^31)");
  if (nnz % 2) return fail(BC_EINVAL, "bc_sources_noalloc: a symmetric CSR has an even nnz");
  if (!row_ptr || (nnz > 0 && !col_idx) || !bc_out || k < 0 || (k > 0 && !src))
    return fail(BC_EINVAL, "bc_sources_noalloc: NULL argument or k < 0");
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  BC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(BC_EINVAL, "bc_sources_noalloc: device index out of range");
  if (!g_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = (unsigned char *)ptr;
  }
  unsigned char *base = g_addr[dev];
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int sms = 0;
  BC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  k_noalloc_clear<<<sms * 4, 256, 0, st>>>(base, n);
  BC_CUDA_TRY(cudaGetLastError());
  if (k > 0) {
    k_noalloc_check<<<sms, 256, 0, st>>>(src, k, n, base);
    BC_CUDA_TRY(cudaGetLastError());
    int bad = 0;
    BC_CUDA_TRY(cudaMemcpyAsync(&bad, base + o_chk, sizeof(int), cudaMemcpyDeviceToHost, st));
    BC_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return fail(BC_EINVAL, "bc_sources_noalloc: source id out of range [0, n)");
  }
  BC_CUDA_TRY(cudaMemsetAsync(bc_out, 0, (size_t)n * sizeof(double), st));
  PlainWS ws;
  ws.n = n;
  ws.depth = (int32_t *)(base + o_depth);
  ws.Q = (int32_t *)(base + o_Q);
  ws.CD = (int32_t *)(base + o_CD);
  ws.lvl_off = (int32_t *)(base + o_loff);
  ws.lvl_eoff = (int32_t *)(base + o_leoff);
  ws.sig = (unsigned long long *)(base + o_sig);
  ws.acc = (unsigned long long *)(base + o_acc);
  ws.r = (double *)(base + o_r);
  ws.xm = (double *)(base + o_xm);
  ws.xe = (int32_t *)(base + o_xe);
  ws.ovf = (uint32_t *)(base + o_ovf);
  ws.vis = (uint32_t *)(base + o_vis);
  ws.front = (uint32_t *)(base + o_front);
  ws.ctl = (PlainCtl *)(base + o_ctl);
  DeviceGraph g;
  g.n = n;
  g.nnz = nnz;
  g.rp = (int32_t *)row_ptr;
  g.ci = (int32_t *)col_idx;
  PlainArgs a;
  memset(&a, 0, sizeof(a));
  a.g = &g;
  a.src = src;
  a.nsrc = k;
  a.bc = bc_out;
  a.max_degree = n;  // any degree is below n: a valid bound for the no-overflow test
  a.alpha = 0.5f;
  a.beta = 24.f;
  int derr = 0;
  bc_status s = plain_run_view(ws, a, sms, 20ull * 1000 * 1000 * 1000, st, &derr);
  if (s) return s;
  if (derr == BCD_TIMEOUT) return fail(BC_ETIMEDOUT, "bc_sources_noalloc: a grid barrier wait passed its limit");
  if (derr) return fail(BC_ECUDA, "bc_sources_noalloc: device error " + std::to_string(derr));
  return BC_OK;
}

// svd_noalloc.cu -- pylom_svd_small_noalloc: the small Jacobi SVD of
// pylom_svd_small with its scratch held in a fixed device array of this
// library instead of a caller-provided workspace.
//
// Who needs this: a caller that cannot hand the library any device memory of
// its own -- for example a Fortran or C flow solver that owns every device
// buffer through its own allocator and calls the SVD between time steps, or a
// loop that must not allocate once it is running (fixed memory budget, no
// allocator reachable from that code).  Such a caller passes only its inputs
// and outputs; the scratch (header + Jacobi working columns, ~1 MiB) is part
// of the loaded library.
//
// Limits and rules:
//   - M <= kNoAllocMaxM (256); larger M is rejected with PYLOM_ERR_SHAPE.
//   - The binary64 sweeps start from R^T without the binary32
//     preconditioning (whose scratch the array does not hold): the same
//     SVD, in more sweeps than pylom_svd_small takes at M = 256.
//   - The array is shared by every call in the process on that device and
//     keeps the last call's contents.  Each call clears the parts that must
//     start at zero (status word, grid-barrier counters, rotation counts)
//     with a memset on its stream before launching.  Two calls that may run
//     at the same time on the GPU (different streams, no ordering) race on
//     the array and give wrong results: order them on one stream.
//   - The array's device address is looked up once per device with
//     cudaGetSymbolAddress, the first time this entry point runs with that
//     device current.  That first call should come before any stream capture.
//     The address is kept for the life of the process: after a
//     cudaDeviceReset the module (and the array) is loaded again elsewhere,
//     so a process that resets a device must not call this entry point
//     again on it (reload the library instead).
//   - Every M up to the limit is checked at run time against the layout the
//     Jacobi kernels carve from the array (header + padded working columns),
//     so a larger layout is refused rather than overrun.
//   - Nothing here calls cudaMalloc, cudaFree or an allocating library.
#include <mutex>

#include "kernels.h"

namespace {

constexpr int64_t kNoAllocMaxM = 256;
constexpr size_t kNoAllocBytes = sizeof(pylom::WsHeader) + 2 * sizeof(double) * kNoAllocMaxM * kNoAllocMaxM;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_svd_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Copies the device-side status and sweep count to the caller's info[2].
__global__ void noalloc_info_kernel(const pylom::WsHeader* h, int* info) {
  info[0] = h->status;
  info[1] = h->sweeps;
}

}  // namespace

extern "C" pylom_status pylom_svd_small_noalloc(const double* R, int64_t M, int64_t ldr, double* U,
                                                int64_t ldu, double* S, double* VT, int64_t ldvt,
                                                int max_sweeps, int* info, void* stream) {
  using namespace pylom;
  set_error_message("");
  if (!R || !U || !S || !VT) {
    set_error_message("pylom_svd_small_noalloc: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (M < 1 || M > kNoAllocMaxM) {
    set_error_message("pylom_svd_small_noalloc: M = %lld is outside [1, %lld], the size its fixed "
                      "scratch holds; use pylom_svd_small with a workspace",
                      (long long)M, (long long)kNoAllocMaxM);
    return PYLOM_ERR_SHAPE;
  }
  if (ldr < M || ldu < M || ldvt < M) {
    set_error_message("pylom_svd_small_noalloc: leading dimension too small");
    return PYLOM_ERR_ARG;
  }
  if (max_sweeps < 1 || max_sweeps > kMaxSweeps) {
    set_error_message("pylom_svd_small_noalloc: max_sweeps must be in [1, %d]", kMaxSweeps);
    return PYLOM_ERR_ARG;
  }
  // the layout the Jacobi kernels carve (padded columns, 256-byte aligned
  // arrays) must fit the fixed array for this M
  if (sizeof(WsHeader) + svd_state_bytes(M, false) > kNoAllocBytes) {
    set_error_message("pylom_svd_small_noalloc: M = %lld needs %zu bytes of scratch, more than the %zu "
                      "the fixed array holds; use pylom_svd_small with a workspace",
                      (long long)M, sizeof(WsHeader) + svd_state_bytes(M, false), kNoAllocBytes);
    return PYLOM_ERR_SHAPE;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_small_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_message("pylom_svd_small_noalloc: device index %d is beyond the %d devices this entry "
                      "point keeps scratch addresses for", dev, kMaxDevices);
    return PYLOM_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_svd_scratch);
      if (e != cudaSuccess || !p) {
        set_error_message("pylom_svd_small_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return PYLOM_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  SvdState ss;
  ss.hdr = (WsHeader*)base;
  svd_state_carve(ss, (char*)base + sizeof(WsHeader), M, false);
  e = cudaMemsetAsync(ss.hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_small_noalloc: header clear: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  e = launch_svd_fp64(ss, R, ldr, U, ldu, S, VT, ldvt, max_sweeps, 0.0, M, st);
  if (e == cudaSuccess && info) {
    noalloc_info_kernel<<<1, 1, 0, st>>>(ss.hdr, info);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_small_noalloc: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

// waits.cu -- pylom_wait_selftest: runs the library's bounded device waits
// into their time limit on purpose, so that failure detection can be tested
// without hanging or faulting the GPU (no counterpart in the paper).
//
// The waits under test are the ones every cooperative kernel of the library
// uses: grid_barrier (common.cuh; the Jacobi sweeps, the cooperative tree,
// the batched SVDs) and mbar_wait (tc05.cuh; the tcgen05 commits of the
// mixed-precision leaves).  Each polls the GPU's global timer and gives up
// after its limit, records PYLOM_ERR_TIMEOUT in the workspace header and
// returns; a grid barrier entered after a time-out returns at once.
#include "kernels.h"
#include "tc05.cuh"

namespace {

constexpr int kSelftestThreads = 128;
constexpr int kSelftestMaxBlocks = 1024;

// kind 0: every block arrives at a grid barrier that expects one arrival
// more than the grid has, so nobody releases it; then at a second barrier,
// which must return at once because the first one timed out.
// kind 1: one mbarrier that nothing arrives on.
__global__ void __launch_bounds__(kSelftestThreads) wait_selftest_kernel(pylom::WsHeader* h, int kind,
                                                                         unsigned long long limit_ns,
                                                                         unsigned* gave_up) {
  using namespace pylom;
  if (kind == 0) {
    const bool first = grid_barrier(h, gridDim.x + 1, limit_ns);
    const bool second = grid_barrier(h, gridDim.x, limit_ns);
    if (threadIdx.x == 0 && !first && !second && gave_up) atomicAdd(gave_up, 1u);
    return;
  }
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) tc05::mbar_init(&mbar, 1);
  __syncthreads();
  const bool done = tc05::mbar_wait(&mbar, 0, limit_ns);
  if (!done && threadIdx.x == 0) {
    raise_status(h, PYLOM_ERR_TIMEOUT);
    if (gave_up) atomicAdd(gave_up, 1u);
  }
  __syncthreads();
}

}  // namespace

extern "C" size_t pylom_wait_selftest_workspace_size(void) { return sizeof(pylom::WsHeader); }

extern "C" pylom_status pylom_wait_selftest(int kind, int blocks, double limit_ms, unsigned* gave_up, void* ws,
                                            size_t ws_bytes, void* stream) {
  using namespace pylom;
  set_error_message("");
  if (kind != 0 && kind != 1) {
    set_error_message("pylom_wait_selftest: kind must be 0 (grid barrier) or 1 (mbarrier)");
    return PYLOM_ERR_ARG;
  }
  if (kind == 1) blocks = 1;
  if (blocks < 1 || blocks > kSelftestMaxBlocks) {
    set_error_message("pylom_wait_selftest: blocks must be in [1, %d]", kSelftestMaxBlocks);
    return PYLOM_ERR_ARG;
  }
  if (!(limit_ms > 0.0) || limit_ms > 2000.0) {
    set_error_message("pylom_wait_selftest: limit_ms must be in (0, 2000]");
    return PYLOM_ERR_ARG;
  }
  if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < sizeof(WsHeader)) {
    set_error_message("pylom_wait_selftest: workspace needs %zu bytes, 256-byte aligned", sizeof(WsHeader));
    return PYLOM_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  WsHeader* h = (WsHeader*)ws;
  cudaError_t e = cudaMemsetAsync(h, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess && gave_up) e = cudaMemsetAsync(gave_up, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    const unsigned long long limit_ns = (unsigned long long)(limit_ms * 1e6);
    wait_selftest_kernel<<<(unsigned)blocks, kSelftestThreads, 0, st>>>(h, kind, limit_ns, gave_up);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error_message("pylom_wait_selftest: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

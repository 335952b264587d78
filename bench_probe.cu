// bench_probe.cu -- arithmetic throughput probes of the benchmark (not part
// of the POD library).  They give the measured denominators of the binary64
// and binary32 rooflines that bench.py reports: the pool's measured-peaks
// file holds HBM and bf16 figures only.
//
// Each thread runs kChains independent dependency chains.  Every chain
// starts from its own accumulator value and takes its own operands (they
// differ by chain index and by lane), and all chains are summed into the
// stored result, so no chain can be merged with another or removed; the
// MMA chains are inline asm volatile as well.  32 warps per SM (4 blocks of
// 256 threads) with 8 chains each keep the pipes issue-bound.
//
// Built by paper_2405_15529_gb300/_build.build_probe() into bench_probe.so;
// loaded by bench.py through ctypes.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kIters = 4096;
constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kMaxSms = 1024;

// D(8x8) += A(8x4) B(4x8) in binary64 on the tensor pipe
__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kThreads) dmma_kernel(double* out, double a, double b) {
  const int lane = threadIdx.x & 31;
  double c0[kChains], c1[kChains], av[kChains], bv[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) {
    c0[q] = 1e-3 * (q + 1) + 1e-7 * lane;
    c1[q] = 2e-3 * (q + 1) - 1e-7 * lane;
    av[q] = a + 1e-3 * q + 1e-6 * lane;
    bv[q] = b * (1.0 + 0.125 * q) + 1e-9 * lane;
  }
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) dmma884(c0[q], c1[q], av[q], bv[q]);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += c0[q] + c1[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_kernel(double* out, double a, double b) {
  double x[kChains], av[kChains], bv[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) {
    x[q] = threadIdx.x + 0.5 * q;
    av[q] = a - 1e-4 * q;
    bv[q] = b + 1e-5 * q;
  }
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], av[q], bv[q]);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) ffma_kernel(double* out, float a, float b) {
  float x[kChains], av[kChains], bv[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) {
    x[q] = threadIdx.x + 0.5f * q;
    av[q] = a - 1e-4f * q;
    bv[q] = b + 1e-5f * q;
  }
  // unrolled so that loop control takes a small share of the issue slots
  // (binary32 FMAs issue every cycle, unlike the binary64 probes)
#pragma unroll 8
  for (int it = 0; it < kIters * 4; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fmaf(x[q], av[q], bv[q]);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Bytes of device scratch the probes store their results to.
extern "C" size_t bench_probe_scratch_bytes(void) {
  return sizeof(double) * (size_t)kMaxSms * kBlocksPerSm * kThreads;
}

// kind 0: binary64 mma.sync.m8n8k4; 1: binary64 FMA; 2: binary32 FMA.
// Runs the loop over every SM of the current device on `stream` three times
// and writes the best of the last two, in TFLOP/s, to *tflops (host).
// Returns 0 on success, 1 on a bad argument, 2 on a CUDA error.
extern "C" int bench_probe_peak(int kind, void* scratch, double* tflops, void* stream) {
  if (!scratch || !tflops || kind < 0 || kind > 2) return 1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  if (nsm > kMaxSms) nsm = kMaxSms;
  const int blocks = nsm * kBlocksPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 2;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return 2;
  }
  double best = 0.0;
  int rc = 0;
  for (int rep = 0; rep < 3 && rc == 0; ++rep) {
    cudaEventRecord(e0, st);
    if (kind == 0)
      dmma_kernel<<<blocks, kThreads, 0, st>>>((double*)scratch, 0.999, 1e-3);
    else if (kind == 1)
      dfma_kernel<<<blocks, kThreads, 0, st>>>((double*)scratch, 0.999, 1e-3);
    else
      ffma_kernel<<<blocks, kThreads, 0, st>>>((double*)scratch, 0.999f, 1e-3f);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = 2;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double threads = (double)blocks * kThreads;
    // an m8n8k4 MMA is 2 * 8 * 8 * 4 flops per warp; an FMA 2 flops per thread
    const double per_chain_step = (kind == 0) ? 2.0 * 8 * 8 * 4 / 32.0 : 2.0;
    const double flops = per_chain_step * kChains * (double)kIters * (kind == 2 ? 4.0 : 1.0) * threads;
    const double tf = flops / (ms * 1e-3) / 1e12;
    if (rep > 0 && tf > best) best = tf;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == 0 && cudaGetLastError() != cudaSuccess) rc = 2;
  if (rc == 0) *tflops = best;
  return rc;
}

// probe.cu -- FP64 tensor-pipe and FP64 FMA throughput probes (see
// include/pylom_probe.h).  Each thread runs kChains independent chains so
// the measured rate is issue-bound, not latency-bound.
#include "../../include/pylom_probe.h"
#include "common.cuh"

namespace {

constexpr int kIters = 4096;
constexpr int kProbeThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kMaxSms = 1024;

__global__ void __launch_bounds__(kProbeThreads) probe_dmma_kernel(double* out, double a, double b) {
  double c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) c[q] = 0.0;
  const double av = a + threadIdx.x;
  for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pylom::dmma884(c[2 * q], c[2 * q + 1], av, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += c[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(double* out, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x + q;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(double* out, float a, float b) {
  float x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x + q;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fmaf(x[q], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" size_t pylom_probe_scratch_bytes(void) {
  return sizeof(double) * (size_t)kMaxSms * kBlocksPerSm * kProbeThreads;
}

extern "C" pylom_status pylom_probe_fp64_peak(int kind, void* scratch, double* tflops, void* stream) {
  if (!scratch || !tflops || kind < 0 || kind > 2) return PYLOM_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PYLOM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PYLOM_ERR_CUDA;
  if (nsm > kMaxSms) nsm = kMaxSms;
  const int blocks = nsm * kBlocksPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PYLOM_ERR_CUDA;
  double best = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    if (kind == 0)
      probe_dmma_kernel<<<blocks, kProbeThreads, 0, st>>>((double*)scratch, 0.999, 1e-3);
    else if (kind == 1)
      probe_dfma_kernel<<<blocks, kProbeThreads, 0, st>>>((double*)scratch, 0.999, 1e-3);
    else
      probe_ffma_kernel<<<blocks, kProbeThreads, 0, st>>>((double*)scratch, 0.999f, 1e-3f);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return PYLOM_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double threads = (double)blocks * kProbeThreads;
    const double flops = (kind == 0) ? 2.0 * 8 * 8 * 4 * 4.0 * (kIters / 4) * (threads / 32.0)
                                     : 2.0 * 8 * kIters * threads;   // FMA kinds: 8 chains x kIters
    const double tf = flops / (ms * 1e-3) / 1e12;
    if (rep > 0 && tf > best) best = tf;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return PYLOM_ERR_CUDA;
  *tflops = best;
  return PYLOM_OK;
}

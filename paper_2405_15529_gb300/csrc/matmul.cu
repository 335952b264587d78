// matmul.cu -- local product of Alg. 4 (matmul_paral of pyLOM, arXiv
// 2405.15529): C = op(A) B in binary64 on the FP64 tensor pipe
// (mma.sync m8n8k4).  The reduction dimension k is split into Z slices whose
// partial products go to the workspace and are summed in slice order, so
// the result does not depend on scheduling.  Alg. 4's all_reduce across
// processes has no counterpart on one device.
#include "kernels.h"

namespace pylom {

constexpr int kMmThreads = 128;   // 4 warps; block tile 32 x 32, warp tile 32 x 8

static int64_t matmul_slices(int64_t m, int64_t n, int64_t k) {
  const int64_t tiles = ((m + 31) / 32) * ((n + 31) / 32);
  int64_t z = 1;
  while (z < 64 && tiles * z < 1024 && k / (z * 2) >= 256) z *= 2;
  return z;
}

size_t matmul_ws_bytes(int64_t m, int64_t n, int64_t k) {
  const int64_t z = matmul_slices(m, n, k);
  return z > 1 ? align256(sizeof(double) * (size_t)z * m * n) : 0;
}

__global__ void __launch_bounds__(kMmThreads) matmul_kernel(int transA, const double* A,
                                                           const double* B, double* out,
                                                           int64_t ldo, int64_t m, int64_t n,
                                                           int64_t k, int64_t lda, int64_t ldb,
                                                           int64_t z, int64_t zstride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int64_t j0 = (int64_t)blockIdx.y * 32 + warp * 8;
  const int64_t nsteps = (k + 3) / 4;
  const int64_t sb = (nsteps * blockIdx.z) / z, se = (nsteps * (blockIdx.z + 1)) / z;
  double acc[4][2];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) acc[mt][0] = acc[mt][1] = 0.0;
  const int64_t jb = j0 + g;
  for (int64_t stp = sb; stp < se; ++stp) {
    const int64_t kk = stp * 4 + t;
    const bool kok = kk < k;
    const double b = (kok && jb < n) ? B[kk + jb * ldb] : 0.0;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const int64_t i = i0 + mt * 8 + g;
      double a = 0.0;
      if (kok && i < m) a = transA ? A[kk + i * lda] : A[i + kk * lda];
      dmma884(acc[mt][0], acc[mt][1], a, b);
    }
  }
  double* o = out + (int64_t)blockIdx.z * zstride;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    const int64_t i = i0 + mt * 8 + g;
    const int64_t j = j0 + 2 * t;
    if (i < m && j < n) o[i + j * ldo] = acc[mt][0];
    if (i < m && j + 1 < n) o[i + (j + 1) * ldo] = acc[mt][1];
  }
}

__global__ void matmul_reduce_kernel(const double* part, double* C, int64_t ldc, int64_t m, int64_t n,
                                     int64_t z) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t q = 0; q < z; ++q) s += part[q * m * n + idx];
    C[(idx % m) + (idx / m) * ldc] = s;
  }
}

cudaError_t launch_matmul_fp64(int transA, const double* A, const double* B, double* C, int64_t m,
                               int64_t n, int64_t k, int64_t lda, int64_t ldb, int64_t ldc,
                               double* ws, cudaStream_t st) {
  const int64_t z = matmul_slices(m, n, k);
  dim3 grid((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)z);
  if (z == 1) {
    matmul_kernel<<<grid, kMmThreads, 0, st>>>(transA, A, B, C, ldc, m, n, k, lda, ldb, 1, 0);
    return cudaGetLastError();
  }
  matmul_kernel<<<grid, kMmThreads, 0, st>>>(transA, A, B, ws, m, m, n, k, lda, ldb, z, m * n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  matmul_reduce_kernel<<<256, 256, 0, st>>>(ws, C, ldc, m, n, z);
  return cudaGetLastError();
}

}  // namespace pylom

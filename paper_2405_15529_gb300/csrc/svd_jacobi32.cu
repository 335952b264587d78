// svd_jacobi32.cu -- single-precision preconditioning of the small SVD
// (Eq. svdqr2 of pyLOM, arXiv 2405.15529) for large M.
//
// One-sided Jacobi in binary64 costs about 5.5 M^3 FP64 instructions per
// sweep, and binary64 runs at a small fraction of the binary32 rate on this
// part, so at M in the thousands the sweeps, not the data, bound the small
// SVD.  Here the sweeps that do most of the rotating run in binary32:
//   1. block one-sided Jacobi on A32 = fl32(R^T): the columns are grouped in
//      blocks of kJB, pairs of blocks (2 kJB columns) are orthogonalised in
//      shared memory by inner Jacobi sweeps (one warp per column pair), the
//      accumulated 2 kJB x 2 kJB rotation is applied to V32, and the blocks
//      follow a round-robin order with one grid barrier per step;
//   2. V = V32 in binary64, made orthogonal to working precision by two
//      Newton-Schulz steps V <- V (3 I - V^T V) / 2 (the error squares each
//      step: about 1e-6, 1e-12, rounding);
//   3. A = R^T V in binary64.
// The binary64 one-sided Jacobi of svd_jacobi.cu then starts from (A, V):
// the columns of A are already orthogonal to about the single-precision
// tolerance, and its quadratic convergence finishes in a few sweeps.  The
// result is the binary64 SVD of R (R^T V_final = A_final with orthogonal
// columns, V_final orthogonal to working precision); only the number of
// binary64 sweeps changes.
#include "kernels.h"

namespace pylom {

constexpr int kJB = 8;                 // columns per block; a pair of blocks = 16 columns, one per warp pair
constexpr int kJ32Threads = 32 * kJB;  // one warp per column pair of a round
// inner sweeps per block pair and step: one (a block-cyclic sweep); 2 and 3
// converged in the same number of outer and binary64 sweeps but took longer
// (M = 256: 12.9 / 15.2 / 16.9 ms; M = 1808: 1.28 / 1.35 / 1.48 s)
constexpr int kJ32Inner = 1;
constexpr int kJ32MaxSweeps = 40;

__global__ void jacobi32_init_kernel(SvdState s, const double* R, int64_t ldr) {
  const int64_t M = s.M, Mb = s.Mb;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * Mb; idx += stride) {
    const int64_t i = idx % M, j = idx / M;
    s.A32[idx] = (j < M) ? (float)R[j + i * ldr] : 0.f;   // A32 = R^T (zero padding columns)
  }
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < Mb * Mb; idx += stride)
    s.V32[idx] = (idx % Mb == idx / Mb) ? 1.f : 0.f;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Cooperative launch; dynamic shared memory: 2 kJB columns of M floats plus
// the 2 kJB x 2 kJB accumulated rotation.
__global__ void __launch_bounds__(kJ32Threads) jacobi32_block_kernel(SvdState s) {
  extern __shared__ float jsm[];
  constexpr int W = 2 * kJB;
  const int64_t M = s.M, Mb = s.Mb;
  float* sA = jsm;                // [W][M]
  float* sJ = sA + W * M;         // [W][W], column-major
  __shared__ unsigned s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nblk = Mb / kJB, npairs = nblk / 2;
  const float tol = 8.f * sqrtf((float)M) * 5.9604645e-8f;   // a few times the rounding level of a dot
  for (int sweep = 0; sweep < kJ32MaxSweeps; ++sweep) {
    unsigned local_rot = 0;
    for (int64_t step = 0; step < nblk - 1; ++step) {
      for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const int64_t p = (pr == 0) ? 0 : ((pr - 1 + step) % (nblk - 1)) + 1;
        const int64_t q = ((nblk - 2 - pr + step) % (nblk - 1)) + 1;
        const int64_t bI = p < q ? p : q, bJ = p < q ? q : p;
        // the 16 columns: block bI then block bJ
        for (int64_t idx = tid; idx < (int64_t)W * M; idx += kJ32Threads) {
          const int l = (int)(idx / M);
          const int64_t r = idx - (int64_t)l * M;
          const int64_t col = (l < kJB) ? bI * kJB + l : bJ * kJB + (l - kJB);
          sA[idx] = s.A32[r + col * M];
        }
        for (int idx = tid; idx < W * W; idx += kJ32Threads) sJ[idx] = (idx % W == idx / W) ? 1.f : 0.f;
        __syncthreads();
        for (int inner = 0; inner < kJ32Inner; ++inner) {
          if (tid == 0) s_rot = 0;
          __syncthreads();
          // round-robin over the W local columns: W - 1 rounds of kJB disjoint pairs
          for (int round = 0; round < W - 1; ++round) {
            const int a = (warp == 0) ? 0 : ((warp - 1 + round) % (W - 1)) + 1;
            const int b = ((W - 2 - warp + round) % (W - 1)) + 1;
            const int i = a < b ? a : b, j = a < b ? b : a;
            float* ai = sA + (int64_t)i * M;
            float* aj = sA + (int64_t)j * M;
            float al = 0.f, be = 0.f, ga = 0.f;
            for (int64_t r = lane; r < M; r += 32) {
              const float x = ai[r], y = aj[r];
              al = fmaf(x, x, al);
              be = fmaf(y, y, be);
              ga = fmaf(x, y, ga);
            }
            al = warp_sum_f(al);
            be = warp_sum_f(be);
            ga = warp_sum_f(ga);
            if (ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
              const float zeta = (be - al) / (2.f * ga);
              const float t = ((zeta >= 0.f) ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
              const float c = 1.f / sqrtf(1.f + t * t);
              const float sn = c * t;
              for (int64_t r = lane; r < M; r += 32) {
                const float x = ai[r], y = aj[r];
                ai[r] = c * x - sn * y;
                aj[r] = sn * x + c * y;
              }
              if (lane < W) {
                const float x = sJ[lane + i * W], y = sJ[lane + j * W];
                sJ[lane + i * W] = c * x - sn * y;
                sJ[lane + j * W] = sn * x + c * y;
              }
              if (lane == 0) atomicAdd(&s_rot, 1u);
            }
            __syncthreads();
          }
          const unsigned rr = s_rot;
          if (inner == 0) local_rot += rr;
          __syncthreads();
          if (rr == 0) break;
        }
        // write the columns back; V32[:, cols] <- V32[:, cols] J
        for (int64_t idx = tid; idx < (int64_t)W * M; idx += kJ32Threads) {
          const int l = (int)(idx / M);
          const int64_t r = idx - (int64_t)l * M;
          const int64_t col = (l < kJB) ? bI * kJB + l : bJ * kJB + (l - kJB);
          s.A32[r + col * M] = sA[idx];
        }
        float* VI = s.V32 + bI * kJB * Mb;
        float* VJ = s.V32 + bJ * kJB * Mb;
        for (int64_t r = tid; r < Mb; r += kJ32Threads) {
          float v[W];
#pragma unroll
          for (int l = 0; l < kJB; ++l) {
            v[l] = VI[r + l * Mb];
            v[kJB + l] = VJ[r + l * Mb];
          }
#pragma unroll 1
          for (int l = 0; l < W; ++l) {   // rolled: keeps the 256 entries of J in shared memory
            float o = 0.f;
#pragma unroll
            for (int m = 0; m < W; ++m) o = fmaf(v[m], sJ[m + l * W], o);
            if (l < kJB) VI[r + l * Mb] = o;
            else VJ[r + (l - kJB) * Mb] = o;
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(s.hdr, gridDim.x)) return;
    }
    if (tid == 0 && local_rot) atomicAdd(&s.rot32[sweep], local_rot);
    if (!grid_barrier(s.hdr, gridDim.x)) return;
    if (ld_acquire_u32(&s.rot32[sweep]) == 0) break;
  }
}

// V (Mp x Mp, binary64) = the leading Mp x Mp block of V32.
__global__ void jacobi32_widen_kernel(SvdState s) {
  const int64_t Mp = s.Mp, Mb = s.Mb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < Mp * Mp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % Mp, j = idx / Mp;
    s.V[idx] = (double)s.V32[i + j * Mb];
  }
}

// V <- (3 V - V G) / 2 with T = V G already formed
__global__ void newton_schulz_kernel(double* V, const double* T, int64_t n) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x)
    V[idx] = 1.5 * V[idx] - 0.5 * T[idx];
}

size_t jacobi32_extra_bytes(int64_t M) {
  if (M < kJac32MinM) return 0;
  const int64_t Mp = M + (M & 1);
  const int64_t Mb = (M + 2 * kJB - 1) / (2 * kJB) * (2 * kJB);
  return align256(sizeof(float) * (size_t)M * Mb) + align256(sizeof(float) * (size_t)Mb * Mb) +
         2 * align256(sizeof(double) * (size_t)Mp * Mp) + align256(sizeof(unsigned) * kJ32MaxSweeps) +
         align256(matmul_ws_bytes(Mp, Mp, Mp) > matmul_ws_bytes(M, Mp, M) ? matmul_ws_bytes(Mp, Mp, Mp)
                                                                           : matmul_ws_bytes(M, Mp, M));
}

void jacobi32_carve(SvdState& s, char* p) {
  const int64_t M = s.M, Mp = s.Mp;
  s.Mb = (M + 2 * kJB - 1) / (2 * kJB) * (2 * kJB);
  s.A32 = (float*)p;    p += align256(sizeof(float) * (size_t)M * s.Mb);
  s.V32 = (float*)p;    p += align256(sizeof(float) * (size_t)s.Mb * s.Mb);
  s.G = (double*)p;     p += align256(sizeof(double) * (size_t)Mp * Mp);
  s.Tm = (double*)p;    p += align256(sizeof(double) * (size_t)Mp * Mp);
  s.rot32 = (unsigned*)p; p += align256(sizeof(unsigned) * kJ32MaxSweeps);
  s.mmws = (double*)p;
}

// Leaves s.A = R^T V and s.V = V (orthogonal), the starting point of the
// binary64 sweeps.
cudaError_t launch_jacobi32_precondition(const SvdState& s, const double* R, int64_t ldr, cudaStream_t st) {
  const int64_t M = s.M, Mp = s.Mp;
  cudaError_t e = cudaMemsetAsync(s.rot32, 0, sizeof(unsigned) * kJ32MaxSweeps, st);
  if (e != cudaSuccess) return e;
  jacobi32_init_kernel<<<256, 256, 0, st>>>(s, R, ldr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = sizeof(float) * ((size_t)2 * kJB * M + 4 * kJB * kJB);
  if ((e = ensure_dyn_smem((const void*)jacobi32_block_kernel, smem)) != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi32_block_kernel, kJ32Threads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
  int64_t grid = (s.Mb / kJB) / 2;
  if (grid > (int64_t)per * sms) grid = (int64_t)per * sms;
  SvdState a = s;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)jacobi32_block_kernel, dim3((unsigned)grid), dim3(kJ32Threads), args,
                                  smem, st);
  if (e != cudaSuccess) return e;
  jacobi32_widen_kernel<<<256, 256, 0, st>>>(s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int it = 0; it < 2; ++it) {
    e = launch_matmul_fp64(1, s.V, s.V, s.G, Mp, Mp, Mp, Mp, Mp, Mp, s.mmws, st);   // G = V^T V
    if (e != cudaSuccess) return e;
    e = launch_matmul_fp64(0, s.V, s.G, s.Tm, Mp, Mp, Mp, Mp, Mp, Mp, s.mmws, st);  // T = V G
    if (e != cudaSuccess) return e;
    newton_schulz_kernel<<<256, 256, 0, st>>>(s.V, s.Tm, Mp * Mp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // A = R^T V (M x Mp; rows of V beyond M meet no row of R)
  return launch_matmul_fp64(1, R, s.V, s.A, M, Mp, M, ldr, Mp, M, s.mmws, st);
}

}  // namespace pylom

// common.cuh -- device helpers shared by the library's kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pylom.h"

namespace pylom {

constexpr int kWarp = 32;

// Header at the start of every workspace (512 bytes).  Each call clears it
// with one cudaMemsetAsync before its first kernel.
// The grid barrier's arrival counter and generation word sit in different
// 128-byte lines, so the waiting blocks' polling does not contend with the
// arrivals' atomics.
struct WsHeader {
  int status;               // first device-side pylom_status raised (0 = OK)
  int sweeps;               // Jacobi sweeps used
  long long r;              // truncation rank chosen by pylom_pod
  unsigned barrier_count;   // grid barrier: arrivals
  unsigned spare;
  unsigned rot[64];         // Jacobi: rotations performed in each sweep
  unsigned char pad0[384 - 24 - 64 * 4];
  unsigned barrier_gen;     // grid barrier: generation (own line)
  unsigned char pad1[512 - 384 - 4];
};
static_assert(sizeof(WsHeader) == 512, "workspace header must be 512 bytes");
constexpr int kMaxSweeps = 64;

__device__ __forceinline__ void raise_status(WsHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

__device__ __forceinline__ int read_status(const WsHeader* h) {
  return *((volatile const int*)&h->status);
}

// FP64 tensor-pipe MMA, D(8x8) += A(8x4) B(4x8).
// Fragment ownership (lane = 4 g + t, g = lane / 4, t = lane % 4):
//   a  = A[g][t],  b = B[t][g],  d0 = D[g][2t], d1 = D[g][2t+1].
__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum K per-thread values over the block; every thread gets the K totals in
// out[0..K).  scratch: K * nwarps doubles of shared memory.  Fixed order,
// so results are bitwise repeatable.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) scratch[q * nwarps + warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += scratch[threadIdx.x * nwarps + w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Warp reduce-scatter of 16 values: lane l ends with the warp total of
// p[(l >> 1) & 15] (16 shuffles and 16 additions per lane in five stages of
// halving exchanges, instead of 16 five-step reductions with 80 additions:
// binary64 additions issue at a small fraction of the binary32 rate on this
// part).  p is clobbered.
__device__ __forceinline__ double warp_reduce_scatter16(double (&p)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double send = hi ? p[i] : p[i + n];
      const double keep = hi ? p[i + n] : p[i];
      p[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return p[0] + __shfl_xor_sync(0xffffffffu, p[0], 1);
}

// block_sum<16> through the reduce-scatter: out[0..16) = the block totals.
// scratch: 16 * nwarps doubles.
__device__ __forceinline__ void block_sum16(double (&v)[16], double* scratch, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const double t = warp_reduce_scatter16(v);
  if ((lane & 1) == 0) scratch[((lane >> 1) & 15) * nwarps + warp] = t;
  __syncthreads();
  if (threadIdx.x < 16) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += scratch[threadIdx.x * nwarps + w];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Loads that bypass L1: data written by other blocks of the same launch.
// Knuth's TwoSum in binary32: s = fl(a + b) and e with a + b = s + e
// exactly (round-to-nearest intrinsics, so no contraction or reordering)
__device__ __forceinline__ void two_sum32(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sum of K binary32 values as the unevaluated pair s + c: every addition's
// rounding error is carried in c, so s + c equals the exact sum up to a
// second-order term of about ((K - 1) eps32)^2 times the sum of magnitudes
template <int K>
__device__ __forceinline__ void sum32_compensated(const float (&x)[K], float& s, float& c) {
  s = 0.f;
  c = 0.f;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    float e;
    two_sum32(s, x[j], s, e);
    c = __fadd_rn(c, e);
  }
}

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// The wait is bounded: after kWaitLimitNs of wall time (global timer) it
// records PYLOM_ERR_TIMEOUT and returns false, and every later barrier
// returns false at once, so no block can wait forever.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// `expected` is the number of arrivals that releases the barrier (the grid
// size); limit_ns bounds the wait.
__device__ __forceinline__ bool grid_barrier(WsHeader* h, unsigned expected,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = read_status(h) != PYLOM_ERR_TIMEOUT;
    if (ok) {
      unsigned gen = ld_acquire_u32(&h->barrier_gen);
      __threadfence();
      unsigned arrived = atomicAdd(&h->barrier_count, 1u);
      if (arrived == expected - 1) {
        atomicExch(&h->barrier_count, 0u);
        __threadfence();
        atomicAdd(&h->barrier_gen, 1u);
      } else {
        const unsigned long long t0 = global_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(&h->barrier_gen) == gen) {
          if ((++polls & 63u) == 0) {
            if (global_ns() - t0 > limit_ns) {
              raise_status(h, PYLOM_ERR_TIMEOUT);
              ok = 0;
              break;
            }
            if (read_status(h) == PYLOM_ERR_TIMEOUT) { ok = 0; break; }
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__host__ __device__ __forceinline__ int64_t leaf_begin(int64_t leaf, int64_t N, int64_t P) {
  return (leaf * N) / P;
}

__host__ __device__ __forceinline__ size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace pylom

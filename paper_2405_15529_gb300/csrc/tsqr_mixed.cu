// tsqr_mixed.cu -- mixed-precision leaves of the POD path (pyLOM, arXiv
// 2405.15529, Alg. 1 / Eqs. svdqr1 and svdqr3) on the 5th-generation tensor
// cores of GB300: FP32 working copy, Householder panels of kNB2 = 32
// columns factored with compensated FP32 sums reduced in FP64 (FP64 scalars
// tau, beta and T), and the block-reflector products on tcgen05 in 3xTF32
// (x = hi + lo, hi exact in TF32; hi*hi + hi*lo + lo*hi accumulated in FP32
// in tensor memory).  The tree, the small SVD and the top-down pass stay in
// binary64 (they are the FP64 path's kernels).
//
// A block-reflector application C := (I - V op(T) V^T) C runs per chunk of
// up to 128 columns of C:
//   W stage:  W^T (128 x 32) = C_chunk^T V   -- MMA M = 128 columns,
//             N = 32 reflectors, K = the rows, 64 rows per shared-memory step;
//   W' = -op(T) W  (FP64 on CUDA cores, split into hi/lo);
//   C stage:  per 256-row tile, two MMAs P (128 x 128) = V_half W' -- M = 128
//             rows, N = 128 columns, K = 32 reflectors; each thread adds its
//             row of P (read from tensor memory) to C.
// One CTA of 8 warps per SM owns all 512 tensor-memory columns (warps w and
// w + 4 read lane quadrant w % 4).  One thread issues the MMAs and commits
// them to an mbarrier; every wait is time-bounded (PYLOM_ERR_TIMEOUT) and
// tensor memory is freed on every exit.
//
// Accumulation: long chains of MMAs into one tensor-memory accumulator drift
// (every accumulate step of the tensor core rounds, and the errors do not
// cancel), so every 64-row step of the W stage writes fresh accumulators
// that the threads fold into compensated FP32 sums, and the hi*hi products
// and the small hi*lo + lo*hi cross terms go to separate accumulators that
// are added on the CUDA cores.
#include "kernels.h"
#include "reflectors.cuh"
#include "tc05.cuh"

namespace pylom {

constexpr int kNB2 = 32;          // panel width
constexpr int kMxThreads = 256;   // 8 warps; warps w and w + 4 share tensor-memory lane quadrant w % 4
constexpr int kCH = 128;          // column chunk
constexpr int kKC = 64;           // rows per W-stage step (MMA K)
constexpr int kRT = 256;          // rows per C-stage tile (two 128-row MMAs)
constexpr uint32_t kTmemCols = 512;   // C stage: two halves x (hi*hi, cross) x 128 columns

// shared-memory plan (bytes); the W-stage and C-stage operands share [0, kOpBytes)
constexpr int kWA = kCH * kKC * 4;                 // 32 KB: W-stage A (C^T chunk, 128 x 64)
constexpr int kWB = kNB2 * kKC * 4;                // 8 KB:  W-stage B (V, 32 x 64)
constexpr int kOffWA = 0, kOffWAlo = kWA, kOffWB = 2 * kWA, kOffWBlo = 2 * kWA + kWB;
constexpr int kCA = 128 * kNB2 * 4;                // 16 KB: C-stage A half (V rows, 128 x 32)
constexpr int kOffCA = 0;                          // hi halves at 0, kCA; lo halves at 2 kCA, 3 kCA
constexpr int kOffCB = 4 * kCA, kOffCBlo = 5 * kCA;  // C-stage B (W'^T, 128 x 32)
constexpr int kOpBytes = 6 * kCA;                  // 96 KB >= the W stage's 80 KB
static_assert(2 * kWA + 2 * kWB <= kOpBytes, "W-stage operands must fit the operand region");
constexpr int kOffW = kOpBytes;                    // W: 32 x 128 fp32 (16 KB)
constexpr int kOffT = kOffW + kNB2 * kCH * 4;      // T: 32 x 32 fp64 (8 KB)
constexpr int kOffRed = kOffT + kNB2 * kNB2 * 8;   // panel reductions: 8 warps x 32 x (s, c) floats
constexpr int kOffOut = kOffRed + 8 * kNB2 * 2 * 4;  // panel broadcasts (512 bytes)
constexpr int kMixSmem = kOffOut + 512;
// the FP64 tree merge reuses the same buffer with the leaf kernel's plan
constexpr int kMergeSmem = (int)kLeafSmemBytes;
constexpr int kMixSmemTotal = kMixSmem > kMergeSmem ? kMixSmem : kMergeSmem;
// a second CTA on the same SM would wait for the first one's tensor memory:
// the shared-memory plan keeps them apart
static_assert(2 * kMixSmemTotal > 228 * 1024, "mixed-leaf CTAs must not share an SM");

struct MixedArgs {
  TsqrState s;
  float* Yf;          // N x M fp32 working copy (ld N) -> reflectors
  double* T2;         // per leaf and panel: kNB2 x kNB2 (row-major) fp64
  float* Pb;          // N x kNB2 row-major panel buffers (leaf rows)
  const void* X;
  int64_t ldx;
  int xtype;
  const double* w;
  int remove_mean;
  double* mean;
};

// V(i, p) of a leaf panel starting at column k (unit diagonal, zeros above)
__device__ __forceinline__ float vval_f(const float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, int64_t i, int p) {
  if (p >= nbk || i >= h) return 0.f;
  const int64_t d = k + p;
  if (i < d) return 0.f;
  if (i == d) return 1.f;
  return Y[i + d * ldy];
}

// Kahan-compensated FP32 accumulation, reduced in FP64
struct KSum32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Compensated FP32 value s + c (TwoSum addition): the cross-thread sums of
// the panel statistics stay at about double-float accuracy without FP64
// arithmetic, which runs at a small fraction of the FP32 rate on this part.
struct F2 {
  float s, c;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.s + b.s;
  const float bb = s - a.s;
  const float e = (a.s - (s - bb)) + (b.s - bb);
  return {s, e + a.c + b.c};
}

// Single-pass panel factorisation (columns [k, k+nbk) of the FP32 leaf) on
// the row-major panel copy Pb (leaf rows k..h-1, 32 floats = 128 bytes per
// row).  Pass jj, over the rows from the previous diagonal on:
//   - finishes column jj-1: scales its sub-diagonal into the reflector
//     v_{jj-1} = u / (alpha - beta) and applies (I - tau v v^T) to the later
//     panel columns;
//   - forms, from the still unscaled column jj (u below the diagonal), the
//     squared norm sum u_i^2 and the dots sum u_i a_ic with every other
//     panel column, as compensated FP32 sums.
// Warp 0 then forms beta, tau and the scale of column jj in FP64 and the
// true dots v_j^T a_c = a_jc + scale * sum u_i a_ic (v_j has a one on the
// diagonal), the forward recurrence of T, and the update factors
// tau * v_j^T a_c for the next pass.  One pass and one reduction per column
// (Householder convention beta = -sign(alpha) |x|, sign(0) = +1).
__device__ void panel_factor_mixed(float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, double* tau_out,
                                   double* sT, double* sred, double* sout, float* Pb) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  float* spart = (float*)sred;     // [warp][32][2] partial sums (s, c)
  float* srow = (float*)sout;      // [32] row j of the panel
  float* sfc = srow + kNB2;        // [32] tau * v_j^T a_c (zero outside (jj, nbk))
  float* sscale = sfc + kNB2;      // [1]  scale of column jj
  // gather: Pb[(i - k) * 32 + c] = Y[i, k + c] (zeros beyond nbk)
  for (int64_t i = k + tid; i < h; i += nthr) {
    float4* pr = (float4*)(Pb + (i - k) * kNB2);
#pragma unroll
    for (int q = 0; q < kNB2 / 4; ++q) {
      float4 v;
      v.x = (4 * q + 0 < nbk) ? Y[i + (k + 4 * q + 0) * ldy] : 0.f;
      v.y = (4 * q + 1 < nbk) ? Y[i + (k + 4 * q + 1) * ldy] : 0.f;
      v.z = (4 * q + 2 < nbk) ? Y[i + (k + 4 * q + 2) * ldy] : 0.f;
      v.w = (4 * q + 3 < nbk) ? Y[i + (k + 4 * q + 3) * ldy] : 0.f;
      pr[q] = v;
    }
  }
  if (tid < kNB2) sfc[tid] = 0.f;
  if (tid == 0) sscale[0] = 0.f;
  __syncthreads();
  for (int jj = 0; jj < nbk; ++jj) {
    const int64_t j = k + jj;
    float fc[kNB2];
#pragma unroll
    for (int c = 0; c < kNB2; ++c) fc[c] = sfc[c];
    const float scp = sscale[0];
    KSum32 acc[kNB2];   // acc[jj] collects sum u_i^2
    for (int64_t i = (jj > 0 ? j - 1 : j) + tid; i < h; i += nthr) {
      float4* pr = (float4*)(Pb + (i - k) * kNB2);
      float row[kNB2];
#pragma unroll
      for (int q = 0; q < kNB2 / 4; ++q) {
        const float4 v4 = pr[q];
        row[4 * q] = v4.x; row[4 * q + 1] = v4.y; row[4 * q + 2] = v4.z; row[4 * q + 3] = v4.w;
      }
      if (jj > 0) {
        // row[jj - 1] re-read from the (L1-resident) row rather than indexed
        // at run time, which would move row[] out of registers
        const float rp = ((const float*)pr)[jj - 1];
        const float v = (i == j - 1) ? 1.f : rp * scp;
        // fc is zero outside (jj - 1, nbk), so the update needs no column test
#pragma unroll
        for (int c = 0; c < kNB2; ++c) row[c] = (c == jj - 1) ? (i > j - 1 ? v : row[c]) : row[c] - fc[c] * v;
      }
      if (i == j) {
#pragma unroll
        for (int c = 0; c < kNB2; ++c) srow[c] = row[c];
      } else if (i > j) {
        float u = 0.f;
#pragma unroll
        for (int c = 0; c < kNB2; ++c) u = (c == jj) ? row[c] : u;
#pragma unroll
        for (int c = 0; c < kNB2; ++c)
          if (c < nbk) acc[c].add(u * row[c]);
      }
      if (jj > 0) {
#pragma unroll
        for (int q = 0; q < kNB2 / 4; ++q)
          pr[q] = make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
      }
    }
    // block reduction of the 32 compensated sums: TwoSum shuffles, then the
    // warps' partials in FP64 by warp 0 (lane c owns value c)
#pragma unroll
    for (int c = 0; c < kNB2; ++c) {
      F2 v{acc[c].s, -acc[c].c};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        F2 w{__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)};
        v = f2_add(v, w);
      }
      if (lane == 0) {
        spart[(warp * kNB2 + c) * 2] = v.s;
        spart[(warp * kNB2 + c) * 2 + 1] = v.c;
      }
    }
    __syncthreads();
    if (warp == 0) {
      const int c = lane;
      double tot = 0.0;
      for (int w = 0; w < nwarps; ++w)
        tot += (double)spart[(w * kNB2 + c) * 2] + (double)spart[(w * kNB2 + c) * 2 + 1];
      const double xx = __shfl_sync(0xffffffffu, tot, jj);
      double tau_j = 0.0, beta = 0.0, scale = 0.0;
      if (lane == 0) {
        const double alpha = (double)srow[jj];
        beta = alpha;
        if (xx != 0.0) {
          const double nrm = sqrt(alpha * alpha + xx);
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau_j = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
      }
      tau_j = __shfl_sync(0xffffffffu, tau_j, 0);
      scale = __shfl_sync(0xffffffffu, scale, 0);
      // w_c = v_j^T a_c (c > jj) or v_c^T v_j (c < jj)
      const double wcv = (c < nbk && c != jj) ? (double)srow[c] + scale * tot : 0.0;
      // T[0:jj, jj] = -tau T[0:jj, 0:jj] w[0:jj]; lane p owns row p
      double tp = 0.0;
      for (int q = 0; q < jj; ++q) {
        const double wq = __shfl_sync(0xffffffffu, wcv, q);
        if (c <= q) tp += sT[c * kNB2 + q] * wq;
      }
      if (c < jj) sT[c * kNB2 + jj] = -tau_j * tp;
      if (c == jj) {
        sT[jj * kNB2 + jj] = tau_j;
        tau_out[jj] = tau_j;
      }
      sfc[c] = (c > jj && c < nbk) ? (float)(tau_j * wcv) : 0.f;
      if (lane == 0) {
        sscale[0] = (float)scale;
        Pb[(j - k) * kNB2 + jj] = (float)beta;
      }
    }
    __syncthreads();
  }
  // scatter the factored panel back; the last column's sub-diagonal still
  // needs its scale
  const float scl = sscale[0];
  for (int64_t i = k + tid; i < h; i += nthr) {
    const float4* pr = (const float4*)(Pb + (i - k) * kNB2);
#pragma unroll
    for (int q = 0; q < kNB2 / 4; ++q) {
      const float4 v = pr[q];
#define PYLOM_SCATTER_ONE(t, e)                                                   \
  {                                                                               \
    const int c = 4 * q + (t);                                                    \
    if (c < nbk) Y[i + (k + c) * ldy] = (c == nbk - 1 && i > k + c) ? (e) * scl : (e); \
  }
      PYLOM_SCATTER_ONE(0, v.x)
      PYLOM_SCATTER_ONE(1, v.y)
      PYLOM_SCATTER_ONE(2, v.z)
      PYLOM_SCATTER_ONE(3, v.w)
#undef PYLOM_SCATTER_ONE
    }
  }
  __syncthreads();
}

// Issue the K-slices of a 3xTF32 product from four shared tiles (byte
// offsets; rows of Kk elements): hi*hi into d_hh, hi*lo + lo*hi into d_x,
// both starting from zero.
__device__ __forceinline__ void issue_3xtf32(uint32_t d_hh, uint32_t d_x, unsigned char* smem, int oa, int oalo,
                                             int ob, int oblo, int Kk, uint32_t idesc) {
  using namespace tc05;
  const uint32_t a_hi = smem_u32(smem + oa), a_lo = smem_u32(smem + oalo);
  const uint32_t b_hi = smem_u32(smem + ob), b_lo = smem_u32(smem + oblo);
  const uint32_t sbo = (uint32_t)(Kk / 4) * 128, lbo = 128;
  for (int kk = 0; kk < Kk / 8; ++kk) {
    const uint32_t o = (uint32_t)kk * 256;
    mma_tf32(d_hh, desc(a_hi + o, lbo, sbo), desc(b_hi + o, lbo, sbo), idesc, kk > 0);
    mma_tf32(d_x, desc(a_hi + o, lbo, sbo), desc(b_lo + o, lbo, sbo), idesc, kk > 0);
    mma_tf32(d_x, desc(a_lo + o, lbo, sbo), desc(b_hi + o, lbo, sbo), idesc, true);
  }
}

// The block-reflector application on tcgen05.  C: leaf-relative FP32 matrix
// (rows r0..h, ld ldc), ncols columns.  TRANS: op(T) = T^T (factorisation) or
// T (modes).  Returns false on a timed-out wait.
// Software pipelining: the global loads of the next W-stage step (and of the
// next C-stage row tile's reflector rows) are issued before waiting on the
// current MMAs, and the C-stage epilogue loads the next 16-column group of C
// while it adds the current one, so the tensor-core work and the folds
// overlap the memory latency.
template <bool TRANS>
__device__ bool block_reflector_tc(const float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, float* C,
                                   int64_t ldc, int ncols, const double* sT, unsigned char* smem, uint32_t tmem,
                                   uint64_t* mbar, uint32_t& phase) {
  using namespace tc05;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp & 3, half = warp >> 2;       // tensor-memory lane quadrant; which half of the work
  const uint32_t lanebase = (uint32_t)(quad * 32) << 16;
  float* sW = (float*)(smem + kOffW);
  const int64_t L = h - k;
  bool ok = true;
  for (int c0 = 0; c0 < ncols && ok; c0 += kCH) {
    const int wc = min(kCH, ncols - c0);
    // ---- W stage: W^T (128 x 32) = C_chunk^T V over all rows ----
    // thread (quad, half, lane) folds W[16 half .. 16 half + 15][32 quad + lane]
    float ws_[16], wc_[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) ws_[p] = wc_[p] = 0.f;
    const int64_t nkc = (L + kKC - 1) / kKC;
    // loads: thread t takes row t % 64 of the step and columns (reflectors)
    // t / 64 + 4 u; consecutive lanes read consecutive rows
    const int lr = tid & (kKC - 1), lg = tid / kKC;
    float xa[kCH / 4], xb[kNB2 / 4];
    auto load_w = [&](int64_t kc) {
      const int64_t row = k + kc * kKC + lr;
      const bool rok = row < h;
#pragma unroll
      for (int u = 0; u < kCH / 4; ++u) {
        const int c = lg + 4 * u;
        xa[u] = (rok && c < wc) ? C[row + (int64_t)(c0 + c) * ldc] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kNB2 / 4; ++u) xb[u] = vval_f(Y, ldy, k, nbk, h, row, lg + 4 * u);
    };
    load_w(0);
    for (int64_t kc = 0; kc < nkc && ok; ++kc) {
#pragma unroll
      for (int u = 0; u < kCH / 4; ++u) {
        float hi, lo;
        split_tf32(xa[u], hi, lo);
        const uint32_t o = cm_off(lg + 4 * u, lr, kKC);
        *(float*)(smem + kOffWA + o) = hi;
        *(float*)(smem + kOffWAlo + o) = lo;
      }
#pragma unroll
      for (int u = 0; u < kNB2 / 4; ++u) {
        float hi, lo;
        split_tf32(xb[u], hi, lo);
        const uint32_t o = cm_off(lg + 4 * u, lr, kKC);
        *(float*)(smem + kOffWB + o) = hi;
        *(float*)(smem + kOffWBlo + o) = lo;
      }
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        issue_3xtf32(tmem, tmem + kNB2, smem, kOffWA, kOffWAlo, kOffWB, kOffWBlo, kKC, idesc_tf32(128, kNB2));
        commit(mbar);
      }
      if (kc + 1 < nkc) load_w(kc + 1);   // in flight while the MMAs run
      const bool w_ok = mbar_wait(mbar, phase);
      phase ^= 1u;
      fence_after();
      ok = !__syncthreads_or(!w_ok);
      if (!ok) break;
      {
        float hh[16], xx[16];
        tmem_ld16(tmem + lanebase + (uint32_t)(16 * half), hh);
        tmem_ld16(tmem + lanebase + (uint32_t)(kNB2 + 16 * half), xx);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float y = (hh[j] + xx[j]) - wc_[j];
          const float t = ws_[j] + y;
          wc_[j] = (t - ws_[j]) - y;
          ws_[j] = t;
        }
      }
      // the next step's MMAs overwrite the accumulators only after the
      // barrier that follows its shared-memory stores
      fence_before();
    }
    if (!ok) break;
    __syncthreads();
    {
      const int c = quad * 32 + lane;
#pragma unroll
      for (int j = 0; j < 16; ++j) sW[(16 * half + j) * kCH + c] = (float)((double)ws_[j] - (double)wc_[j]);
    }
    __syncthreads();
    // ---- W' = -op(T) W, as B = W'^T (row = column c, K = p), split ----
    for (int idx = tid; idx < kCH * kNB2; idx += blockDim.x) {
      const int c = idx % kCH, p = idx / kCH;
      double s = 0.0;
      if (TRANS) {
        for (int q = 0; q <= p; ++q) s += sT[q * kNB2 + p] * (double)sW[q * kCH + c];
      } else {
        for (int q = p; q < kNB2; ++q) s += sT[p * kNB2 + q] * (double)sW[q * kCH + c];
      }
      float hi, lo;
      split_tf32((float)(-s), hi, lo);
      const uint32_t o = cm_off(c, p, kNB2);
      *(float*)(smem + kOffCB + o) = hi;
      *(float*)(smem + kOffCBlo + o) = lo;
    }
    // ---- C stage: per 256-row tile, P = V_tile W' (two 128-row MMAs); C += P ----
    const int64_t nrt = (L + kRT - 1) / kRT;
    float xv[kNB2];
    auto load_v = [&](int64_t rt) {
      const int64_t row = k + rt * kRT + tid;
#pragma unroll
      for (int p = 0; p < kNB2; ++p) xv[p] = vval_f(Y, ldy, k, nbk, h, row, p);
    };
    load_v(0);
    for (int64_t rt = 0; rt < nrt && ok; ++rt) {
      const int64_t rb = k + rt * kRT;
      {
        const int hv = tid >> 7, r = tid & 127;   // half of the tile, row within it
#pragma unroll
        for (int p = 0; p < kNB2; ++p) {
          float hi, lo;
          split_tf32(xv[p], hi, lo);
          const uint32_t o = cm_off(r, p, kNB2);
          *(float*)(smem + kOffCA + hv * kCA + o) = hi;
          *(float*)(smem + kOffCA + (2 + hv) * kCA + o) = lo;
        }
      }
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
#pragma unroll
        for (int hv = 0; hv < 2; ++hv)
          issue_3xtf32(tmem + hv * 256, tmem + hv * 256 + kCH, smem, kOffCA + hv * kCA, kOffCA + (2 + hv) * kCA,
                       kOffCB, kOffCBlo, kNB2, idesc_tf32(128, kCH));
        commit(mbar);
      }
      if (rt + 1 < nrt) load_v(rt + 1);
      const int64_t row = rb + 128 * half + 32 * quad + lane;
      const bool rok = row < h;
      float* crow = C + row + (int64_t)c0 * ldc;
      const uint32_t tbase = tmem + lanebase + (uint32_t)(half * 256);
      float cv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) cv[j] = (rok && j < wc) ? crow[(int64_t)j * ldc] : 0.f;
      const bool w_ok = mbar_wait(mbar, phase);
      phase ^= 1u;
      fence_after();
      ok = !__syncthreads_or(!w_ok);
      if (!ok) break;
      for (int cc = 0; cc < kCH; cc += 16) {
        float cn[16];
        if (cc + 16 < kCH) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cn[j] = (rok && cc + 16 + j < wc) ? crow[(int64_t)(cc + 16 + j) * ldc] : 0.f;
        }
        float v[16], vx[16];
        tmem_ld16(tbase + (uint32_t)cc, v);
        tmem_ld16(tbase + (uint32_t)(kCH + cc), vx);
        if (rok) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cc + j < wc) crow[(int64_t)(cc + j) * ldc] = cv[j] + (v[j] + vx[j]);
        }
        if (cc + 16 < kCH) {
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[j] = cn[j];
        }
      }
      fence_before();
    }
    __syncthreads();
  }
  return ok;
}

template <typename TX>
__device__ void mixed_prologue(const MixedArgs& a, float* Y, int64_t ldy, int64_t r0, int64_t h) {
  const TX* X = (const TX*)a.X;
  const int64_t M = a.s.M;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < h; i += blockDim.x) {
    const int64_t n = r0 + i;
    double xbar = 0.0;
    if (a.remove_mean) {
      double sum = 0.0;
      for (int64_t m = 0; m < M; ++m) sum += (double)X[n + m * a.ldx];
      xbar = sum / (double)M;
    }
    if (a.mean) a.mean[n] = xbar;
    double sw = 1.0;
    if (a.w) {
      const double wn = a.w[n];
      if (!(wn > 0.0) || !isfinite(wn)) bad = 1;
      sw = sqrt(wn);
    }
    for (int64_t m = 0; m < M; ++m) {
      const double x = (double)X[n + m * a.ldx];
      if (!isfinite(x)) bad = 1;
      Y[i + m * ldy] = (float)(sw * (x - xbar));
    }
  }
  if (bad) raise_status(a.s.hdr, PYLOM_ERR_NONFINITE);
}

__global__ void __launch_bounds__(kMxThreads) leaf_qr_mixed_kernel(MixedArgs a) {
  extern __shared__ __align__(128) unsigned char msm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const TsqrState& s = a.s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t leaf = blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M, ldy = s.N;
  const int64_t npan = (M + kNB2 - 1) / kNB2;
  float* Y = a.Yf + r0;
  double* sT = (double*)(msm + kOffT);
  double* sred = (double*)(msm + kOffRed);
  double* sout = (double*)(msm + kOffOut);
  if (a.xtype == PYLOM_F32)
    mixed_prologue<float>(a, Y, ldy, r0, h);
  else
    mixed_prologue<double>(a, Y, ldy, r0, h);
  if (tid == 0) tc05::mbar_init(&mbar, 1);
  if (warp == 0) tc05::tmem_alloc(&tmem_base, kTmemCols);
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t k = 0; k < M && ok; k += kNB2) {
    const int nbk = (int)((M - k) < kNB2 ? (M - k) : kNB2);
    for (int idx = tid; idx < kNB2 * kNB2; idx += blockDim.x) sT[idx] = 0.0;
    __syncthreads();
    panel_factor_mixed(Y, ldy, k, nbk, h, s.tau + leaf * M + k, sT, sred, sout, a.Pb + r0 * kNB2);
    __syncthreads();
    double* Tg = a.T2 + (leaf * npan + k / kNB2) * kNB2 * kNB2;
    for (int idx = tid; idx < kNB2 * kNB2; idx += blockDim.x) Tg[idx] = sT[idx];
    if (k + nbk < M)
      ok = block_reflector_tc<true>(Y, ldy, k, nbk, h, Y + (k + nbk) * ldy, ldy, (int)(M - k - nbk), sT, msm, tmem,
                                    &mbar, phase);
    __syncthreads();
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
  if (!ok) {
    if (tid == 0) raise_status(s.hdr, PYLOM_ERR_TIMEOUT);
    return;
  }
  // leaf R (FP64) into its slot, then the FP64 tree
  double* Rl = s.Rs + leaf * M * M;
  for (int64_t idx = tid; idx < M * M; idx += blockDim.x) {
    const int64_t i = idx % M, j = idx / M;
    Rl[idx] = (i <= j) ? (double)Y[i + j * ldy] : 0.0;
  }
  __threadfence();
  __syncthreads();
  double* mT = (double*)msm;
  double* mred = mT + kSmT;
  double* mout = mred + kSmRed;
  double* mW = mout + kSmOut;
  double* mWp = mW + kSmW;
  if (s.climb) tree_climb(s, leaf, mT, mred, mout, mW, mWp);
}

// Per leaf: U_leaf = Q_leaf [B_leaf; 0] in FP32 on tcgen05 (panels last to
// first, op(T) = T), then Phi = U / sqrt(w) if asked.
__global__ void __launch_bounds__(kMxThreads) modes_mixed_kernel(TsqrState s, const float* Yf, const double* T2,
                                                                int64_t r_fixed, const double* w, int physical,
                                                                float* U, int64_t ldu, int64_t* r_out) {
  extern __shared__ __align__(128) unsigned char msm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t leaf = blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M;
  const int64_t npan = (M + kNB2 - 1) / kNB2;
  const int64_t r = (r_fixed >= 0) ? r_fixed : s.hdr->r;
  if (leaf == 0 && tid == 0 && r_out) *r_out = r;
  float* C = U + r0;
  const double* Bl = s.B + leaf * M * s.rmax;
  for (int64_t c = 0; c < r; ++c)
    for (int64_t i = tid; i < h; i += blockDim.x) C[i + c * ldu] = (i < M) ? (float)Bl[i + c * M] : 0.f;
  double* sT = (double*)(msm + kOffT);
  if (tid == 0) tc05::mbar_init(&mbar, 1);
  if (warp == 0) tc05::tmem_alloc(&tmem_base, kTmemCols);
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool ok = true;
  const float* Y = Yf + r0;
  for (int64_t pan = npan - 1; pan >= 0 && ok; --pan) {
    const int64_t k = pan * kNB2;
    const int nbk = (int)((M - k) < kNB2 ? (M - k) : kNB2);
    const double* Tg = T2 + (leaf * npan + pan) * kNB2 * kNB2;
    for (int idx = tid; idx < kNB2 * kNB2; idx += blockDim.x) sT[idx] = Tg[idx];
    __syncthreads();
    ok = block_reflector_tc<false>(Y, s.N, k, nbk, h, C, ldu, (int)r, sT, msm, tmem, &mbar, phase);
    __syncthreads();
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
  if (!ok) {
    if (tid == 0) raise_status(s.hdr, PYLOM_ERR_TIMEOUT);
    return;
  }
  if (physical && w) {
    for (int64_t i = tid; i < h; i += blockDim.x) {
      const float iw = (float)(1.0 / sqrt(w[r0 + i]));
      for (int64_t c = 0; c < r; ++c) C[i + c * ldu] *= iw;
    }
  }
}

// Adjoint support: per leaf, C_leaf := Q_leaf^T C_leaf in FP32 on tcgen05
// (panels in factorisation order, op(T) = T^T), then the leaf's top M rows
// go to its binary64 slot Z (M x r, the start of the tree's bottom-up pass).
__global__ void __launch_bounds__(kMxThreads) leaf_qt_mixed_kernel(TsqrState s, const float* Yf, const double* T2,
                                                                  float* C, int64_t r, double* Z) {
  extern __shared__ __align__(128) unsigned char msm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t leaf = blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M;
  const int64_t npan = (M + kNB2 - 1) / kNB2;
  double* sT = (double*)(msm + kOffT);
  if (tid == 0) tc05::mbar_init(&mbar, 1);
  if (warp == 0) tc05::tmem_alloc(&tmem_base, kTmemCols);
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  bool ok = true;
  const float* Y = Yf + r0;
  float* Cl = C + r0;
  for (int64_t pan = 0; pan < npan && ok; ++pan) {
    const int64_t k = pan * kNB2;
    const int nbk = (int)((M - k) < kNB2 ? (M - k) : kNB2);
    const double* Tg = T2 + (leaf * npan + pan) * kNB2 * kNB2;
    for (int idx = tid; idx < kNB2 * kNB2; idx += blockDim.x) sT[idx] = Tg[idx];
    __syncthreads();
    ok = block_reflector_tc<true>(Y, s.N, k, nbk, h, Cl, s.N, (int)r, sT, msm, tmem, &mbar, phase);
    __syncthreads();
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
  if (!ok) {
    if (tid == 0) raise_status(s.hdr, PYLOM_ERR_TIMEOUT);
    return;
  }
  double* Zl = Z + leaf * M * r;
  for (int64_t idx = tid; idx < M * r; idx += blockDim.x) Zl[idx] = (double)Cl[(idx % M) + (idx / M) * s.N];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

size_t mixed_extra_bytes(int64_t N, int64_t M, int64_t P) {
  const int64_t npan = (M + kNB2 - 1) / kNB2;
  return align256(sizeof(float) * (size_t)N * M) + align256(sizeof(double) * (size_t)P * npan * kNB2 * kNB2) +
         align256(sizeof(float) * (size_t)N * kNB2);
}

cudaError_t launch_tsqr_mixed(const TsqrState& s, char* extra, const void* X, int64_t ldx, int xtype,
                              const double* w, int remove_mean, double* mean, cudaStream_t st) {
  static bool attr = false;
  cudaError_t e;
  if (!attr) {
    e = cudaFuncSetAttribute(leaf_qr_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMixSmemTotal);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(modes_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMixSmemTotal);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t npan = (s.M + kNB2 - 1) / kNB2;
  char* t2 = extra + align256(sizeof(float) * (size_t)s.N * s.M);
  char* pb = t2 + align256(sizeof(double) * (size_t)s.P * npan * kNB2 * kNB2);
  MixedArgs a{s, (float*)extra, (double*)t2, (float*)pb, X, ldx, xtype, w, remove_mean, mean};
  leaf_qr_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || s.climb) return e;
  return launch_tree_coop(s, st);
}

cudaError_t launch_modes_mixed(const TsqrState& s, char* extra, const double* Ur, int64_t ldur, int64_t r_fixed,
                               const double* w, int physical, float* U, int64_t ldu, int64_t* r_out, cudaStream_t st,
                               cudaEvent_t mid) {
  cudaError_t e = launch_down_pass_fp64(s, Ur, ldur, r_fixed, st);
  if (e != cudaSuccess) return e;
  if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
  const float* Yf = (const float*)extra;
  const double* T2 = (const double*)(extra + align256(sizeof(float) * (size_t)s.N * s.M));
  modes_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(s, Yf, T2, r_fixed, w, physical, U, ldu, r_out);
  return cudaGetLastError();
}

cudaError_t launch_leaf_qt_mixed(const TsqrState& s, char* extra, float* C, int64_t r, double* Z, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(leaf_qt_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMixSmemTotal);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(modes_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMixSmemTotal);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const float* Yf = (const float*)extra;
  const double* T2 = (const double*)(extra + align256(sizeof(float) * (size_t)s.N * s.M));
  leaf_qt_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(s, Yf, T2, C, r, Z);
  return cudaGetLastError();
}

}  // namespace pylom

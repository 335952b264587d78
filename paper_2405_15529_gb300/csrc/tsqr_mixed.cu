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
//             N = 32 reflectors, K = the rows, 32 rows per shared-memory stage;
//   W' = -op(T) W  (FP64 on CUDA cores, split into hi/lo);
//   C stage:  per 128-row tile, P (128 x 128) = V_tile W' -- M = 128 rows,
//             N = 128 columns, K = 32 reflectors; each thread adds its row of
//             P (read from tensor memory) to C.
// One thread issues the MMAs and commits them to an mbarrier; every wait is
// time-bounded (PYLOM_ERR_TIMEOUT) and tensor memory is freed on every exit.
//
// Accumulation: long chains of MMAs into one tensor-memory accumulator drift
// (every accumulate step of the tensor core rounds, and the errors do not
// cancel), so every 32-row stage of the W stage writes fresh accumulators
// that the threads fold into compensated FP32 sums, and the hi*hi products
// and the small hi*lo + lo*hi cross terms go to separate accumulators that
// are added on the CUDA cores.
#include "kernels.h"
#include "reflectors.cuh"
#include "tc05.cuh"

namespace pylom {

constexpr int kNB2 = 32;          // panel width
constexpr int kMxThreads = 128;   // 4 warps = the 4 tensor-memory lane quadrants
constexpr int kCH = 128;          // column chunk
constexpr int kRT = 128;          // row tile (C stage)
constexpr int kKC = 32;           // rows per W-stage shared-memory stage
constexpr uint32_t kTmemCols = 256;   // C stage: hi*hi and cross-term accumulators, 128 columns each

// shared-memory plan (bytes)
constexpr int kTileA = kCH * kKC * 4;           // 16 KB: one 128 x 32 fp32 tile
constexpr int kOffA = 0;                        // A hi (W stage: C^T chunk; C stage: V rows)
constexpr int kOffAlo = kOffA + kTileA;         // A lo
constexpr int kOffB = kOffAlo + kTileA;         // B hi (W stage: V 32 x 32 uses 4 KB; C stage: W'^T 128 x 32)
constexpr int kOffBlo = kOffB + kTileA;         // B lo
constexpr int kOffW = kOffBlo + kTileA;         // W: 32 x 128 fp32 (16 KB)
constexpr int kOffT = kOffW + kNB2 * kCH * 4;   // T: 32 x 32 fp64 (8 KB)
constexpr int kOffRed = kOffT + kNB2 * kNB2 * 8;  // reductions: 32 x 4 warps doubles + 64 outputs
constexpr int kMixSmem = kOffRed + (kNB2 * 4 + 64) * 8;
// the FP64 tree merge reuses the same buffer with the leaf kernel's plan
constexpr int kMergeSmem = (int)kLeafSmemBytes;
constexpr int kMixSmemTotal = kMixSmem > kMergeSmem ? kMixSmem : kMergeSmem;

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

template <int K>
__device__ __forceinline__ void block_sum_d(double (&v)[K], double* scratch, double* out) {
  block_sum<K>(v, scratch, out);
}

// Panel factorisation (columns [k, k+nbk) of the FP32 leaf), the same
// two-pass-per-column scheme as the FP64 leaves: scale v_j and form its dot
// products with the panel, then update the panel and the next norm.  Sums
// are compensated FP32 per thread and FP64 across threads.
// The passes run on a row-major copy of the panel (Pb: leaf rows k..h-1, 32
// contiguous floats = 128 bytes per row), so every pass streams contiguous
// rows instead of 32 columns that are N elements apart; the panel is
// gathered before and scattered back to the column-major leaf after.
__device__ void panel_factor_mixed(float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, double* tau_out,
                                   double* sT, double* sred, double* sout, float* Pb) {
  const int tid = threadIdx.x, nthr = blockDim.x;
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
  __syncthreads();
  double xx;
  {
    KSum32 ks;
    for (int64_t i = k + 1 + tid; i < h; i += nthr) {
      const float a = Pb[(i - k) * kNB2];
      ks.add(a * a);
    }
    double v[1] = {ks.get()};
    block_sum_d<1>(v, sred, sout);
    xx = sout[0];
  }
  for (int jj = 0; jj < nbk; ++jj) {
    const int64_t j = k + jj;
    const double alpha = (double)Pb[(j - k) * kNB2 + jj];
    double tau_j = 0.0, beta = alpha, scale = 0.0;
    if (xx != 0.0) {
      const double nrm = sqrt(alpha * alpha + xx);
      beta = (alpha >= 0.0) ? -nrm : nrm;
      tau_j = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    const float scf = (float)scale;
    KSum32 acc[kNB2];
    for (int64_t i = j + tid; i < h; i += nthr) {
      float row[kNB2];
      const float4* pr = (const float4*)(Pb + (i - k) * kNB2);
#pragma unroll
      for (int q = 0; q < kNB2 / 4; ++q) {
        const float4 v4 = pr[q];
        row[4 * q] = v4.x; row[4 * q + 1] = v4.y; row[4 * q + 2] = v4.z; row[4 * q + 3] = v4.w;
      }
      float rj = 0.f;   // row[jj] without a runtime index (keeps row[] in registers)
#pragma unroll
      for (int c = 0; c < kNB2; ++c)
        if (c == jj) rj = row[c];
      float v = 1.f;
      if (i != j) {
        v = rj * scf;
        Pb[(i - k) * kNB2 + jj] = v;
      }
#pragma unroll
      for (int c = 0; c < kNB2; ++c)
        if (c < nbk && c != jj) acc[c].add(v * row[c]);
    }
    double dv[kNB2];
#pragma unroll
    for (int c = 0; c < kNB2; ++c) dv[c] = acc[c].get();
    block_sum_d<kNB2>(dv, sred, sout);
    if (tid == 0) {
      Pb[(j - k) * kNB2 + jj] = (float)beta;
      tau_out[jj] = tau_j;
      for (int p = 0; p < jj; ++p) {
        double s = 0.0;
        for (int q = p; q < jj; ++q) s += sT[p * kNB2 + q] * sout[q];
        sT[p * kNB2 + jj] = -tau_j * s;
      }
      sT[jj * kNB2 + jj] = tau_j;
    }
    float fc[kNB2];
#pragma unroll
    for (int c = 0; c < kNB2; ++c) fc[c] = (c > jj && c < nbk) ? (float)(tau_j * sout[c]) : 0.f;
    KSum32 nx;
    if (jj + 1 < nbk) {
      for (int64_t i = j + tid; i < h; i += nthr) {
        float4* pr = (float4*)(Pb + (i - k) * kNB2);
        float row[kNB2];
#pragma unroll
        for (int q = 0; q < kNB2 / 4; ++q) {
          const float4 v4 = pr[q];
          row[4 * q] = v4.x; row[4 * q + 1] = v4.y; row[4 * q + 2] = v4.z; row[4 * q + 3] = v4.w;
        }
        float rj = 0.f;
#pragma unroll
        for (int c = 0; c < kNB2; ++c)
          if (c == jj) rj = row[c];
        const float v = (i == j) ? 1.f : rj;
        float rn = 0.f;
#pragma unroll
        for (int c = 0; c < kNB2; ++c) {
          if (c > jj) row[c] -= fc[c] * v;
          if (c == jj + 1) rn = row[c];
        }
        if (i > j + 1) nx.add(rn * rn);
        // write back the updated columns (the leading ones are unchanged)
#pragma unroll
        for (int q = 0; q < kNB2 / 4; ++q)
          if (4 * q + 3 > jj) pr[q] = make_float4(row[4 * q], row[4 * q + 1], row[4 * q + 2], row[4 * q + 3]);
      }
    }
    double nv[1] = {nx.get()};
    block_sum_d<1>(nv, sred, sout);
    xx = sout[0];
  }
  // scatter the factored panel (R above the diagonal, reflectors below) back
  for (int64_t i = k + tid; i < h; i += nthr) {
    const float4* pr = (const float4*)(Pb + (i - k) * kNB2);
#pragma unroll
    for (int q = 0; q < kNB2 / 4; ++q) {
      const float4 v = pr[q];
      if (4 * q + 0 < nbk) Y[i + (k + 4 * q + 0) * ldy] = v.x;
      if (4 * q + 1 < nbk) Y[i + (k + 4 * q + 1) * ldy] = v.y;
      if (4 * q + 2 < nbk) Y[i + (k + 4 * q + 2) * ldy] = v.z;
      if (4 * q + 3 < nbk) Y[i + (k + 4 * q + 3) * ldy] = v.w;
    }
  }
  __syncthreads();
}

// Issue the K-slices of a 3xTF32 product from the four shared tiles (rows
// of Kk elements): hi*hi into d_hh, hi*lo + lo*hi into d_x, both starting
// from zero.
__device__ __forceinline__ void issue_3xtf32(uint32_t d_hh, uint32_t d_x, unsigned char* smem, int Kk,
                                             uint32_t idesc) {
  using namespace tc05;
  const uint32_t a_hi = smem_u32(smem + kOffA), a_lo = smem_u32(smem + kOffAlo);
  const uint32_t b_hi = smem_u32(smem + kOffB), b_lo = smem_u32(smem + kOffBlo);
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
template <bool TRANS>
__device__ bool block_reflector_tc(const float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, float* C,
                                   int64_t ldc, int ncols, const double* sT, unsigned char* smem, uint32_t tmem,
                                   uint64_t* mbar, uint32_t& phase) {
  using namespace tc05;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* sW = (float*)(smem + kOffW);
  const int64_t L = h - k;
  bool ok = true;
  for (int c0 = 0; c0 < ncols && ok; c0 += kCH) {
    const int wc = min(kCH, ncols - c0);
    // ---- W stage: W^T (128 x 32) = C_chunk^T V over all rows ----
    // thread (warp w, lane l) owns column c = 32 w + l of the chunk and folds
    // each stage's partial W[0..31][c] into compensated FP32 sums
    float ws_[kNB2], wc_[kNB2];
#pragma unroll
    for (int p = 0; p < kNB2; ++p) ws_[p] = wc_[p] = 0.f;
    const int64_t nkc = (L + kKC - 1) / kKC;
    for (int64_t kc = 0; kc < nkc && ok; ++kc) {
      const int64_t rb = k + kc * kKC;
      // A = C^T chunk: row = column c (0..127), K = row i (0..31); warp w
      // takes columns c = w + 4u, lane = row; 8 loads in flight per batch
      {
        const int64_t row = rb + lane;
        const bool rok = row < h;
        for (int cb = 0; cb < kCH; cb += 32) {
          float x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = cb + warp + 4 * u;
            x[u] = (rok && c < wc) ? C[row + (int64_t)(c0 + c) * ldc] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            float hi, lo;
            split_tf32(x[u], hi, lo);
            const uint32_t o = cm_off(cb + warp + 4 * u, lane, kKC);
            *(float*)(smem + kOffA + o) = hi;
            *(float*)(smem + kOffAlo + o) = lo;
          }
        }
        // B = V chunk: row = reflector p (0..31), K = row i
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = vval_f(Y, ldy, k, nbk, h, rb + lane, warp + 4 * u);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float hi, lo;
          split_tf32(x[u], hi, lo);
          const uint32_t o = cm_off(warp + 4 * u, lane, kKC);
          *(float*)(smem + kOffB + o) = hi;
          *(float*)(smem + kOffBlo + o) = lo;
        }
      }
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        issue_3xtf32(tmem, tmem + kNB2, smem, kKC, idesc_tf32(128, kNB2));
        commit(mbar);
      }
      const bool w_ok = mbar_wait(mbar, phase);
      phase ^= 1u;
      fence_after();
      ok = !__syncthreads_or(!w_ok);
      if (!ok) break;
      const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
      for (int p0 = 0; p0 < kNB2; p0 += 16) {
        float hh[16], xx[16];
        tmem_ld16(tmem + lanebase + (uint32_t)p0, hh);
        tmem_ld16(tmem + lanebase + (uint32_t)(kNB2 + p0), xx);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float y = (hh[j] + xx[j]) - wc_[p0 + j];
          const float t = ws_[p0 + j] + y;
          wc_[p0 + j] = (t - ws_[p0 + j]) - y;
          ws_[p0 + j] = t;
        }
      }
      fence_before();
      __syncthreads();
    }
    if (!ok) break;
    {
      const int c = warp * 32 + lane;
#pragma unroll
      for (int p = 0; p < kNB2; ++p) sW[p * kCH + c] = (float)((double)ws_[p] - (double)wc_[p]);
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
      *(float*)(smem + kOffB + o) = hi;
      *(float*)(smem + kOffBlo + o) = lo;
    }
    // ---- C stage: per 128-row tile, P = V_tile W'; C += P ----
    const int64_t nrt = (L + kRT - 1) / kRT;
    for (int64_t rt = 0; rt < nrt && ok; ++rt) {
      const int64_t rb = k + rt * kRT;
      // A = V rows: row = r (0..127), K = p (0..31); thread t takes row t,
      // all 32 loads issued before use
      {
        const int r = tid;
        float x[kNB2];
#pragma unroll
        for (int p = 0; p < kNB2; ++p) x[p] = vval_f(Y, ldy, k, nbk, h, rb + r, p);
#pragma unroll
        for (int p = 0; p < kNB2; ++p) {
          float hi, lo;
          split_tf32(x[p], hi, lo);
          const uint32_t o = cm_off(r, p, kNB2);
          *(float*)(smem + kOffA + o) = hi;
          *(float*)(smem + kOffAlo + o) = lo;
        }
      }
      fence_smem_async();
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        issue_3xtf32(tmem, tmem + kCH, smem, kNB2, idesc_tf32(128, kCH));
        commit(mbar);
      }
      const bool w_ok = mbar_wait(mbar, phase);
      phase ^= 1u;
      fence_after();
      ok = !__syncthreads_or(!w_ok);
      if (!ok) break;
      const int64_t row = rb + warp * 32 + lane;
      float v[16], vx[16];
      for (int cc = 0; cc < kCH; cc += 16) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kCH + cc), vx);
        if (row < h) {
          float cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cv[j] = (cc + j < wc) ? C[row + (int64_t)(c0 + cc + j) * ldc] : 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cc + j < wc) C[row + (int64_t)(c0 + cc + j) * ldc] = cv[j] + (v[j] + vx[j]);
        }
      }
      fence_before();
      __syncthreads();
    }
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
  double* sout = sred + kNB2 * 4;
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

}  // namespace pylom

// tsqr_mixed.cu -- mixed-precision leaves of the POD path (pyLOM, arXiv
// 2405.15529, Alg. 1 / Eqs. svdqr1 and svdqr3) on the 5th-generation tensor
// cores of GB300: FP32 working copy, Householder panels of kNB2 = 32
// columns factored by chunked TSQR and Householder reconstruction (T in
// FP64), and the block-reflector products on tcgen05 in 3xTF32
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

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
// TMA ring of the factorisation's W stage: per 64-row step, the raw FP32
// boxes of the C chunk (64 rows x 128 columns) and of the panel (64 x 32),
// two stages.  The steps start at the panel's first row rounded down to a
// multiple of 4 (a 16-byte boundary), so every step's box is aligned.
constexpr int kTmaRows = kKC;
constexpr int kRawC = kTmaRows * kCH * 4;          // 32,768 B
constexpr int kRawV = kTmaRows * kNB2 * 4;         // 8,192 B
constexpr int kStageBytes = kRawC + kRawV;
constexpr int kOffRaw = kOffT + kNB2 * kNB2 * 8;
static_assert(kOffRaw % 128 == 0 && kRawC % 128 == 0, "TMA destinations must be 128-byte aligned");
constexpr int kMixSmem = kOffRaw + 2 * kStageBytes;
// the FP64 tree merge reuses the same buffer with the leaf kernel's plan
constexpr int kMergeSmem = (int)kLeafSmemBytes;
constexpr int kMixSmemTotal = kMixSmem > kMergeSmem ? kMixSmem : kMergeSmem;
// a second CTA on the same SM would wait for the first one's tensor memory:
// the shared-memory plan keeps them apart
static_assert(2 * kMixSmemTotal > 228 * 1024, "mixed-leaf CTAs must not share an SM");

// Leading dimension of the FP32 working copy: N rounded up to a multiple of
// 4, so every column starts on a 16-byte boundary (TMA strides).
__host__ __device__ __forceinline__ int64_t yf_ld(int64_t N) { return (N + 3) & ~int64_t(3); }

struct MixedArgs {
  TsqrState s;
  float* Yf;          // N x M fp32 working copy (ld yf_ld(N)) -> reflectors
  double* T2;         // per leaf and panel: kNB2 x kNB2 (row-major) fp64
  float* Pb;          // panel scratch: (N / 128 + P + 1) chunk slots of kHrSlot floats
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

// ---------------------------------------------------------------------------
// Panel factorisation: chunked TSQR + Householder reconstruction
// ---------------------------------------------------------------------------
// The panel A (L = h - k rows, nbk <= 32 columns) is too tall for the SM's
// on-chip memory, so a column-by-column Householder sweep would stream it
// once per column.  Instead (three passes over the panel):
//   1. every 128-row chunk is factored by one warp in registers
//      (Householder, lane = rows lane + 32 q), chunk R to scratch, the
//      chunk's reflectors back into the panel;
//   2. the chunk R factors are merged pairwise up a binary tree (a warp per
//      merge, lane = column; a merge's reflectors replace the right child's
//      R), then the explicit Q (L x nbk) of the panel is formed top-down:
//      the root block I is pushed through the merges and every chunk's
//      reflectors, and written over the panel;
//   3. Householder reconstruction (Ballard et al., "Reconstructing
//      Householder vectors from tall-skinny QR", 2015): with signs
//      s_j = -sign of the pivot, the LU factorisation without pivoting
//      Q - [S; 0] = V U gives the unit lower trapezoidal reflector matrix V,
//      T = -U S V1^-T (upper triangular, tau_j = T_jj in [1, 2]) and
//      R = S R_tsqr, so that (I - V T V^T)[R; 0] = A, the same compact WY
//      form the column sweep produces.  V's rows below the top block are
//      the rows of Q U^-1 (one pass, a thread per row).
constexpr int kCR = 128;                                   // rows per chunk (4 per lane)
constexpr int kHrSlot = 2 * kNB2 * kNB2 + 2 * kNB2;        // floats per chunk: R / node reflectors, Q block, taus
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp transpose-reduction: lane l ends with the sum over the warp of p[l]
// (31 shuffles in five stages of independent exchanges, instead of one
// five-step reduction per entry).  p is clobbered.
__device__ __forceinline__ float reduce_scatter32(float (&p)[kNB2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = hi ? p[i] : p[i + o];
      const float keep = hi ? p[i + o] : p[i];
      p[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return p[0];
}

// Householder scalars for [alpha; x] with xx = |x|^2 (convention beta = -sign(alpha) |.|, sign(0) = +1)
__device__ __forceinline__ void house_scalars(float alpha, float xx, float& tau, float& beta, float& scale) {
  tau = 0.f;
  beta = alpha;
  scale = 0.f;
  if (xx > 0.f) {
    const float nrm = sqrtf(fmaf(alpha, alpha, xx));
    beta = alpha >= 0.f ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = 1.f / (alpha - beta);
  }
}

// Step 1: Householder QR of each 128-row chunk, one warp per chunk.
__device__ void hr_chunks(float* Y, int64_t ldy, int64_t k, int nbk, int64_t L, int64_t nc, float* hs) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t c = warp; c < nc; c += nw) {
    const int64_t base = k + c * kCR;
    const int64_t nrow = (L - c * kCR) < kCR ? (L - c * kCR) : kCR;
    float a[4][kNB2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t row = lane + 32 * q;
#pragma unroll
      for (int col = 0; col < kNB2; ++col)
        a[q][col] = (row < nrow && col < nbk) ? Y[base + row + (k + col) * ldy] : 0.f;
    }
    float mytau = 0.f;
#pragma unroll
    for (int j = 0; j < kNB2; ++j) {
      if (j < nbk) {
        float xx = (lane > j) ? a[0][j] * a[0][j] : 0.f;
#pragma unroll
        for (int q = 1; q < 4; ++q) xx = fmaf(a[q][j], a[q][j], xx);
        xx = warp_sumf(xx);
        const float alpha = __shfl_sync(kFull, a[0][j], j);
        float tau, beta, scale;
        house_scalars(alpha, xx, tau, beta, scale);
        if (lane > j) a[0][j] *= scale;
#pragma unroll
        for (int q = 1; q < 4; ++q) a[q][j] *= scale;
        if (lane == j) mytau = tau;
        // v's entry in this lane's first row: the reflector below the
        // diagonal, its unit diagonal, zeros above
        const float v0 = (lane > j) ? a[0][j] : (lane == j ? 1.f : 0.f);
        if (j + 1 < kNB2) {
          float pd[kNB2];
#pragma unroll
          for (int col = 0; col < kNB2; ++col) {
            float d = (col > j) ? v0 * a[0][col] : 0.f;
#pragma unroll
            for (int q = 1; q < 4; ++q) d = (col > j) ? fmaf(a[q][j], a[q][col], d) : 0.f;
            pd[col] = d;
          }
          const float mine = reduce_scatter32(pd) * tau;   // tau v^T a_col for col = lane
#pragma unroll
          for (int col = j + 1; col < kNB2; ++col) {
            const float d = __shfl_sync(kFull, mine, col);
            a[0][col] = fmaf(-d, v0, a[0][col]);
#pragma unroll
            for (int q = 1; q < 4; ++q) a[q][col] = fmaf(-d, a[q][j], a[q][col]);
          }
        }
        if (lane == j) a[0][j] = beta;
      }
    }
    float* Rc = hs + c * kHrSlot;
#pragma unroll
    for (int col = 0; col < kNB2; ++col) Rc[lane * kNB2 + col] = (col >= lane) ? a[0][col] : 0.f;
    Rc[2 * kNB2 * kNB2 + lane] = mytau;   // chunk taus
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t row = lane + 32 * q;
      if (row < nrow) {
#pragma unroll
        for (int col = 0; col < kNB2; ++col)
          if (col < nbk) Y[base + row + (k + col) * ldy] = a[q][col];
      }
    }
  }
}

// Step 2a: merge the upper triangles Ra (left) and Rb (right): [Ra; Rb] =
// H [R; 0]; R replaces Ra, the reflectors' lower parts (column j: rows
// 0..j of the bottom half) replace Rb, their taus go to tn.  Lane = column.
__device__ void hr_merge(float* Ra, float* Rb, float* tn, int nbk) {
  const int lane = threadIdx.x & 31;
  float ra[kNB2], rb[kNB2];
#pragma unroll
  for (int r = 0; r < kNB2; ++r) {
    ra[r] = Ra[r * kNB2 + lane];
    rb[r] = (r <= lane) ? Rb[r * kNB2 + lane] : 0.f;
  }
  float mytau = 0.f;
#pragma unroll
  for (int j = 0; j < kNB2; ++j) {
    if (j < nbk) {
      float xo = 0.f;
#pragma unroll
      for (int r = 0; r <= j; ++r) xo = fmaf(rb[r], rb[r], xo);
      const float xx = __shfl_sync(kFull, xo, j);
      const float alpha = __shfl_sync(kFull, ra[j], j);
      float tau, beta, scale;
      house_scalars(alpha, xx, tau, beta, scale);
      float vb[kNB2];
#pragma unroll
      for (int r = 0; r <= j; ++r) vb[r] = __shfl_sync(kFull, rb[r], j) * scale;
      if (lane > j) {
        float d = ra[j];
#pragma unroll
        for (int r = 0; r <= j; ++r) d = fmaf(vb[r], rb[r], d);
        d *= tau;
        ra[j] -= d;
#pragma unroll
        for (int r = 0; r <= j; ++r) rb[r] = fmaf(-d, vb[r], rb[r]);
      }
      if (lane == j) {
        ra[j] = beta;
#pragma unroll
        for (int r = 0; r <= j; ++r) rb[r] = vb[r];
        mytau = tau;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kNB2; ++r) {
    Ra[r * kNB2 + lane] = ra[r];
    Rb[r * kNB2 + lane] = rb[r];
  }
  tn[lane] = mytau;
}

// Step 2b: [Bi; Bj] = H [Bi; 0] for the merge whose reflectors sit in Vn
// (H = H_0 ... H_{nbk-1}, applied last to first).  Lane = column.
__device__ void hr_down(float* Bi, float* Bj, const float* Vn, const float* tn, int nbk) {
  const int lane = threadIdx.x & 31;
  float xt[kNB2], xb[kNB2];
#pragma unroll
  for (int r = 0; r < kNB2; ++r) {
    xt[r] = Bi[r * kNB2 + lane];
    xb[r] = 0.f;
  }
#pragma unroll
  for (int j = kNB2 - 1; j >= 0; --j) {
    if (j < nbk) {
      const float tau = tn[j];
      float vb[kNB2];
#pragma unroll
      for (int r = 0; r <= j; ++r) vb[r] = Vn[r * kNB2 + j];
      float d = xt[j];
#pragma unroll
      for (int r = 0; r <= j; ++r) d = fmaf(vb[r], xb[r], d);
      d *= tau;
      xt[j] -= d;
#pragma unroll
      for (int r = 0; r <= j; ++r) xb[r] = fmaf(-d, vb[r], xb[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < kNB2; ++r) {
    Bi[r * kNB2 + lane] = xt[r];
    Bj[r * kNB2 + lane] = xb[r];
  }
}

// Step 2c: the chunk's rows of the explicit Q: H_chunk [B_c; 0], written
// over the chunk's reflectors.  Lane = rows lane + 32 q.
__device__ void hr_chunk_q(float* Y, int64_t ldy, int64_t k, int nbk, int64_t L, int64_t c, const float* hs) {
  const int lane = threadIdx.x & 31;
  const int64_t base = k + c * kCR;
  const int64_t nrow = (L - c * kCR) < kCR ? (L - c * kCR) : kCR;
  const float* Bc = hs + c * kHrSlot + kNB2 * kNB2;
  const float* tch = hs + c * kHrSlot + 2 * kNB2 * kNB2;
  float x[4][kNB2];
#pragma unroll
  for (int col = 0; col < kNB2; ++col) {
    x[0][col] = Bc[lane * kNB2 + col];
    x[1][col] = x[2][col] = x[3][col] = 0.f;
  }
  // reflector j's entries of this lane's rows, loaded two reflectors ahead
  // of their use so the loads' latency overlaps the applications
  auto load_v = [&](int j, float (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t row = lane + 32 * q;
      v[q] = (j < 0) ? 0.f : ((row == j) ? 1.f : ((row > j && row < nrow) ? Y[base + row + (k + j) * ldy] : 0.f));
    }
  };
  float v1[4], v2[4];
  load_v(nbk - 1, v1);
  load_v(nbk - 2, v2);
#pragma unroll 1
  for (int j = nbk - 1; j >= 0; --j) {
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = v1[q];
      v1[q] = v2[q];
    }
    load_v(j - 2, v2);
    const float tau = tch[j];
    float pd[kNB2];
#pragma unroll
    for (int col = 0; col < kNB2; ++col) {
      float d = v[0] * x[0][col];
#pragma unroll
      for (int q = 1; q < 4; ++q) d = fmaf(v[q], x[q][col], d);
      pd[col] = d;
    }
    const float mine = reduce_scatter32(pd) * tau;   // tau v^T x_col for col = lane
#pragma unroll
    for (int col = 0; col < kNB2; ++col) {
      const float d = __shfl_sync(kFull, mine, col);
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q][col] = fmaf(-d, v[q], x[q][col]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t row = lane + 32 * q;
    if (row < nrow) {
#pragma unroll
      for (int col = 0; col < kNB2; ++col)
        if (col < nbk) Y[base + row + (k + col) * ldy] = x[q][col];
    }
  }
}

// The panel [k, k + nbk) of the leaf (rows k .. h-1): reflectors below the
// diagonal, R on and above it, T (FP64, row-major) in sT, taus in tau_out.
// sf: >= 33 * 32 * 2 + 64 floats of shared memory; hs: the leaf's scratch
// (ceil((h - k) / 128) chunk slots).
__device__ void panel_tsqr_hr(float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, double* tau_out, double* sT,
                              float* sf, float* hs) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int64_t L = h - k;
  const int64_t nc = (L + kCR - 1) / kCR;
  hr_chunks(Y, ldy, k, nbk, L, nc, hs);
  __syncthreads();
  int64_t top = 0;
  for (int64_t st = 1; st < nc; st *= 2) {
    for (int64_t i = (int64_t)warp * 2 * st; i < nc; i += (int64_t)nw * 2 * st)
      if (i + st < nc) hr_merge(hs + i * kHrSlot, hs + (i + st) * kHrSlot, hs + (i + st) * kHrSlot + 2 * kNB2 * kNB2 + kNB2, nbk);
    top = st;
    __syncthreads();
  }
  // root R (row-major) to shared memory before the Q blocks overwrite nothing of it
  float* sU = sf;                      // 32 x 33: U of the LU, then reused
  float* sR = sf + 32 * 33;            // 32 x 33: root R
  float* sS = sR + 32 * 33;            // 32 signs
  float* sD = sS + 32;                 // 32 reciprocals of U's diagonal
  for (int idx = tid; idx < kNB2 * kNB2; idx += nthr) sR[(idx / kNB2) * 33 + idx % kNB2] = hs[idx];
  // B_0 = I
  for (int idx = tid; idx < kNB2 * kNB2; idx += nthr)
    hs[kNB2 * kNB2 + idx] = (idx / kNB2 == idx % kNB2 && idx % kNB2 < nbk) ? 1.f : 0.f;
  __syncthreads();
  for (int64_t st = top; st >= 1; st /= 2) {
    for (int64_t i = (int64_t)warp * 2 * st; i < nc; i += (int64_t)nw * 2 * st)
      if (i + st < nc)
        hr_down(hs + i * kHrSlot + kNB2 * kNB2, hs + (i + st) * kHrSlot + kNB2 * kNB2, hs + (i + st) * kHrSlot,
                hs + (i + st) * kHrSlot + 2 * kNB2 * kNB2 + kNB2, nbk);
    __syncthreads();
  }
  for (int64_t c = warp; c < nc; c += nw) hr_chunk_q(Y, ldy, k, nbk, L, c, hs);
  __syncthreads();
  // modified LU of the top block Q1 - S (warp 0, lane = column)
  if (warp == 0) {
    float q[kNB2];
#pragma unroll
    for (int r = 0; r < kNB2; ++r) q[r] = (r < nbk && lane < nbk) ? Y[k + r + (k + lane) * ldy] : 0.f;
#pragma unroll
    for (int j = 0; j < kNB2; ++j) {
      if (j < nbk) {
        const float pj = __shfl_sync(kFull, q[j], j);
        const float sj = pj >= 0.f ? -1.f : 1.f;
        const float u = pj - sj;                     // |u| >= 1
        if (lane == j) {
          q[j] = u;
#pragma unroll
          for (int r = j + 1; r < kNB2; ++r) q[r] /= u;
        }
        if (lane == 0) sS[j] = sj;
        float l[kNB2];
#pragma unroll
        for (int r = j + 1; r < kNB2; ++r) l[r] = __shfl_sync(kFull, q[r], j);
        if (lane > j) {
#pragma unroll
          for (int r = j + 1; r < kNB2; ++r) q[r] = fmaf(-l[r], q[j], q[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kNB2; ++r) sU[r * 33 + lane] = q[r];   // U on and above the diagonal, L1 below
    sD[lane] = (lane < nbk) ? 1.f / q[lane] : 0.f;
  }
  __syncthreads();
  // V rows below the top block: y = x U^-1 (a thread per row)
  for (int64_t i = k + nbk + tid; i < h; i += nthr) {
    float y[kNB2];
#pragma unroll
    for (int col = 0; col < kNB2; ++col) y[col] = (col < nbk) ? Y[i + (k + col) * ldy] : 0.f;
#pragma unroll
    for (int j = 0; j < kNB2; ++j) {
      if (j < nbk) {
        float acc = y[j];
#pragma unroll
        for (int l = 0; l < j; ++l) acc = fmaf(-y[l], sU[l * 33 + j], acc);
        y[j] = acc * sD[j];
      }
    }
#pragma unroll
    for (int col = 0; col < kNB2; ++col)
      if (col < nbk) Y[i + (k + col) * ldy] = y[col];
  }
  // top block: V1 strictly below the diagonal, R = S R_tsqr on and above it
  for (int idx = tid; idx < nbk * nbk; idx += nthr) {
    const int r = idx % nbk, col = idx / nbk;
    Y[k + r + (k + col) * ldy] = (r > col) ? sU[r * 33 + col] : sS[r] * sR[r * 33 + col];
  }
  // T = -U S V1^-T in FP64 (warp 0, lane = column): Z = V1^-T by back
  // substitution of V1^T Z = I, then T[p][c] = -sum_m U[p][m] s_m Z[m][c]
  if (warp == 0) {
    double z[kNB2];
#pragma unroll
    for (int r = kNB2 - 1; r >= 0; --r) {
      double acc = (r == lane) ? 1.0 : 0.0;
#pragma unroll
      for (int m = r + 1; m < kNB2; ++m) acc -= (double)sU[m * 33 + r] * z[m];   // V1[m][r]
      z[r] = (r <= lane && r < nbk && lane < nbk) ? acc : 0.0;
    }
#pragma unroll
    for (int p = 0; p < kNB2; ++p) {
      double acc = 0.0;
#pragma unroll
      for (int m = p; m < kNB2; ++m) acc += (double)sU[p * 33 + m] * (double)sS[m] * z[m];
      sT[p * kNB2 + lane] = (p <= lane && lane < nbk) ? -acc : 0.0;
    }
    if (lane < nbk) tau_out[lane] = -(double)sU[lane * 33 + lane] * (double)sS[lane];
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

// The W stage's 3xTF32 product in two MMAs per K-slice: the B tile holds
// the hi rows (reflectors 0..31) followed by the lo rows (32..63), so one
// N = 64 MMA gives hi*hi (accumulator columns 0..31) and hi*lo (32..63), and
// an N = 32 MMA gives lo*hi into d_x2 (two MMAs of 3xTF32 work per K-slice
// instead of three).
__device__ __forceinline__ void issue_w_3xtf32(uint32_t d_wide, uint32_t d_x2, unsigned char* smem, int Kk) {
  using namespace tc05;
  const uint32_t a_hi = smem_u32(smem + kOffWA), a_lo = smem_u32(smem + kOffWAlo);
  const uint32_t b_hi = smem_u32(smem + kOffWB);
  static_assert(kOffWBlo == kOffWB + kWB, "the lo rows of B follow its hi rows");
  const uint32_t sbo = (uint32_t)(Kk / 4) * 128, lbo = 128;
  for (int kk = 0; kk < Kk / 8; ++kk) {
    const uint32_t o = (uint32_t)kk * 256;
    mma_tf32(d_wide, desc(a_hi + o, lbo, sbo), desc(b_hi + o, lbo, sbo), idesc_tf32(128, 2 * kNB2), kk > 0);
    mma_tf32(d_x2, desc(a_lo + o, lbo, sbo), desc(b_hi + o, lbo, sbo), idesc_tf32(128, kNB2), kk > 0);
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
// The TMA form of the W stage (TMA = true: the factorisation's trailing
// updates, C and V both columns of the leaf's FP32 working copy): per 64-row
// step one cp.async.bulk.tensor box of the C chunk and one of the panel land
// in a two-stage shared-memory ring, two steps ahead of the MMAs; the threads
// split them into the TF32 operand tiles from shared memory.  tmC / tmV: the
// working copy's tensor maps (boxes of kTmaRows rows x 128 / 32 columns);
// grow0: the working-copy row of the leaf's row 0; ccol0: the working-copy
// column of C's column 0; fullbar[2] / tphase: the ring's mbarriers and
// their phase bits.
struct TmaW {
  const CUtensorMap* tmC;
  const CUtensorMap* tmV;
  int64_t grow0, ccol0;
  uint64_t* fullbar;
  uint32_t* tphase;
};

// wh >= 0 (register path): C is zero from leaf row wh on, so the W stage
// sums rows k..wh-1 only.
template <bool TRANS, bool TMA = false>
__device__ bool block_reflector_tc(const float* Y, int64_t ldy, int64_t k, int nbk, int64_t h, float* C,
                                   int64_t ldc, int ncols, const double* sT, unsigned char* smem, uint32_t tmem,
                                   uint64_t* mbar, uint32_t& phase, TmaW tw = TmaW{}, int64_t wh = -1) {
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
    const int64_t Lw = (!TMA && wh > k && wh < h) ? wh - k : L;
    const int64_t nkc = (Lw + kKC - 1) / kKC;
    // staging map: warp instruction u of warp w covers core matrix u * 8 + w
    // of the operand (8 operand rows x 4 K elements, 128 contiguous bytes of
    // shared memory), so the split stores are free of bank conflicts; lane l
    // holds operand row 8 g + l / 4 and K element 4 q + l % 4 of it
    const int lrow = lane >> 2, lk = lane & 3;
    // the MMA and fold of one step, common to both forms
    auto mma_and_fold = [&]() -> bool {
      const bool w_ok = mbar_wait(mbar, phase);
      phase ^= 1u;
      fence_after();
      if (__syncthreads_or(!w_ok)) return false;
      float hh[16], x1[16], x2[16];
      tmem_ld16(tmem + lanebase + (uint32_t)(16 * half), hh);
      tmem_ld16(tmem + lanebase + (uint32_t)(kNB2 + 16 * half), x1);
      tmem_ld16(tmem + lanebase + (uint32_t)(2 * kNB2 + 16 * half), x2);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float y = (hh[j] + (x1[j] + x2[j])) - wc_[j];
        const float t = ws_[j] + y;
        wc_[j] = (t - ws_[j]) - y;
        ws_[j] = t;
      }
      // the next step's MMAs overwrite the accumulators only after the
      // barrier that follows its shared-memory stores
      fence_before();
      return true;
    };
    if constexpr (TMA) {
      // every thread's earlier global writes (the panel, the previous
      // updates of C) are ordered before the tensor-memory-access reads
      asm volatile("fence.proxy.async;" ::: "memory");
      __syncthreads();
      // steps cover working-copy rows xa + 64 kc .. xa + 64 kc + 63 from the
      // panel's first row rounded down to a multiple of 4; rows of a step
      // outside the panel's rows k .. h-1 (up to 3 above it, the ragged end
      // below it, the other leaves' rows, rows past N read as zeros) meet a
      // zero reflector entry, so the C tile is taken whole and only the
      // reflector operand is masked
      const int64_t xa = (tw.grow0 + k) & ~int64_t(3);
      const int64_t ioff = xa - tw.grow0;          // leaf row of a step's first row, minus 64 kc
      const int64_t nkt = (tw.grow0 + h - xa + kKC - 1) / kKC;
      auto issue = [&](int64_t kc) {   // thread 0
        const int st = (int)(kc & 1);
        const int32_t x0 = (int32_t)(xa + kc * kKC);
        unsigned char* dst = smem + kOffRaw + st * kStageBytes;
        fence_smem_async();
        mbar_arrive_expect_tx(&tw.fullbar[st], (uint32_t)kStageBytes);
        tma_load_2d(dst, tw.tmC, x0, (int32_t)(tw.ccol0 + c0), &tw.fullbar[st]);
        tma_load_2d(dst + kRawC, tw.tmV, x0, (int32_t)k, &tw.fullbar[st]);
      };
      if (tid == 0) {
        issue(0);
        if (nkt > 1) issue(1);
      }
      int64_t issued = nkt > 1 ? 2 : 1, consumed = 0;
      // A-operand map: warp instruction u of warp w and lane 8 q + j move the
      // 16 bytes (4 K elements) of operand row c = 8 cg + j, K group
      // g = 8 gg + (j + s) % 8, with 32 u + 4 w + q = cg + 16 gg + 32 s: eight
      // lanes read eight different 16-byte bank groups of the box and write
      // eight different ones of the core-matrix tile
      const int jl = lane & 7, ql = lane >> 3;
      for (int64_t kc = 0; kc < nkt && ok; ++kc) {
        const int st = (int)(kc & 1);
        const bool got = mbar_wait(&tw.fullbar[st], (*tw.tphase >> st) & 1u);
        *tw.tphase ^= 1u << st;
        ++consumed;
        ok = !__syncthreads_or(!got);
        if (!ok) break;
        const float* rc = (const float*)(smem + kOffRaw + st * kStageBytes);
        const float* rv = rc + kTmaRows * kCH;
#pragma unroll 2
        for (int u = 0; u < 8; ++u) {
          const int wq = u * 32 + warp * 4 + ql;
          const int cg = wq & 15, gg = (wq >> 4) & 1, sh = wq >> 5;
          const int c = cg * 8 + jl, g = gg * 8 + ((jl + sh) & 7);
          const float4 x = *(const float4*)(rc + c * kTmaRows + 4 * g);
          float4 hi, lo;
          split_tf32(x.x, hi.x, lo.x);
          split_tf32(x.y, hi.y, lo.y);
          split_tf32(x.z, hi.z, lo.z);
          split_tf32(x.w, hi.w, lo.w);
          const uint32_t o = cm_off(c, 4 * g, kKC);
          *(float4*)(smem + kOffWA + o) = hi;
          *(float4*)(smem + kOffWAlo + o) = lo;
        }
        const int64_t ibase = ioff + kc * kKC;    // leaf row of K element 0
        // B operand (32 reflectors x 64 K), the same map on 4 row groups:
        // entry (i, p) of the panel's reflector matrix -- zero above the
        // diagonal and past the leaf, one on it
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int wq = u * 32 + warp * 4 + ql;
          const int cg = wq & 3, gg = (wq >> 2) & 1, sh = wq >> 3;
          const int pp = cg * 8 + jl, g = gg * 8 + ((jl + sh) & 7);
          const float4 raw = *(const float4*)(rv + pp * kTmaRows + 4 * g);
          const int64_t d = k + pp;
          const int64_t i0 = ibase + 4 * g;
          float x[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t i = i0 + e;
            x[e] = (pp < nbk && i < h && i >= d) ? ((i == d) ? 1.f : x[e]) : 0.f;
          }
          float4 hi, lo;
          split_tf32(x[0], hi.x, lo.x);
          split_tf32(x[1], hi.y, lo.y);
          split_tf32(x[2], hi.z, lo.z);
          split_tf32(x[3], hi.w, lo.w);
          const uint32_t o = cm_off(pp, 4 * g, kKC);
          *(float4*)(smem + kOffWB + o) = hi;
          *(float4*)(smem + kOffWBlo + o) = lo;
        }
        fence_smem_async();
        fence_before();
        __syncthreads();     // the stage is read out: it may be refilled
        fence_after();
        if (tid == 0) {
          if (kc + 2 < nkt) issue(kc + 2);
          issue_w_3xtf32(tmem, tmem + 2 * kNB2, smem, kKC);
          commit(mbar);
        }
        if (kc + 2 < nkt) ++issued;
        ok = mma_and_fold();
      }
      if (!ok) {
        // wait (bounded) for the boxes still in flight before giving up
        if (tid == 0)
          for (int64_t q = consumed; q < issued; ++q) {
            const int st = (int)(q & 1);
            mbar_wait(&tw.fullbar[st], (*tw.tphase >> st) & 1u);
            *tw.tphase ^= 1u << st;
          }
        break;
      }
    } else {
      float xa[kCH / 4], xb[kNB2 / 4];
      auto load_w = [&](int64_t kc) {
#pragma unroll
        for (int u = 0; u < kCH / 4; ++u) {          // A: 16 row groups x 16 K groups
          const int cmi = u * 8 + warp;
          const int c = (cmi & 15) * 8 + lrow;
          const int64_t row = k + kc * kKC + (cmi >> 4) * 4 + lk;
          xa[u] = (row < h && c < wc) ? C[row + (int64_t)(c0 + c) * ldc] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kNB2 / 4; ++u) {         // B: 4 reflector groups x 16 K groups
          const int cmi = u * 8 + warp;
          const int64_t row = k + kc * kKC + (cmi >> 2) * 4 + lk;
          xb[u] = vval_f(Y, ldy, k, nbk, h, row, (cmi & 3) * 8 + lrow);
        }
      };
      load_w(0);
      for (int64_t kc = 0; kc < nkc && ok; ++kc) {
#pragma unroll
        for (int u = 0; u < kCH / 4; ++u) {
          const int cmi = u * 8 + warp;
          float hi, lo;
          split_tf32(xa[u], hi, lo);
          const uint32_t o = cm_off((cmi & 15) * 8 + lrow, (cmi >> 4) * 4 + lk, kKC);
          *(float*)(smem + kOffWA + o) = hi;
          *(float*)(smem + kOffWAlo + o) = lo;
        }
#pragma unroll
        for (int u = 0; u < kNB2 / 4; ++u) {
          const int cmi = u * 8 + warp;
          float hi, lo;
          split_tf32(xb[u], hi, lo);
          const uint32_t o = cm_off((cmi & 3) * 8 + lrow, (cmi >> 2) * 4 + lk, kKC);
          *(float*)(smem + kOffWB + o) = hi;
          *(float*)(smem + kOffWBlo + o) = lo;
        }
        fence_smem_async();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
          issue_w_3xtf32(tmem, tmem + 2 * kNB2, smem, kKC);
          commit(mbar);
        }
        if (kc + 1 < nkc) load_w(kc + 1);   // in flight while the MMAs run
        ok = mma_and_fold();
      }
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
    // V tile: thread t stages row t of the tile (whole 128-byte reflector
    // rows from global memory; a core-matrix-ordered map was slower here)
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
    // kPro independent loads in flight per thread (one 8-warp CTA per SM)
    constexpr int kPro = 16;
    double xbar = 0.0;
    if (a.remove_mean) {
      double sum = 0.0;
      for (int64_t m0 = 0; m0 < M; m0 += kPro) {
        double xv[kPro];
#pragma unroll
        for (int u = 0; u < kPro; ++u) xv[u] = (m0 + u < M) ? (double)X[n + (m0 + u) * a.ldx] : 0.0;
#pragma unroll
        for (int u = 0; u < kPro; ++u) sum += xv[u];
      }
      xbar = sum / (double)M;
    }
    if (a.mean) a.mean[n] = xbar;
    double sw = 1.0;
    if (a.w) {
      const double wn = a.w[n];
      if (!(wn > 0.0) || !isfinite(wn)) bad = 1;
      sw = sqrt(wn);
    }
    for (int64_t m0 = 0; m0 < M; m0 += kPro) {
      double xv[kPro];
#pragma unroll
      for (int u = 0; u < kPro; ++u) xv[u] = (m0 + u < M) ? (double)X[n + (m0 + u) * a.ldx] : 0.0;
#pragma unroll
      for (int u = 0; u < kPro; ++u) {
        if (m0 + u < M) {
          if (!isfinite(xv[u])) bad = 1;
          Y[i + (m0 + u) * ldy] = (float)(sw * (xv[u] - xbar));
        }
      }
    }
  }
  if (bad) raise_status(a.s.hdr, PYLOM_ERR_NONFINITE);
}

// Binary32 snapshots: the same Y without per-element binary64 work (on this
// GPU two conversions, an add, a subtract and a multiply in the binary64
// pipe per sample cost a fifth of the leaf kernel at M = 256).  The mean is
// summed in chunks of kPro by compensated binary32 sums (sum32_compensated)
// whose pairs are added in binary64; the binary64 mean and sqrt(w) are then
// split into binary32 pairs (hi + lo, 48 significant bits), x - mean is
// formed as d + e by TwoSum and the rest of the mean folded into e, and the
// product with sqrt(w) is rounded once more by two FMAs: Y is within a few
// units in the last place of fl32(sqrt(w) (x - mean)) in binary64.
__device__ void mixed_prologue_f32(const MixedArgs& a, float* Y, int64_t ldy, int64_t r0, int64_t h) {
  const float* X = (const float*)a.X;
  const int64_t M = a.s.M;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < h; i += blockDim.x) {
    const int64_t n = r0 + i;
    const float* xr = X + n;
    constexpr int kPro = 16;
    double xbar = 0.0;
    if (a.remove_mean) {
      double acc = 0.0;
      for (int64_t m0 = 0; m0 < M; m0 += kPro) {
        float xv[kPro];
#pragma unroll
        for (int u = 0; u < kPro; ++u) xv[u] = (m0 + u < M) ? xr[(m0 + u) * a.ldx] : 0.f;
        float s, c;
        sum32_compensated(xv, s, c);
        acc += (double)s + (double)c;
      }
      xbar = acc / (double)M;
    }
    if (a.mean) a.mean[n] = xbar;
    double sw = 1.0;
    if (a.w) {
      const double wn = a.w[n];
      if (!(wn > 0.0) || !isfinite(wn)) bad = 1;
      sw = sqrt(wn);
    }
    const float xh = (float)xbar, xl = (float)(xbar - (double)xh);
    const float sh = (float)sw, sl = (float)(sw - (double)sh);
    for (int64_t m0 = 0; m0 < M; m0 += kPro) {
      float xv[kPro];
#pragma unroll
      for (int u = 0; u < kPro; ++u) xv[u] = (m0 + u < M) ? xr[(m0 + u) * a.ldx] : 0.f;
#pragma unroll
      for (int u = 0; u < kPro; ++u) {
        if (m0 + u < M) {
          if (!isfinite(xv[u])) bad = 1;
          float d, e;
          two_sum32(xv[u], -xh, d, e);
          const float lo = __fsub_rn(e, xl);
          Y[i + (m0 + u) * ldy] = __fmaf_rn(d, sh, __fmaf_rn(d, sl, __fmul_rn(lo, sh)));
        }
      }
    }
  }
  if (bad) raise_status(a.s.hdr, PYLOM_ERR_NONFINITE);
}

__global__ void __launch_bounds__(kMxThreads) leaf_qr_mixed_kernel(MixedArgs a, const __grid_constant__ CUtensorMap tmC,
                                                                  const __grid_constant__ CUtensorMap tmV) {
  extern __shared__ __align__(128) unsigned char msm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t fullbar[2];
  __shared__ uint32_t tmem_base;
  const TsqrState& s = a.s;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t leaf = blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M, ldy = yf_ld(s.N);
  const int64_t npan = (M + kNB2 - 1) / kNB2;
  float* Y = a.Yf + r0;
  double* sT = (double*)(msm + kOffT);
  if (a.xtype == PYLOM_F32)
    mixed_prologue_f32(a, Y, ldy, r0, h);
  else
    mixed_prologue<double>(a, Y, ldy, r0, h);
  if (tid == 0) {
    tc05::mbar_init(&mbar, 1);
    tc05::mbar_init(&fullbar[0], 1);
    tc05::mbar_init(&fullbar[1], 1);
  }
  uint32_t tphase = 0;
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
    panel_tsqr_hr(Y, ldy, k, nbk, h, s.tau + leaf * M + k, sT, (float*)msm, a.Pb + (r0 / kCR + leaf) * kHrSlot);
    __syncthreads();
    double* Tg = a.T2 + (leaf * npan + k / kNB2) * kNB2 * kNB2;
    for (int idx = tid; idx < kNB2 * kNB2; idx += blockDim.x) Tg[idx] = sT[idx];
    if (k + nbk < M)
      ok = block_reflector_tc<true, true>(Y, ldy, k, nbk, h, Y + (k + nbk) * ldy, ldy, (int)(M - k - nbk), sT, msm,
                                          tmem, &mbar, phase, TmaW{&tmC, &tmV, r0, k + nbk, fullbar, &tphase});
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
    // the first panel applied meets [B; 0]: its W stage sums rows k..M-1 only
    ok = block_reflector_tc<false>(Y, yf_ld(s.N), k, nbk, h, C, ldu, (int)r, sT, msm, tmem, &mbar, phase, TmaW{},
                                   pan == npan - 1 ? M : -1);
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
    ok = block_reflector_tc<true>(Y, yf_ld(s.N), k, nbk, h, Cl, s.N, (int)r, sT, msm, tmem, &mbar, phase);
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
  return align256(sizeof(float) * (size_t)yf_ld(N) * M) + align256(sizeof(double) * (size_t)P * npan * kNB2 * kNB2) +
         align256(sizeof(float) * (size_t)(N / kCR + P + 1) * kHrSlot);
}

// Tensor map of the FP32 working copy (N x M, column-major, leading
// dimension yf_ld(N)) with boxes of kTmaRows rows x `cols` columns;
// out-of-range parts of a box read zeros.
static cudaError_t encode_yf_map(CUtensorMap* map, float* Yf, int64_t N, int64_t M, int cols) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess) return e;
      if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
      encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
  }
  // rows past N (the padding of the leading dimension) are out of range:
  // they read as zeros, never as uninitialised memory
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)yf_ld(N) * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTmaRows, (cuuint32_t)cols};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)Yf, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tsqr_mixed(const TsqrState& s, char* extra, const void* X, int64_t ldx, int xtype,
                              const double* w, int remove_mean, double* mean, cudaStream_t st, cudaEvent_t mid) {
  cudaError_t e;
  if ((e = ensure_dyn_smem((const void*)leaf_qr_mixed_kernel, kMixSmemTotal)) != cudaSuccess) return e;
  if ((e = ensure_dyn_smem((const void*)modes_mixed_kernel, kMixSmemTotal)) != cudaSuccess) return e;
  const int64_t npan = (s.M + kNB2 - 1) / kNB2;
  char* t2 = extra + align256(sizeof(float) * (size_t)yf_ld(s.N) * s.M);
  char* pb = t2 + align256(sizeof(double) * (size_t)s.P * npan * kNB2 * kNB2);
  MixedArgs a{s, (float*)extra, (double*)t2, (float*)pb, X, ldx, xtype, w, remove_mean, mean};
  CUtensorMap tmC, tmV;
  if ((e = encode_yf_map(&tmC, a.Yf, s.N, s.M, kCH)) != cudaSuccess) return e;
  if ((e = encode_yf_map(&tmV, a.Yf, s.N, s.M, kNB2)) != cudaSuccess) return e;
  leaf_qr_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(a, tmC, tmV);
  e = cudaGetLastError();
  if (e == cudaSuccess && mid) e = cudaEventRecord(mid, st);
  if (e != cudaSuccess || s.climb) return e;
  return launch_tree(s, st);
}

cudaError_t launch_modes_mixed(const TsqrState& s, char* extra, const double* Ur, int64_t ldur, int64_t r_fixed,
                               const double* w, int physical, float* U, int64_t ldu, int64_t* r_out, cudaStream_t st,
                               cudaEvent_t mid) {
  cudaError_t e = launch_down_pass_fp64(s, Ur, ldur, r_fixed, st);
  if (e != cudaSuccess) return e;
  if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
  const float* Yf = (const float*)extra;
  const double* T2 = (const double*)(extra + align256(sizeof(float) * (size_t)yf_ld(s.N) * s.M));
  modes_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(s, Yf, T2, r_fixed, w, physical, U, ldu, r_out);
  return cudaGetLastError();
}

cudaError_t launch_leaf_qt_mixed(const TsqrState& s, char* extra, float* C, int64_t r, double* Z, cudaStream_t st) {
  {
    cudaError_t e = ensure_dyn_smem((const void*)leaf_qt_mixed_kernel, kMixSmemTotal);
    if (e == cudaSuccess) e = ensure_dyn_smem((const void*)modes_mixed_kernel, kMixSmemTotal);
    if (e != cudaSuccess) return e;
  }
  const float* Yf = (const float*)extra;
  const double* T2 = (const double*)(extra + align256(sizeof(float) * (size_t)yf_ld(s.N) * s.M));
  leaf_qt_mixed_kernel<<<(unsigned)s.P, kMxThreads, kMixSmemTotal, st>>>(s, Yf, T2, C, r, Z);
  return cudaGetLastError();
}

}  // namespace pylom

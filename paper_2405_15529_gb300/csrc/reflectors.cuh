// reflectors.cuh -- shared device code of the FP64 TSQR kernels: the
// shared-memory plan of a leaf-sized block, the reflector accessors of leaf
// panels and tree-node panels, and the block-reflector application on the
// FP64 tensor pipe.  Included by tsqr_fp64.cu and pod_backward.cu.
#pragma once
#include "kernels.h"

namespace pylom {

constexpr int kLeafThreads = 256;
constexpr int kCW = 256;   // column chunk of a block-reflector application
constexpr int kTPW = 4;    // 8-column tiles per warp in W = V^T C

// Shared-memory plan of the leaf / modes kernels (doubles).
constexpr int kSmT = kNB * kNB;
constexpr int kSmRed = kNB * 32;
constexpr int kSmOut = 32;
constexpr int kSmW = kNB * kCW;
constexpr size_t kLeafSmemBytes = sizeof(double) * (kSmT + kSmRed + kSmOut + 2 * kSmW);

// Entry (i, p) of a leaf panel's reflector matrix V (panel starts at
// column k, nbk reflectors, h rows): zero above the diagonal, one on it,
// stored below.
struct LeafV {
  const double* A;
  int64_t lda, k, h;
  int nbk;
  __device__ __forceinline__ double operator()(int64_t i, int p) const {
    if (p >= nbk || i >= h) return 0.0;
    const int64_t d = k + p;
    if (i < d) return 0.0;
    if (i == d) return 1.0;
    return A[i + d * lda];
  }
};

// Bottom half of a tree-node panel's reflectors: reflector c = k + p is
// [e_c (top); u_c (bottom rows 0..c)] and u_c is stored in column c of the
// right child's slot.  Loads bypass L1 (the slot was written by another
// block).  The e_c halves are the identity "top" block of the application.
struct MergeV {
  const double* Rb;
  int64_t M, k;
  int nbk;
  __device__ __forceinline__ double operator()(int64_t i, int p) const {
    if (p >= nbk) return 0.0;
    const int64_t c = k + p;
    return (i <= c) ? ldcg(Rb + i + c * M) : 0.0;
  }
};

template <bool CG>
__device__ __forceinline__ double ld_c(const double* p) {
  if (CG) return ldcg(p);
  return *p;
}

// C[r0:r1, 0:ncols] := (I - V op(T) V^T) C[r0:r1, 0:ncols] with op(T) = T^T
// (TRANS: applies Q_panel^T, the factorisations' trailing update) or T
// (applies Q_panel, the modes product).  V(i, p) comes from the functor.  If
// `top` is given, the panel's reflectors also carry an identity block acting
// on the nbk rows top[0:nbk, 0:ncols] (ld ldtop): the tree-node case.
// The contractions W = V^T C and C -= V W' run on the FP64 tensor pipe
// (mma.sync m8n8k4); W is reduced over row slices in a fixed order, so
// results are bitwise repeatable.  CG: load C through L2 only.  wr1 >= 0:
// C is zero from row wr1 on, so W sums rows r0..wr1-1 only.
template <bool TRANS, bool CG, class VF>
__device__ void block_reflector(const VF& V, int nbk, int64_t r0, int64_t r1, double* C, int64_t ldc,
                                int ncols, double* top, int64_t ldtop, const double* sT, double* sW,
                                double* sWp, int64_t wr1 = -1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t L = r1 - r0;
  const int64_t r1w = (wr1 >= r0 && wr1 < r1) ? wr1 : r1;   // rows of the W sums
  const int64_t nsteps = (r1w - r0 + 3) / 4;
  for (int c0 = 0; c0 < ncols; c0 += kCW) {
    const int wc = min(kCW, ncols - c0);
    const int NT = (wc + 7) / 8;
    const int G = (NT + kTPW - 1) / kTPW;
    const int S = (G >= nwarps) ? 1 : nwarps / G;
    const int WcP = G * kTPW * 8;
    // phase 1: partial W = V^T C over S slices of the rows
    for (int u = warp; u < G * S; u += nwarps) {
      const int gi = u % G, si = u / G;
      const int64_t sb = (nsteps * si) / S, se = (nsteps * (si + 1)) / S;
      double acc[2][kTPW][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int tt = 0; tt < kTPW; ++tt) acc[mt][tt][0] = acc[mt][tt][1] = 0.0;
      for (int64_t stp = sb; stp < se; ++stp) {
        const int64_t row = r0 + stp * 4 + t;
        const bool rok = row < r1w;
        const double a0 = rok ? V(row, g) : 0.0;
        const double a1 = rok ? V(row, 8 + g) : 0.0;
#pragma unroll
        for (int tt = 0; tt < kTPW; ++tt) {
          const int col = (gi * kTPW + tt) * 8 + g;
          const double b = (rok && col < wc) ? ld_c<CG>(C + row + (int64_t)(c0 + col) * ldc) : 0.0;
          dmma884(acc[0][tt][0], acc[0][tt][1], a0, b);
          dmma884(acc[1][tt][0], acc[1][tt][1], a1, b);
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int tt = 0; tt < kTPW; ++tt) {
          const int p = mt * 8 + g;
          const int col = (gi * kTPW + tt) * 8 + 2 * t;
          sWp[(si * kNB + p) * WcP + col] = acc[mt][tt][0];
          sWp[(si * kNB + p) * WcP + col + 1] = acc[mt][tt][1];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kNB * WcP; idx += blockDim.x) {
      double s = 0.0;
      for (int si = 0; si < S; ++si) s += sWp[si * kNB * WcP + idx];
      if (top) {
        const int p = idx / WcP, col = idx - p * WcP;
        if (p < nbk && col < wc) s += ld_c<true>(top + p + (int64_t)(c0 + col) * ldtop);
      }
      sW[idx] = s;
    }
    __syncthreads();
    // phase 2: sWp = -op(T) W
    for (int idx = threadIdx.x; idx < kNB * WcP; idx += blockDim.x) {
      const int p = idx / WcP, col = idx - p * WcP;
      double s = 0.0;
      if (TRANS) {
        for (int q = 0; q <= p; ++q) s += sT[q * kNB + p] * sW[q * WcP + col];
      } else {
        for (int q = p; q < kNB; ++q) s += sT[p * kNB + q] * sW[q * WcP + col];
      }
      sWp[idx] = -s;
    }
    __syncthreads();
    if (top) {
      for (int idx = threadIdx.x; idx < nbk * wc; idx += blockDim.x) {
        const int p = idx / wc, col = idx - p * wc;
        double* tp = top + p + (int64_t)(c0 + col) * ldtop;
        *tp = ld_c<true>(tp) + sWp[p * WcP + col];
      }
    }
    // phase 3: C += V (-W')
    const int64_t nrt = (L + 7) / 8;
    for (int64_t rt = warp; rt < nrt; rt += nwarps) {
      const int64_t i0 = r0 + rt * 8;
      const int64_t row = i0 + g;
      const bool rok = row < r1;
      double a[4];
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) a[ks] = rok ? V(row, ks * 4 + t) : 0.0;
      for (int ct = 0; ct < NT; ++ct) {
        const int col = ct * 8 + 2 * t;
        double* cp = C + row + (int64_t)(c0 + col) * ldc;
        double d0 = (rok && col < wc) ? ld_c<CG>(cp) : 0.0;
        double d1 = (rok && col + 1 < wc) ? ld_c<CG>(cp + ldc) : 0.0;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          dmma884(d0, d1, a[ks], sWp[(ks * 4 + t) * WcP + ct * 8 + g]);
        if (rok && col < wc) cp[0] = d0;
        if (rok && col + 1 < wc) cp[ldc] = d1;
      }
    }
    __syncthreads();
  }
}

// Panel factorisation of columns [k, k+nbk) of the stacked pair [Rt; Rb]
// of two upper-triangular M x M factors (the buffer C of Alg. 1, receiver's
// R on top).  Reflector c touches only row c of the top and rows 0..c of the
// bottom: v_c = [e_c; u_c], u_c stored in column c of Rb (rows 0..c), the
// merged R overwrites Rt.  T (row-major, upper) follows the same forward
// recurrence as the leaves, with v_p^T v_c = u_p^T u_c (the e parts are
// disjoint).  Loads bypass L1: the partner's slot was written by another
// block.  sout needs 2 kNB doubles.
static __device__ void merge_panel_factor(double* Rt, double* Rb, int64_t M, int64_t k, int nbk,
                                   double* tau_out, double* sT, double* sred, double* sout) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  double* sd = sout + kNB;   // tau_c * (v_c^T column) of the panel columns
  double xx;
  {
    double v[1] = {0.0};
    for (int64_t i = tid; i <= k; i += nthr) {
      const double a = ldcg(Rb + i + k * M);
      v[0] += a * a;
    }
    block_sum<1>(v, sred, sout);
    xx = sout[0];
  }
  for (int jj = 0; jj < nbk; ++jj) {
    const int64_t c = k + jj;
    // thread 0 forms the reflector's scalars (FP64 square roots and divisions
    // are slow on this part; every thread repeating them cost more than the
    // column's dot products) and broadcasts them
    if (tid == 0) {
      const double alpha = ldcg(Rt + c + c * M);
      double tau0 = 0.0, beta0 = alpha, scale0 = 0.0;
      if (xx != 0.0) {
        const double nrm = sqrt(alpha * alpha + xx);
        beta0 = (alpha >= 0.0) ? -nrm : nrm;
        tau0 = (beta0 - alpha) / beta0;
        scale0 = 1.0 / (alpha - beta0);
      }
      sd[kNB - 3] = tau0;
      sd[kNB - 2] = beta0;
      sd[kNB - 1] = scale0;
    }
    __syncthreads();
    const double tau_c = sd[kNB - 3], beta = sd[kNB - 2], scale = sd[kNB - 1];
    __syncthreads();
    // pass A: u_c = scale * bottom column c; dots of u_c with the bottom part
    // of the later panel columns (q > jj) and with earlier reflectors (q < jj)
    double acc[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) acc[q] = 0.0;
    for (int64_t i = tid; i <= c; i += nthr) {
      const double u = ldcg(Rb + i + c * M) * scale;
      Rb[i + c * M] = u;
#pragma unroll
      for (int q = 0; q < kNB; ++q)
        if (q < nbk && q != jj) acc[q] += u * ldcg(Rb + i + (k + q) * M);
    }
    static_assert(kNB == 16, "the reduce-scatter sums 16 panel columns");
    block_sum16(acc, sred, sout);
    // column jj of T, one row per thread (rows 0..jj-1)
    if (tid < jj) {
      double s = 0.0;
      for (int q = tid; q < jj; ++q) s += sT[tid * kNB + q] * sout[q];
      sT[tid * kNB + jj] = -tau_c * s;
    }
    if (tid == 0) {
      Rt[c + c * M] = beta;
      tau_out[jj] = tau_c;
      sT[jj * kNB + jj] = tau_c;
    }
    if (tid > jj && tid < nbk) {
      // the e_c part of v_c contributes the top entry Rt[c, k+q]
      double* tp = Rt + c + (k + tid) * M;
      const double d = (sout[tid] + ldcg(tp)) * tau_c;
      sd[tid] = d;
      *tp = ldcg(tp) - d;
    }
    __syncthreads();
    // pass B: bottom rows 0..c of the later panel columns; squared norm of
    // the next column's bottom rows 0..c+1
    double nx[1] = {0.0};
    if (jj + 1 < nbk) {
      for (int64_t i = tid; i <= c + 1; i += nthr) {
        const double u = (i <= c) ? ldcg(Rb + i + c * M) : 0.0;
#pragma unroll
        for (int q = 0; q < kNB; ++q) {
          if (q > jj && q < nbk) {
            double* bp = Rb + i + (k + q) * M;
            double a = ldcg(bp);
            if (i <= c) {
              a -= sd[q] * u;
              *bp = a;
            }
            if (q == jj + 1) nx[0] += a * a;
          }
        }
      }
    }
    block_sum<1>(nx, sred, sout);
    xx = sout[0];
  }
}

// The same panel factorisation with the panel staged in shared memory: the
// bottom rows 0 .. k+nbk-1 of the panel columns of Rb and the kNB x kNB top
// block of Rt are loaded once, the column steps run from shared memory (no
// L2 round trip per column) on four warps -- one per SM sub-partition, so
// the panel's FP64 FMAs use every FP64 unit of the SM -- synchronised by a
// 128-thread named barrier three times per column, and the panel is written
// back.  The arithmetic is the column sweep above, term for term; only the
// order of the partial sums differs.  The other warps of the block wait.
// sP: (k + nbk) * kNB + kNB * kNB + kMergeStageExtra doubles of shared memory.
constexpr int kMergeStageExtra = 4 * kNB + 4 + 4 + 2 * kNB;
constexpr int kMergeStageThreads = 128;
constexpr int64_t kMergeStageDoubles = 2 * kSmW;   // the sW / sWp buffers, free while a panel is factored
__host__ __device__ constexpr bool merge_panel_staged(int64_t M) {
  return M * kNB + kNB * kNB + kMergeStageExtra <= kMergeStageDoubles;
}

__device__ __forceinline__ void stage_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

static __device__ void merge_panel_factor_staged(double* Rt, double* Rb, int64_t M, int64_t k, int nbk,
                                                 double* tau_out, double* sT, double* sP) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NT = kMergeStageThreads;
  const int64_t nr = k + nbk;
  double* Pb = sP;               // Pb[i + q nr] = Rb[i, k + q], rows 0 .. nr-1
  double* Pt = sP + nr * kNB;    // Pt[r + q kNB] = Rt[k + r, k + q]
  double* red = Pt + kNB * kNB;  // per-warp partial dot products (4 x kNB)
  double* red2 = red + 4 * kNB;  // per-warp partial norms
  double* sc = red2 + 4;         // tau, beta, scale of the current column
  double* sdot = sc + 4;         // the column step's dot products (kNB)
  double* sdv = sdot + kNB;      // the multiples of v_c subtracted from the later columns (kNB)
  for (int64_t idx = tid; idx < nr * nbk; idx += nthr) {
    const int64_t i = idx % nr, q = idx / nr;
    Pb[i + q * nr] = ldcg(Rb + i + (k + q) * M);
  }
  for (int idx = tid; idx < nbk * nbk; idx += nthr) {
    const int r = idx % nbk, q = idx / nbk;
    Pt[r + q * kNB] = ldcg(Rt + (k + r) + (k + q) * M);
  }
  __syncthreads();
  if (tid < NT) {
    double nx = 0.0;
    for (int64_t i = tid; i <= k; i += NT) nx += Pb[i] * Pb[i];
    nx = warp_sum(nx);
    if (lane == 0) red2[warp] = nx;
    stage_bar();
    double xx = red2[0] + red2[1] + red2[2] + red2[3];
    for (int jj = 0; jj < nbk; ++jj) {
      const int64_t c = k + jj;
      // thread 0 forms the reflector's scalars (FP64 square roots and
      // divisions are slow on this part) and shares them
      if (tid == 0) {
        const double alpha = Pt[jj + jj * kNB];
        double tau0 = 0.0, beta0 = alpha, scale0 = 0.0;
        if (xx != 0.0) {
          const double nrm = sqrt(alpha * alpha + xx);
          beta0 = (alpha >= 0.0) ? -nrm : nrm;
          tau0 = (beta0 - alpha) / beta0;
          scale0 = 1.0 / (alpha - beta0);
        }
        sc[0] = tau0;
        sc[1] = beta0;
        sc[2] = scale0;
      }
      stage_bar();
      const double tau_c = sc[0], beta = sc[1], scale = sc[2];
      // pass A: u_c = scale * bottom column c; dots with the other panel columns
      double acc[kNB];
#pragma unroll
      for (int q = 0; q < kNB; ++q) acc[q] = 0.0;
      for (int64_t i = tid; i <= c; i += NT) {
        const double u = Pb[i + jj * nr] * scale;
        Pb[i + jj * nr] = u;
#pragma unroll
        for (int q = 0; q < kNB; ++q)
          if (q < nbk && q != jj) acc[q] += u * Pb[i + q * nr];
      }
      {
        const double t = warp_reduce_scatter16(acc);
        if ((lane & 1) == 0) red[warp * kNB + ((lane >> 1) & 15)] = t;
      }
      stage_bar();
      // thread q totals column q's dot product and, for the later panel
      // columns, the multiple d_q of v_c to subtract (the e_c part of v_c
      // meets the top row c)
      if (tid < kNB) {
        const int q = tid;
        const double tq = (red[q] + red[kNB + q]) + (red[2 * kNB + q] + red[3 * kNB + q]);
        sdot[q] = tq;
        sdv[q] = (q > jj && q < nbk) ? (tq + Pt[jj + q * kNB]) * tau_c : 0.0;
      }
      stage_bar();
      double d[kNB];
#pragma unroll
      for (int q = 0; q < kNB; ++q) d[q] = sdv[q];
      // pass B: bottom rows 0..c of the later panel columns, and the squared
      // norm of the next column's rows 0..c+1
      nx = 0.0;
      if (jj + 1 < nbk) {
        for (int64_t i = tid; i <= c + 1; i += NT) {
          const double u = (i <= c) ? Pb[i + jj * nr] : 0.0;
#pragma unroll
          for (int q = 0; q < kNB; ++q) {
            if (q > jj && q < nbk) {
              double a = Pb[i + q * nr];
              if (i <= c) {
                a -= d[q] * u;
                Pb[i + q * nr] = a;
              }
              if (q == jj + 1) nx += a * a;
            }
          }
        }
      }
      nx = warp_sum(nx);
      if (lane == 0) red2[warp] = nx;
      stage_bar();   // every thread has read red and Pt row jj
      // column jj of T, one row per thread (rows 0..jj-1)
      if (tid < jj) {
        double sacc = 0.0;
        for (int q = tid; q < jj; ++q) sacc += sT[tid * kNB + q] * sdot[q];
        sT[tid * kNB + jj] = -tau_c * sacc;
      }
      if (tid == 0) {
        Pt[jj + jj * kNB] = beta;
        tau_out[jj] = tau_c;
        sT[jj * kNB + jj] = tau_c;
#pragma unroll
        for (int q = 0; q < kNB; ++q)
          if (q > jj && q < nbk) Pt[jj + q * kNB] -= d[q];
      }
      xx = red2[0] + red2[1] + red2[2] + red2[3];
    }
  }
  __syncthreads();
  for (int64_t idx = tid; idx < nr * nbk; idx += nthr) {
    const int64_t i = idx % nr, q = idx / nr;
    Rb[i + (k + q) * M] = Pb[i + q * nr];
  }
  for (int idx = tid; idx < nbk * nbk; idx += nthr) {
    const int r = idx % nbk, q = idx / nbk;
    Rt[(k + r) + (k + q) * M] = Pt[r + q * kNB];
  }
  __syncthreads();
}

// QR of [Rt; Rb] by panels of kNB columns: structured panel factorisation,
// then the block reflector applied to the trailing columns on the FP64
// tensor pipe (bottom rows 0..k+nbk-1 through u, top rows k..k+nbk-1 as the
// identity block).  Flops (2/3) M^3 as in the paper's cost model.
static __device__ void tree_merge(double* Rt, double* Rb, double* tau, int64_t M, double* sT, double* sred,
                           double* sout, double* sW, double* sWp) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int64_t k = 0; k < M; k += kNB) {
    const int nbk = (int)((M - k) < kNB ? (M - k) : kNB);
    for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = 0.0;
    __syncthreads();
    if (merge_panel_staged(M))
      merge_panel_factor_staged(Rt, Rb, M, k, nbk, tau + k, sT, sW);
    else
      merge_panel_factor(Rt, Rb, M, k, nbk, tau + k, sT, sred, sout);
    __syncthreads();
    if (k + nbk < M) {
      MergeV V{Rb, M, k, nbk};
      block_reflector<true, true>(V, nbk, 0, k + nbk, Rb + (k + nbk) * M, M, (int)(M - k - nbk),
                                  Rt + k + (k + nbk) * M, M, sT, sW, sWp);
    }
    __syncthreads();
  }
}

// Binary tree of Alg. 1 run by the block that finished leaf `leaf`: at step
// 2^l the subtree rooted at `node` pairs with node ^ 2^l; a missing partner
// (>= P) passes R up unchanged; the first block to arrive at a merge leaves,
// the second merges (left child's R on top, as the receiver keeps its R in
// the upper half of C in Alg. 1).  Shared-memory buffers as the leaf's.
static __device__ void tree_climb(const TsqrState& s, int64_t leaf, double* sT, double* sred, double* sout,
                                  double* sW, double* sWp) {
  __shared__ unsigned s_prev;
  const int tid = threadIdx.x;
  const int64_t M = s.M;
  int64_t node = leaf;
  for (int64_t step = 1; step < s.P; step <<= 1) {
    int64_t left, right;
    if (node & step) {
      left = node - step;
      right = node;
    } else {
      right = node + step;
      if (right >= s.P) continue;
      left = node;
    }
    if (tid == 0) s_prev = atomicAdd(&s.arrive[right], 1u);
    __syncthreads();
    const unsigned prev = s_prev;
    __syncthreads();
    if (prev == 0) return;  // first to arrive: the partner merges
    __threadfence();
    tree_merge(s.Rs + left * M * M, s.Rs + right * M * M, s.tau_tree + right * M, M, sT, sred, sout, sW, sWp);
    __threadfence();
    __syncthreads();
    node = left;
  }
}

}  // namespace pylom

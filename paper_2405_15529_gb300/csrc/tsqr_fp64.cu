// tsqr_fp64.cu -- binary64 TSQR (Alg. 1 of pyLOM, arXiv 2405.15529) on one
// GB300, plus the top-down pass and the modes product U = Q U_r (Eq. svdqr3).
//
// Layout (all column-major):
//   Y   N x M   the weighted, mean-removed snapshot matrix, overwritten leaf
//               by leaf with Householder vectors (unit diagonal implicit).
//   T   per leaf and panel: the kNB x kNB upper-triangular factor of the
//               compact-WY form Q_panel = I - V T V^T.
//   Rs  per leaf an M x M slot: the leaf R, then either the merged R (left
//               child, the receiver of Alg. 1) or the merge's reflectors
//               (right child, the sender).
//
// The paper's processes become row blocks ("leaves", one thread block
// each) and its binary-tree reduction becomes last-arriver merges across
// thread blocks: at every level the block that finishes second merges the
// pair (left child's R on top, as the receiver keeps its own R in the upper
// half of C in Alg. 1), so no block ever waits on another.
#include <stdlib.h>
#include <string.h>

#include "kernels.h"
#include "reflectors.cuh"

namespace pylom {

// Householder factorisation of the panel A[k:h, k:k+nbk] (Eq. svdqr1 on a
// row block), textbook convention beta = -sign(alpha)|x|, sign(0) = +1.
// Builds T (row-major kNB x kNB, upper) by the forward recurrence
// T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j).  Scalar FP64, one pass
// over the panel rows per column: the pass of column j scales v_j, applies
// reflector j to the later columns and, on the rows below j + 1, sums the
// products of the updated column j + 1 with every panel column (reflectors
// 0..j, itself, the later columns).  With those sums d_c, the dot products
// reflector j + 1 needs are scale_{j+1} d_c + A[j+1, c] (its unit entry
// meets row j + 1), so one block reduction per column serves the next
// column's norm, its update and its T column.
// Scratch: sred (block sums in [0, 16 nwarps), the next column's dot
// products at kPdDot, its scalars at kPdScal), sout (block totals; tau_j
// times the dot products at 16..31).
constexpr int kPdDot = 256, kPdScal = 288;
__device__ void panel_factor(double* A, int64_t lda, int64_t k, int nbk, int64_t h, double* tau_out,
                             double* sT, double* sred, double* sout) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  double* sdot = sred + kPdDot;     // v_j^T a_c (c != j)
  double* sts = sout + kNB;         // tau_j v_j^T a_c
  double acc[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) acc[c] = 0.0;
  // column k: d_c = sum over rows below k of A[i, k] A[i, k + c] (c = 0: the norm)
  for (int64_t i = k + 1 + tid; i < h; i += nthr) {
    const double a0 = A[i + k * lda];
#pragma unroll
    for (int c = 0; c < kNB; ++c)
      if (c < nbk) acc[c] += a0 * A[i + (k + c) * lda];
  }
  block_sum16(acc, sred, sout);
  for (int jj = 0; jj < nbk; ++jj) {
    const int64_t j = k + jj;
    // thread 0 forms the reflector's scalars and dot products (binary64
    // square roots and divisions are slow on this part) and broadcasts them
    if (tid == 0) {
      const double alpha = A[j + j * lda], xx = sout[jj];
      double tau_j = 0.0, beta = alpha, scale = 0.0;
      if (xx != 0.0) {
        const double nrm = sqrt(alpha * alpha + xx);
        beta = (alpha >= 0.0) ? -nrm : nrm;
        tau_j = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      for (int c = 0; c < nbk; ++c) {
        const double d = (c == jj) ? 0.0 : scale * sout[c] + A[j + (k + c) * lda];
        sdot[c] = d;
        sts[c] = tau_j * d;
      }
      sred[kPdScal] = tau_j;
      sred[kPdScal + 1] = beta;
      sred[kPdScal + 2] = scale;
      tau_out[jj] = tau_j;
    }
    __syncthreads();
    const double tau_j = sred[kPdScal], beta = sred[kPdScal + 1], scale = sred[kPdScal + 2];
    // column jj of T, one row per thread (rows 0..jj-1)
    if (tid < jj) {
      double s = 0.0;
      for (int q = tid; q < jj; ++q) s += sT[tid * kNB + q] * sdot[q];
      sT[tid * kNB + jj] = -tau_j * s;
    }
    if (tid == 0) sT[jj * kNB + jj] = tau_j;
    const bool more = jj + 1 < nbk;
#pragma unroll
    for (int c = 0; c < kNB; ++c) acc[c] = 0.0;
    for (int64_t i = j + tid; i < h; i += nthr) {
      double v;
      if (i == j) {
        v = 1.0;
        A[j + j * lda] = beta;
      } else {
        v = A[i + j * lda] * scale;
        A[i + j * lda] = v;
      }
      double row[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c) row[c] = (c < nbk && c != jj) ? A[i + (k + c) * lda] : 0.0;
#pragma unroll
      for (int c = 0; c < kNB; ++c)
        if (c > jj && c < nbk) {
          row[c] -= sts[c] * v;
          A[i + (k + c) * lda] = row[c];
        }
      if (more && i > j + 1) {
        double a1 = 0.0;   // row[jj + 1], selected without indexing the array at run time
#pragma unroll
        for (int c = 1; c < kNB; ++c)
          if (c == jj + 1) a1 = row[c];
#pragma unroll
        for (int c = 0; c < kNB; ++c)
          if (c < nbk) acc[c] += a1 * ((c == jj) ? v : row[c]);
      }
    }
    if (more) block_sum16(acc, sred, sout);
  }
}

struct LeafArgs {
  TsqrState s;
  const void* X;
  int64_t ldx;
  int xtype;
  const double* w;
  int remove_mean;
  double* mean;
};

template <typename TX>
__device__ void leaf_prologue(const LeafArgs& a, double* A, int64_t lda, int64_t r0, int64_t h) {
  const TX* X = (const TX*)a.X;
  const int64_t M = a.s.M;
  int bad = 0;
  for (int64_t i = threadIdx.x; i < h; i += blockDim.x) {
    const int64_t n = r0 + i - a.s.row0;   // row in the (chunk) buffers
    // kPro independent loads in flight per thread (the leaf has few warps)
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
          A[i + (m0 + u) * lda] = sw * (xv[u] - xbar);
        }
      }
    }
  }
  if (bad) raise_status(a.s.hdr, PYLOM_ERR_NONFINITE);
}

__global__ void __launch_bounds__(kLeafThreads) leaf_qr_kernel(LeafArgs a) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sred = sT + kSmT;
  double* sout = sred + kSmRed;
  double* sW = sout + kSmOut;
  double* sWp = sW + kSmW;
  const TsqrState& s = a.s;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t leaf = s.leaf0 + blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M, lda = s.ldy;
  double* A = s.Y + (r0 - s.row0);

  if (a.xtype == PYLOM_F32)
    leaf_prologue<float>(a, A, lda, r0, h);
  else
    leaf_prologue<double>(a, A, lda, r0, h);
  __syncthreads();

  for (int64_t k = 0; k < M; k += kNB) {
    const int nbk = (int)((M - k) < kNB ? (M - k) : kNB);
    for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = 0.0;
    __syncthreads();
    panel_factor(A, lda, k, nbk, h, s.tau + leaf * M + k, sT, sred, sout);
    __syncthreads();
    double* Tg = s.T + (leaf * s.npan + k / kNB) * kSmT;
    for (int idx = tid; idx < kSmT; idx += nthr) Tg[idx] = sT[idx];
    if (k + nbk < M) {
      LeafV V{A, lda, k, h, nbk};
      block_reflector<true, false>(V, nbk, k, h, A + (k + nbk) * lda, lda, (int)(M - k - nbk),
                                   nullptr, 0, sT, sW, sWp);
    }
    __syncthreads();
  }

  // leaf R into its slot (zeros below the diagonal)
  double* Rl = s.Rs + leaf * M * M;
  for (int64_t idx = tid; idx < M * M; idx += nthr) {
    const int64_t i = idx % M, j = idx / M;
    Rl[idx] = (i <= j) ? A[i + j * lda] : 0.0;
  }
  __threadfence();
  __syncthreads();

  if (s.climb) tree_climb(s, leaf, sT, sred, sout, sW, sWp);
}

// Top-down pass (the broadcast loop of Alg. 1): at a merge of `left` and
// `right`, [B_left; B_right] = Q_node [B_left; 0], applying the node's
// reflectors in reverse order.  One warp per column of B.
__global__ void __launch_bounds__(256) down_pass_kernel(TsqrState s, int64_t step, int64_t r_fixed) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t left = (int64_t)blockIdx.x * 2 * step, right = left + step;
  if (right >= s.P) return;
  const int64_t r = (r_fixed >= 0) ? r_fixed : s.hdr->r;
  const int64_t col = (int64_t)blockIdx.y * nwarps + warp;
  if (col >= r) return;
  const int64_t M = s.M;
  double* Bt = s.B + left * M * s.rmax + col * M;
  double* Bb = s.B + right * M * s.rmax + col * M;
  const double* U = s.Rs + right * M * M;
  const double* tau = s.tau_tree + right * M;
  for (int64_t i = lane; i < M; i += 32) Bb[i] = 0.0;
  __syncwarp();
  for (int64_t c = M - 1; c >= 0; --c) {
    const double tc = tau[c];
    if (tc == 0.0) continue;
    double acc = 0.0;
    for (int64_t i = lane; i <= c; i += 32) acc += U[i + c * M] * Bb[i];
    acc = (warp_sum(acc) + Bt[c]) * tc;
    __syncwarp();
    if (lane == 0) Bt[c] -= acc;
    for (int64_t i = lane; i <= c; i += 32) Bb[i] -= acc * U[i + c * M];
    __syncwarp();
  }
}

// B_root = first r columns of Ur (or the identity when Ur is null).
__global__ void init_root_kernel(TsqrState s, const double* Ur, int64_t ldur, int64_t r_fixed) {
  const int64_t r = (r_fixed >= 0) ? r_fixed : s.hdr->r;
  const int64_t M = s.M;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * r;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, c = idx / M;
    s.B[idx] = Ur ? Ur[i + c * ldur] : (i == c ? 1.0 : 0.0);
  }
}

// Per leaf: U_leaf = Q_leaf [B_leaf; 0], the panels applied last to first
// (Q_leaf = Q_panel0 Q_panel1 ...), then Phi = U / sqrt(w) if asked.
__global__ void __launch_bounds__(kLeafThreads) modes_kernel(TsqrState s, int64_t r_fixed,
                                                            const double* w, int physical,
                                                            double* U, int64_t ldu,
                                                            int64_t* r_out) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sW = sT + kSmT + kSmRed + kSmOut;
  double* sWp = sW + kSmW;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t leaf = s.leaf0 + blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M;
  const int64_t r = (r_fixed >= 0) ? r_fixed : s.hdr->r;
  if (leaf == 0 && tid == 0 && r_out) *r_out = r;
  double* C = U + (r0 - s.row0);
  const double* Bl = s.B + leaf * M * s.rmax;
  for (int64_t c = 0; c < r; ++c)
    for (int64_t i = tid; i < h; i += nthr) C[i + c * ldu] = (i < M) ? Bl[i + c * M] : 0.0;
  __syncthreads();
  const double* A = s.Y + (r0 - s.row0);
  for (int64_t pan = s.npan - 1; pan >= 0; --pan) {
    const int64_t k = pan * kNB;
    const int nbk = (int)((M - k) < kNB ? (M - k) : kNB);
    const double* Tg = s.T + (leaf * s.npan + pan) * kSmT;
    for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = Tg[idx];
    __syncthreads();
    LeafV V{A, s.ldy, k, h, nbk};
    // the first panel applied meets [B; 0]: its W sums only rows k..M-1
    block_reflector<false, false>(V, nbk, k, h, C, ldu, (int)r, nullptr, 0, sT, sW, sWp,
                                  pan == s.npan - 1 ? M : -1);
    __syncthreads();
  }
  if (physical && w) {
    for (int64_t i = tid; i < h; i += nthr) {
      const double iw = 1.0 / sqrt(w[r0 - s.row0 + i]);
      for (int64_t c = 0; c < r; ++c) C[i + c * ldu] *= iw;
    }
  }
}

__global__ void copy_root_kernel(TsqrState s, double* R, int64_t ldr) {
  const int64_t M = s.M;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * M;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, j = idx / M;
    R[i + j * ldr] = (i <= j) ? s.Rs[idx] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Which tree: the last-arriver climb inside the leaf kernel overlaps the
// merges with leaves still running and wins while there are few leaves and
// a merge is cheap.  From kCoopTreeMinP leaves on the leaves finish
// together and the climb's top levels are single-block merges in sequence;
// below kCoopTreeMinM columns the column-block pipeline (tree_pipe.cu) then
// overlaps the levels instead, and from kCoopTreeMinM columns on, where one
// merge is too much work for one block, the cooperative tree spreads every
// merge over all blocks level by level.  The environment variable
// PYLOM_TREE ("climb", "coop" or "pipe") overrides the choice.
static const char* tree_env() { return getenv("PYLOM_TREE"); }

bool use_climb_tree(int64_t M, int64_t P) {
  const char* env = tree_env();
  if (P <= 1) return true;
  if (env && strcmp(env, "climb") == 0) return true;
  if (env && (strcmp(env, "coop") == 0 || strcmp(env, "pipe") == 0)) return false;
  return M < kCoopTreeMinM && P < kCoopTreeMinP;
}

bool use_pipe_tree(int64_t M, int64_t P) {
  if (use_climb_tree(M, P)) return false;
  const char* env = tree_env();
  if (env && strcmp(env, "pipe") == 0) return true;
  if (env && strcmp(env, "coop") == 0) return false;
  return M < kCoopTreeMinM;
}

cudaError_t launch_tree(const TsqrState& s, cudaStream_t st) {
  return s.pipe ? launch_tree_pipe(s, st) : launch_tree_coop(s, st);
}

size_t tsqr_state_bytes(int64_t N, int64_t M, int64_t P, int64_t rmax, bool with_y) {
  const int64_t npan = (M + kNB - 1) / kNB;
  size_t b = 0;
  if (with_y) b += align256(sizeof(double) * (size_t)N * M);
  b += align256(sizeof(double) * (size_t)P * M);
  b += align256(sizeof(double) * (size_t)P * npan * kNB * kNB);
  b += align256(sizeof(double) * (size_t)P * M * M);
  b += align256(sizeof(double) * (size_t)P * M);
  b += align256(sizeof(unsigned) * (size_t)P);
  b += align256(sizeof(double) * (size_t)2 * ((P + 1) / 2) * kSmT);
  b += align256(sizeof(double) * (size_t)P * npan * kSmT);
  b += align256(sizeof(double) * (size_t)P * M * rmax);
  return b;
}

void tsqr_state_carve(TsqrState& s, char* base, int64_t N, int64_t M, int64_t P, int64_t rmax, bool with_y) {
  s.N = N;
  s.M = M;
  s.P = P;
  s.npan = (M + kNB - 1) / kNB;
  s.rmax = rmax;
  char* p = base;
  s.Y = with_y ? (double*)p : nullptr;
  if (with_y) p += align256(sizeof(double) * (size_t)N * M);
  s.tau = (double*)p;      p += align256(sizeof(double) * (size_t)P * M);
  s.T = (double*)p;        p += align256(sizeof(double) * (size_t)P * s.npan * kNB * kNB);
  s.Rs = (double*)p;       p += align256(sizeof(double) * (size_t)P * M * M);
  s.tau_tree = (double*)p; p += align256(sizeof(double) * (size_t)P * M);
  s.arrive = (unsigned*)p; p += align256(sizeof(unsigned) * (size_t)P);
  s.Tt = (double*)p;       p += align256(sizeof(double) * (size_t)2 * ((P + 1) / 2) * kSmT);
  s.Tn = (double*)p;       p += align256(sizeof(double) * (size_t)P * s.npan * kSmT);
  s.B = rmax > 0 ? (double*)p : nullptr;
  s.climb = use_climb_tree(M, P) ? 1 : 0;
  s.pipe = use_pipe_tree(M, P) ? 1 : 0;
  s.leaf0 = 0;
  s.Pl = P;
  s.row0 = 0;
  s.ldy = N;
}

cudaError_t launch_tsqr_fp64(const TsqrState& s, const void* X, int64_t ldx, int xtype,
                             const double* w, int remove_mean, double* mean, cudaStream_t st, cudaEvent_t mid) {
  cudaError_t e;
  if ((e = ensure_dyn_smem((const void*)leaf_qr_kernel, kLeafSmemBytes)) != cudaSuccess) return e;
  if ((e = ensure_dyn_smem((const void*)modes_kernel, kLeafSmemBytes)) != cudaSuccess) return e;
  LeafArgs a{s, X, ldx, xtype, w, remove_mean, mean};
  leaf_qr_kernel<<<(unsigned)s.Pl, kLeafThreads, kLeafSmemBytes, st>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess && mid) e = cudaEventRecord(mid, st);
  // a launch over a slice of the leaves (streamed) leaves the cooperative
  // tree to its caller, after the last slice
  if (e != cudaSuccess || s.climb || s.Pl != s.P) return e;
  return launch_tree(s, st);
}

cudaError_t launch_copy_root_r(const TsqrState& s, double* R, int64_t ldr, cudaStream_t st) {
  copy_root_kernel<<<64, 256, 0, st>>>(s, R, ldr);
  return cudaGetLastError();
}

cudaError_t launch_down_pass_fp64(const TsqrState& s, const double* Ur, int64_t ldur, int64_t r_fixed,
                                  cudaStream_t st) {
  init_root_kernel<<<64, 256, 0, st>>>(s, Ur, ldur, r_fixed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t top = 1;
  while (top * 2 < s.P) top *= 2;
  const unsigned ycols = (unsigned)((s.rmax + 7) / 8);
  for (int64_t step = (s.P > 1 ? top : 0); step >= 1; step >>= 1) {
    const int64_t merges = (s.P - step + 2 * step - 1) / (2 * step);
    dim3 grid((unsigned)merges, ycols);
    down_pass_kernel<<<grid, 256, 0, st>>>(s, step, r_fixed);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_modes_fp64(const TsqrState& s, const double* Ur, int64_t ldur, int64_t r_fixed,
                              const double* w, int physical, double* U, int64_t ldu,
                              int64_t* r_out, cudaStream_t st, cudaEvent_t mid) {
  cudaError_t e = launch_down_pass_fp64(s, Ur, ldur, r_fixed, st);
  if (e != cudaSuccess) return e;
  if (mid) {
    e = cudaEventRecord(mid, st);
    if (e != cudaSuccess) return e;
  }
  modes_kernel<<<(unsigned)s.Pl, kLeafThreads, kLeafSmemBytes, st>>>(s, r_fixed, w, physical, U, ldu,
                                                                     r_out);
  return cudaGetLastError();
}

cudaError_t launch_leaf_modes_fp64(const TsqrState& s, int64_t r_fixed, const double* w, int physical, double* U,
                                   int64_t ldu, int64_t* r_out, cudaStream_t st) {
  const cudaError_t e = ensure_dyn_smem((const void*)modes_kernel, kLeafSmemBytes);
  if (e != cudaSuccess) return e;
  modes_kernel<<<(unsigned)s.Pl, kLeafThreads, kLeafSmemBytes, st>>>(s, r_fixed, w, physical, U, ldu, r_out);
  return cudaGetLastError();
}

}  // namespace pylom

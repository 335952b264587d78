// pod_backward.cu -- hand-written adjoint of the POD path (TSQR + small SVD
// + U = Q U_r, Eqs. svdqr1-svdqr3 of pyLOM, arXiv 2405.15529): given
// cotangents of the returned modes U_r (N x r), singular values S (M) and
// right vectors V^T (M x M), it returns the cotangent of X.
//
// Composition (Y_w = W^(1/2)(X - mean); Y_w = Q R; R = U_R S V^T; U = Q U_R),
// differentiated as the thin SVD of Y_w expressed in the TSQR factors:
//   1. Zt = Q^T dU (M x M, first r columns nonzero): every leaf applies its
//      Q_leaf^T to its rows of dU (the stored reflectors, panel by panel),
//      then the tree applies each node's Q^T bottom-up -- Q is recomputed
//      from the reflectors, never kept.
//   2. Small FP64 algebra on M x M matrices (the square SVD adjoint of R):
//      K  = (F o (U_R^T Zt - Zt^T U_R)) S + diag(dS) + S (F o (V^T dV - dV^T V)),
//           F_ij = 1/(s_j^2 - s_i^2);
//      dR = U_R K V^T;   B = dR - Zt S^-1 V^T;   C = S_r^-1 V_r^T.
//   3. dY = Q [B; 0] + dU C  (top-down pass + leaf products with M columns).
//   4. dX = W^(1/2) dY, minus each row's mean if the mean was removed.
// Writing the QR adjoint and the SVD adjoint separately would need R^-T,
// which does not exist once the mean is removed (Y_w 1 = 0 makes R
// singular); in the composition R^-T cancels, and only the singular values
// of modes that carry a cotangent are inverted.  Degenerate pairs
// (s_i == s_j, i != j) contribute no coupling term.
#include "kernels.h"
#include "reflectors.cuh"

namespace pylom {

// dU (N x r) -> C (N x r, ld N), with W^(-1/2) applied for physical modes.
__global__ void bw_load_du_kernel(const double* dU, int64_t lddu, const double* w, int physical,
                                  double* C, int64_t N, int64_t r) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * r; idx += stride) {
    const int64_t n = idx % N, c = idx / N;
    double v = dU ? dU[n + c * lddu] : 0.0;
    if (physical && w) v /= sqrt(w[n]);
    C[idx] = v;
  }
}

// Per leaf: C_leaf := Q_leaf^T C_leaf (panels in factorisation order, T^T),
// then the top M rows go to the leaf's Z slot (M x r).
__global__ void __launch_bounds__(kLeafThreads) bw_leaf_qt_kernel(TsqrState s, double* C, double* Z,
                                                                  int64_t r) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sW = sT + kSmT + kSmRed + kSmOut;
  double* sWp = sW + kSmW;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t leaf = blockIdx.x;
  const int64_t r0 = leaf_begin(leaf, s.N, s.P);
  const int64_t h = leaf_begin(leaf + 1, s.N, s.P) - r0;
  const int64_t M = s.M;
  const double* A = s.Y + r0;
  double* Cl = C + r0;
  for (int64_t pan = 0; pan < s.npan; ++pan) {
    const int64_t k = pan * kNB;
    const int nbk = (int)((M - k) < kNB ? (M - k) : kNB);
    const double* Tg = s.T + (leaf * s.npan + pan) * kSmT;
    for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = Tg[idx];
    __syncthreads();
    LeafV V{A, s.N, k, h, nbk};
    block_reflector<true, false>(V, nbk, k, h, Cl, s.N, (int)r, nullptr, 0, sT, sW, sWp);
    __syncthreads();
  }
  double* Zl = Z + leaf * M * r;
  for (int64_t idx = tid; idx < M * r; idx += nthr) Zl[idx] = Cl[(idx % M) + (idx / M) * s.N];
}

// Up pass at tree step `step`: [Z_left; Z_right] := Q_node^T [Z_left; Z_right],
// reflectors in factorisation order; Z_left then holds the parent's block.
// One warp per column.
__global__ void __launch_bounds__(256) bw_up_pass_kernel(TsqrState s, double* Z, int64_t r, int64_t step) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t left = (int64_t)blockIdx.x * 2 * step, right = left + step;
  if (right >= s.P) return;
  const int64_t col = (int64_t)blockIdx.y * nwarps + warp;
  if (col >= r) return;
  const int64_t M = s.M;
  double* Zt = Z + left * M * r + col * M;
  double* Zb = Z + right * M * r + col * M;
  const double* U = s.Rs + right * M * M;
  const double* tau = s.tau_tree + right * M;
  for (int64_t c = 0; c < M; ++c) {
    const double tc = tau[c];
    if (tc == 0.0) continue;
    double acc = 0.0;
    for (int64_t i = lane; i <= c; i += 32) acc += U[i + c * M] * Zb[i];
    acc = (warp_sum(acc) + Zt[c]) * tc;
    __syncwarp();
    if (lane == 0) Zt[c] -= acc;
    for (int64_t i = lane; i <= c; i += 32) Zb[i] -= acc * U[i + c * M];
    __syncwarp();
  }
}

// C = alpha op(A) op(B) + beta C, small FP64 matrices, 16 x 16 shared tiles.
__global__ void bw_gemm_kernel(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               double beta, double* C, int64_t ldc) {
  __shared__ double sa[16][17], sb[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t i = (int64_t)blockIdx.y * 16 + ty;   // row of C
  const int64_t j = (int64_t)blockIdx.x * 16 + tx;   // column of C
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < k; k0 += 16) {
    // sa[ty][tx] = op(A)[i][k0 + tx]; sb[ty][tx] = op(B)[k0 + ty][j]
    const int64_t ka = k0 + tx, kb = k0 + ty;
    double av = 0.0, bv = 0.0;
    if (i < m && ka < k) av = ta ? A[ka + i * lda] : A[i + ka * lda];
    if (j < n && kb < k) bv = tb ? B[j + kb * ldb] : B[kb + j * ldb];
    sa[ty][tx] = av;
    sb[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += sa[ty][q] * sb[q][tx];
    __syncthreads();
  }
  if (i < m && j < n) C[i + j * ldc] = alpha * acc + (beta != 0.0 ? beta * C[i + j * ldc] : 0.0);
}

// K = (F o G1) S + diag(dS) + S (F o G2) with G = A - A^T, in place of K.
__global__ void bw_svd_core_kernel(const double* A1, const double* A2, const double* S,
                                   const double* dS, double* K, int64_t M) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * M; idx += stride) {
    const int64_t i = idx % M, j = idx / M;
    if (i == j) {
      K[idx] = dS ? dS[i] : 0.0;
      continue;
    }
    const double si = S[i], sj = S[j];
    const double den = sj * sj - si * si;
    const double f = (den != 0.0) ? 1.0 / den : 0.0;
    const double g1 = A1[i + j * M] - A1[j + i * M];
    const double g2 = A2[i + j * M] - A2[j + i * M];
    K[idx] = f * (g1 * sj + si * g2);
  }
}

// C (rows x M, ld rows) = diag(1 / S[0:rows]) VT[0:rows, :].
__global__ void bw_scale_rows_kernel(const double* VT, int64_t ldvt, const double* S, double* C,
                                     int64_t rows, int64_t M) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < rows * M; idx += stride) {
    const int64_t i = idx % rows, j = idx / rows;
    C[i + j * rows] = VT[i + j * ldvt] / S[i];
  }
}

// dY += dU C (N x r times r x M) on the FP64 tensor pipe: each warp owns
// 8-row tiles and sweeps all 8-column tiles; k = r in steps of 4.
__global__ void __launch_bounds__(256) bw_add_du_c_kernel(const double* dU, const double* Cm,
                                                          int64_t ldcm, double* dY, int64_t N,
                                                          int64_t M, int64_t r) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nrt = (N + 7) / 8;
  for (int64_t rt = warp; rt < nrt; rt += nwarps) {
    const int64_t row = rt * 8 + g;
    for (int64_t c0 = 0; c0 < M; c0 += 8) {
      const int64_t col = c0 + 2 * t;
      double d0 = (row < N && col < M) ? dY[row + col * N] : 0.0;
      double d1 = (row < N && col + 1 < M) ? dY[row + (col + 1) * N] : 0.0;
      for (int64_t k0 = 0; k0 < r; k0 += 4) {
        const int64_t ka = k0 + t;
        const double a = (row < N && ka < r) ? dU[row + ka * N] : 0.0;
        const double b = (ka < r && c0 + g < M) ? Cm[ka + (c0 + g) * ldcm] : 0.0;
        dmma884(d0, d1, a, b);
      }
      if (row < N && col < M) dY[row + col * N] = d0;
      if (row < N && col + 1 < M) dY[row + (col + 1) * N] = d1;
    }
  }
}

// dX = W^(1/2) dY, then minus each row's mean (adjoint of mean removal).
template <typename TX, typename TY>
__global__ void bw_finalize_kernel(const TY* dY, const double* w, int remove_mean, TX* dX,
                                   int64_t lddx, int64_t N, int64_t M) {
  for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    const double sw = w ? sqrt(w[n]) : 1.0;
    double mu = 0.0;
    if (remove_mean) {
      double sum = 0.0;
      for (int64_t m = 0; m < M; ++m) sum += sw * (double)dY[n + m * N];
      mu = sum / (double)M;
    }
    for (int64_t m = 0; m < M; ++m) dX[n + m * lddx] = (TX)(sw * (double)dY[n + m * N] - mu);
  }
}

// Mixed path: dU (N x r, binary64) -> C (FP32, ld N), W^(-1/2) for physical modes.
__global__ void bw_load_du_f32_kernel(const double* dU, int64_t lddu, const double* w, int physical, float* C,
                                      int64_t N, int64_t r) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * r; idx += stride) {
    const int64_t n = idx % N, c = idx / N;
    double v = dU[n + c * lddu];
    if (physical && w) v /= sqrt(w[n]);
    C[idx] = (float)v;
  }
}

// Mixed path: dY (FP32, N x M) += C (N x r) Cm (r x M, binary64, ld r) in
// FP32; Cm staged per block in shared memory (r <= M <= 4096 columns are
// taken 64 at a time).
__global__ void __launch_bounds__(256) bw_add_du_c_f32_kernel(const float* C, const double* Cm, int64_t ldcm,
                                                              float* dY, int64_t N, int64_t M, int64_t r) {
  extern __shared__ float scm[];   // r x 64
  for (int64_t m0 = 0; m0 < M; m0 += 64) {
    const int64_t mw = (M - m0) < 64 ? (M - m0) : 64;
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < r * mw; idx += blockDim.x) {
      const int64_t c = idx % r, m = idx / r;
      scm[c + m * r] = (float)Cm[c + (m0 + m) * ldcm];
    }
    __syncthreads();
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
      for (int64_t m = 0; m < mw; ++m) {
        float acc = 0.f;
        for (int64_t c = 0; c < r; ++c) acc = fmaf(C[n + c * N], scm[c + m * r], acc);
        dY[n + (m0 + m) * N] += acc;
      }
    }
  }
}

struct BwLayout {
  double* C;      // N x r
  double* Z;      // P x M x r
  double* B;      // P x M x M (down-pass blocks)
  double* A1;     // M x M
  double* A2;     // M x M
  double* K;      // M x M
  double* T1;     // M x M
  double* Bm;     // M x M
  double* Cm;     // r x M (ld r)
  double* dY;     // N x M
};

size_t pod_backward_bytes(int64_t N, int64_t M, int64_t P, int64_t r) {
  size_t b = sizeof(WsHeader);
  b += align256(sizeof(double) * (size_t)N * r);
  b += align256(sizeof(double) * (size_t)P * M * r);
  b += align256(sizeof(double) * (size_t)P * M * M);
  b += 5 * align256(sizeof(double) * (size_t)M * M);
  b += align256(sizeof(double) * (size_t)r * M);
  b += align256(sizeof(double) * (size_t)N * M);
  return b;
}

static BwLayout carve_backward(char* base, int64_t N, int64_t M, int64_t P, int64_t r) {
  BwLayout L;
  char* p = base + sizeof(WsHeader);
  L.C = (double*)p;  p += align256(sizeof(double) * (size_t)N * r);
  L.Z = (double*)p;  p += align256(sizeof(double) * (size_t)P * M * r);
  L.B = (double*)p;  p += align256(sizeof(double) * (size_t)P * M * M);
  L.A1 = (double*)p; p += align256(sizeof(double) * (size_t)M * M);
  L.A2 = (double*)p; p += align256(sizeof(double) * (size_t)M * M);
  L.K = (double*)p;  p += align256(sizeof(double) * (size_t)M * M);
  L.T1 = (double*)p; p += align256(sizeof(double) * (size_t)M * M);
  L.Bm = (double*)p; p += align256(sizeof(double) * (size_t)M * M);
  L.Cm = (double*)p; p += align256(sizeof(double) * (size_t)r * M);
  L.dY = (double*)p;
  return L;
}

static cudaError_t gemm(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                        cudaStream_t st) {
  dim3 blk(16, 16), grd((unsigned)((n + 15) / 16), (unsigned)((m + 15) / 16));
  bw_gemm_kernel<<<grd, blk, 0, st>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  return cudaGetLastError();
}

cudaError_t launch_pod_backward(const TsqrState& fs, const double* UR, const double* S, const double* VT,
                                int64_t ldvt, const double* dU, int64_t lddu, const double* dS,
                                const double* dVT, int64_t lddvt, const double* w, int remove_mean,
                                int physical, int64_t r, void* dX, int64_t lddx, int dxtype,
                                char* bw_base, char* mixed_extra, cudaStream_t st) {
  const int64_t N = fs.N, M = fs.M, P = fs.P;
  BwLayout L = carve_backward(bw_base, N, M, P, r);
  const bool mixed = mixed_extra != nullptr;   // FP32 reflectors of a mixed-precision forward
  float* C32 = (float*)L.C;
  float* dY32 = (float*)L.dY;
  cudaError_t e;
  // 1. Z = Q^T dU
  if (mixed && dU && r > 0) {
    bw_load_du_f32_kernel<<<1024, 256, 0, st>>>(dU, lddu, w, physical, C32, N, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_leaf_qt_mixed(fs, mixed_extra, C32, r, L.Z, st)) != cudaSuccess) return e;
    for (int64_t step = 1; step < P; step <<= 1) {
      const int64_t merges = (P - step + 2 * step - 1) / (2 * step);
      dim3 grid((unsigned)merges, (unsigned)((r + 7) / 8));
      bw_up_pass_kernel<<<grid, 256, 0, st>>>(fs, L.Z, r, step);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else if (dU && r > 0) {
    bw_load_du_kernel<<<1024, 256, 0, st>>>(dU, lddu, w, physical, L.C, N, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = ensure_dyn_smem((const void*)bw_leaf_qt_kernel, kLeafSmemBytes)) != cudaSuccess) return e;
    bw_leaf_qt_kernel<<<(unsigned)P, kLeafThreads, kLeafSmemBytes, st>>>(fs, L.C, L.Z, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int64_t step = 1; step < P; step <<= 1) {
      const int64_t merges = (P - step + 2 * step - 1) / (2 * step);
      dim3 grid((unsigned)merges, (unsigned)((r + 7) / 8));
      bw_up_pass_kernel<<<grid, 256, 0, st>>>(fs, L.Z, r, step);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else {
    if ((e = cudaMemsetAsync(L.Z, 0, sizeof(double) * (size_t)M * (r > 0 ? r : 1), st)) != cudaSuccess)
      return e;
  }
  // 2. small algebra.  A1 = U_R^T Zt (only the first r columns are nonzero)
  if ((e = cudaMemsetAsync(L.A1, 0, sizeof(double) * (size_t)M * M, st)) != cudaSuccess) return e;
  if (r > 0 && (e = gemm(1, 0, M, r, M, 1.0, UR, M, L.Z, M, 0.0, L.A1, M, st)) != cudaSuccess) return e;
  // A2 = V^T dV = VT dVT^T
  if (dVT) {
    if ((e = gemm(0, 1, M, M, M, 1.0, VT, ldvt, dVT, lddvt, 0.0, L.A2, M, st)) != cudaSuccess) return e;
  } else if ((e = cudaMemsetAsync(L.A2, 0, sizeof(double) * (size_t)M * M, st)) != cudaSuccess) {
    return e;
  }
  bw_svd_core_kernel<<<256, 256, 0, st>>>(L.A1, L.A2, S, dS, L.K, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // dR = U_R K V^T = U_R (K VT), into Bm
  if ((e = gemm(0, 0, M, M, M, 1.0, L.K, M, VT, ldvt, 0.0, L.T1, M, st)) != cudaSuccess) return e;
  if ((e = gemm(0, 0, M, M, M, 1.0, UR, M, L.T1, M, 0.0, L.Bm, M, st)) != cudaSuccess) return e;
  if (r > 0) {
    // C = S_r^-1 V_r^T (r x M); B -= Zt S^-1 V^T = Z C
    bw_scale_rows_kernel<<<256, 256, 0, st>>>(VT, ldvt, S, L.Cm, r, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = gemm(0, 0, M, M, r, -1.0, L.Z, M, L.Cm, r, 1.0, L.Bm, M, st)) != cudaSuccess) return e;
  }
  // 3. dY = Q [B; 0] (top-down pass + leaf products, r = M columns) ...
  TsqrState ds = fs;
  ds.B = L.B;
  ds.rmax = M;
  if (mixed) {
    e = launch_modes_mixed(ds, mixed_extra, L.Bm, M, M, nullptr, 0, dY32, N, nullptr, st, nullptr);
    if (e != cudaSuccess) return e;
    if (dU && r > 0) {
      bw_load_du_f32_kernel<<<1024, 256, 0, st>>>(dU, lddu, w, physical, C32, N, r);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      bw_add_du_c_f32_kernel<<<1216, 256, sizeof(float) * (size_t)r * 64, st>>>(C32, L.Cm, r, dY32, N, M, r);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (dxtype == PYLOM_F32)
      bw_finalize_kernel<float, float><<<1024, 256, 0, st>>>(dY32, w, remove_mean, (float*)dX, lddx, N, M);
    else
      bw_finalize_kernel<double, float><<<1024, 256, 0, st>>>(dY32, w, remove_mean, (double*)dX, lddx, N, M);
    return cudaGetLastError();
  }
  if ((e = launch_modes_fp64(ds, L.Bm, M, M, nullptr, 0, L.dY, N, nullptr, st)) != cudaSuccess) return e;
  // ... + dU_w C (dU reloaded: step 1 transformed its copy in place)
  if (dU && r > 0) {
    bw_load_du_kernel<<<1024, 256, 0, st>>>(dU, lddu, w, physical, L.C, N, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bw_add_du_c_kernel<<<1216, 256, 0, st>>>(L.C, L.Cm, r, L.dY, N, M, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 4. dX = W^(1/2) dY (minus row means)
  if (dxtype == PYLOM_F32)
    bw_finalize_kernel<float, double><<<1024, 256, 0, st>>>(L.dY, w, remove_mean, (float*)dX, lddx, N, M);
  else
    bw_finalize_kernel<double, double><<<1024, 256, 0, st>>>(L.dY, w, remove_mean, (double*)dX, lddx, N, M);
  return cudaGetLastError();
}

}  // namespace pylom

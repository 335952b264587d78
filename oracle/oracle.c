/*
 * oracle.c -- plain, slow FP64 CPU oracle for the POD / TSQR-SVD path of
 * pyLOM (Eiximeno et al., arXiv 2405.15529).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * What it computes is the plain definition the method reaches exactly (up
 * to rounding order): the SVD of Y_w = diag(sqrt(w)) (X - xbar 1^T), the
 * snapshot matrix with its temporal mean removed (Alg. 2) and, optionally,
 * scaled by square-root cell volumes.  Chan's QR-then-SVD route (Eqs.
 * svdqr1-svdqr3, Sec. 3.1) is an identity, so the oracle runs it without
 * any blocking or tree: one unblocked Householder QR of the whole matrix,
 * a one-sided (Hestenes) Jacobi SVD of R, and U = Q [U_r; 0].
 *
 * Conventions (the readings the CUDA path follows too; they are listed,
 * with reasons, in the design notes):
 *   - X is N x M, column-major (N gridpoints, M snapshots).
 *   - Householder vectors follow the textbook convention
 *     beta = -sign(alpha) ||x||, sign(0) = +1, v[0] = 1 implicit.
 *   - Singular values are sorted descending, ties kept in index order.
 *   - Each pair (u_i, v_i) is flipped so that the entry of v_i with the
 *     largest magnitude is positive (lowest index on an exact tie).
 *   - Truncation keeps r = min{k : sum_{i<=k} s_i^2 / sum_i s_i^2 >= energy}
 *     (Sec. 3.1 cumulative energy), capped at r_max; energy <= 0 means
 *     r = r_max.
 *
 * Floating point: all arithmetic is IEEE binary64, plain left-to-right
 * sums.  OpenMP splits independent columns or rows only (no change in any
 * single value's summation order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define A_(i, j) A[(int64_t)(j) * lda + (i)]

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Temporal mean removal and square-root cell-volume weighting.
 * Alg. 2 (POD algorithm, Appendix B): mean over the n_t snapshots of each
 * gridpoint, subtracted from every snapshot.  The weights are not in the
 * paper; they make the Euclidean SVD of Y_w the discrete form of the
 * volume-integral orthonormality of Sec. 2.1.
 * mean may be NULL; w may be NULL (uniform weights).
 * ------------------------------------------------------------------------ */
void oracle_center_weight(const double* X, int64_t N, int64_t M, int64_t ldx,
                          const double* w, int remove_mean, double* Y,
                          int64_t ldy, double* mean) {
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    double xbar = 0.0;
    if (remove_mean) {
      double s = 0.0;
      for (int64_t m = 0; m < M; ++m) s += X[m * ldx + n];
      xbar = s / (double)M;
    }
    if (mean) mean[n] = xbar;
    double sw = w ? sqrt(w[n]) : 1.0;
    for (int64_t m = 0; m < M; ++m) Y[m * ldy + n] = sw * (X[m * ldx + n] - xbar);
  }
}

/* ------------------------------------------------------------------------
 * Unblocked Householder QR, A = Q [R; 0] (Eq. svdqr1).
 * On return the upper triangle of A (rows 0..m-1) holds R and the part
 * below the diagonal holds the Householder vectors v_j (v_j[j] = 1 is
 * implicit).  Q = H_0 H_1 ... H_{m-1}, H_j = I - tau_j v_j v_j^T.
 * Requires n >= m.
 * ------------------------------------------------------------------------ */
void oracle_householder_qr(double* A, int64_t n, int64_t m, int64_t lda,
                           double* tau) {
  for (int64_t j = 0; j < m; ++j) {
    double alpha = A_(j, j);
    double xx = 0.0;
    for (int64_t i = j + 1; i < n; ++i) xx += A_(i, j) * A_(i, j);
    if (xx == 0.0) {            /* nothing below the diagonal: H_j = I */
      tau[j] = 0.0;
      continue;
    }
    double norm = sqrt(alpha * alpha + xx);
    double beta = (alpha >= 0.0) ? -norm : norm;
    tau[j] = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t i = j + 1; i < n; ++i) A_(i, j) *= scal;
    A_(j, j) = beta;
    /* apply H_j to the trailing columns */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < m; ++k) {
      double s = A_(j, k);
      for (int64_t i = j + 1; i < n; ++i) s += A_(i, j) * A_(i, k);
      s *= tau[j];
      A_(j, k) -= s;
      for (int64_t i = j + 1; i < n; ++i) A_(i, k) -= s * A_(i, j);
    }
  }
}

/* C := Q C for the Q stored by oracle_householder_qr (C is n x k). */
void oracle_apply_q(const double* A, int64_t n, int64_t m, int64_t lda,
                    const double* tau, double* C, int64_t k, int64_t ldc) {
  for (int64_t j = m - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < k; ++c) {
      double* col = C + c * ldc;
      double s = col[j];
      for (int64_t i = j + 1; i < n; ++i) s += A_(i, j) * col[i];
      s *= tau[j];
      col[j] -= s;
      for (int64_t i = j + 1; i < n; ++i) col[i] -= s * A_(i, j);
    }
  }
}

/* ------------------------------------------------------------------------
 * One-sided (Hestenes) Jacobi SVD of an n x m matrix A, n >= m
 * (used on the m x m R of Eq. svdqr2).  Cyclic-by-row sweeps; the pair
 * (i, j) is rotated when |a_i.a_j| > tol sqrt(|a_i|^2 |a_j|^2) with
 * tol = n * 2^-53; a sweep without rotations ends the iteration.
 * On return: A's columns are a_i = s_i u_i (unsorted), S[i] = |a_i|,
 * V (m x m) the accumulated rotations.  Returns the sweeps used, or -1 if
 * max_sweeps were not enough.
 * ------------------------------------------------------------------------ */
int oracle_jacobi_svd(double* A, int64_t n, int64_t m, int64_t lda, double* S,
                      double* V, int64_t ldv, int max_sweeps) {
  const double tol = (double)n * ldexp(1.0, -53);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) V[j * ldv + i] = (i == j) ? 1.0 : 0.0;
  int sweep = 0, converged = 0;
  while (sweep < max_sweeps && !converged) {
    int rotated = 0;
    for (int64_t i = 0; i < m - 1; ++i) {
      for (int64_t j = i + 1; j < m; ++j) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t k = 0; k < n; ++k) {
          alpha += A_(k, i) * A_(k, i);
          beta += A_(k, j) * A_(k, j);
          gamma += A_(k, i) * A_(k, j);
        }
        if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t k = 0; k < n; ++k) {
          double ai = A_(k, i), aj = A_(k, j);
          A_(k, i) = c * ai - s * aj;
          A_(k, j) = s * ai + c * aj;
        }
        for (int64_t k = 0; k < m; ++k) {
          double vi = V[i * ldv + k], vj = V[j * ldv + k];
          V[i * ldv + k] = c * vi - s * vj;
          V[j * ldv + k] = s * vi + c * vj;
        }
      }
    }
    ++sweep;
    if (!rotated) converged = 1;
  }
  for (int64_t i = 0; i < m; ++i) {
    double ss = 0.0;
    for (int64_t k = 0; k < n; ++k) ss += A_(k, i) * A_(k, i);
    S[i] = sqrt(ss);
  }
  return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------
 * Post-processing of a Jacobi result: sort descending (stable), normalise
 * the left vectors, complete the basis where a singular value is exactly
 * zero, and apply the sign convention.  A: n x m (columns s_i u_i on entry,
 * u_i on return); V: m x m.
 * ------------------------------------------------------------------------ */
static void sort_normalise_sign(double* A, int64_t n, int64_t m, int64_t lda,
                                double* S, double* V, int64_t ldv) {
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * m);
  for (int64_t i = 0; i < m; ++i) perm[i] = i;
  /* stable insertion sort on descending S */
  for (int64_t i = 1; i < m; ++i) {
    int64_t p = perm[i];
    int64_t k = i;
    while (k > 0 && S[perm[k - 1]] < S[p]) { perm[k] = perm[k - 1]; --k; }
    perm[k] = p;
  }
  double* A2 = (double*)malloc(sizeof(double) * n * m);
  double* V2 = (double*)malloc(sizeof(double) * m * m);
  double* S2 = (double*)malloc(sizeof(double) * m);
  for (int64_t c = 0; c < m; ++c) {
    int64_t p = perm[c];
    S2[c] = S[p];
    for (int64_t k = 0; k < n; ++k) A2[c * n + k] = A_(k, p);
    for (int64_t k = 0; k < m; ++k) V2[c * m + k] = V[p * ldv + k];
  }
  for (int64_t c = 0; c < m; ++c) {
    S[c] = S2[c];
    for (int64_t k = 0; k < n; ++k) A_(k, c) = (S2[c] > 0.0) ? A2[c * n + k] / S2[c] : 0.0;
    for (int64_t k = 0; k < m; ++k) V[c * ldv + k] = V2[c * m + k];
  }
  /* basis completion for exactly-zero singular values (Gram-Schmidt of
   * unit vectors against the vectors already present, twice). */
  int64_t next_e = 0;
  for (int64_t c = 0; c < m; ++c) {
    if (S[c] > 0.0) continue;
    for (; next_e < n; ++next_e) {
      for (int64_t k = 0; k < n; ++k) A_(k, c) = (k == next_e) ? 1.0 : 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t q = 0; q < m; ++q) {
          if (q == c || (S[q] == 0.0 && q > c)) continue;
          double d = 0.0;
          for (int64_t k = 0; k < n; ++k) d += A_(k, q) * A_(k, c);
          for (int64_t k = 0; k < n; ++k) A_(k, c) -= d * A_(k, q);
        }
      }
      double nn = 0.0;
      for (int64_t k = 0; k < n; ++k) nn += A_(k, c) * A_(k, c);
      nn = sqrt(nn);
      if (nn > 0.5) {
        for (int64_t k = 0; k < n; ++k) A_(k, c) /= nn;
        ++next_e;
        break;
      }
    }
  }
  /* sign convention: largest-magnitude entry of v_i positive */
  for (int64_t c = 0; c < m; ++c) {
    int64_t kmax = 0;
    double vmax = -1.0;
    for (int64_t k = 0; k < m; ++k) {
      double a = fabs(V[c * ldv + k]);
      if (a > vmax) { vmax = a; kmax = k; }
    }
    if (V[c * ldv + kmax] < 0.0) {
      for (int64_t k = 0; k < m; ++k) V[c * ldv + k] = -V[c * ldv + k];
      for (int64_t k = 0; k < n; ++k) A_(k, c) = -A_(k, c);
    }
  }
  free(perm); free(A2); free(V2); free(S2);
}

/* Full SVD of an n x m matrix (n >= m) by Jacobi, sorted and sign-fixed:
 * A := U (n x m), S (m), V (m x m).  Returns sweeps or -1. */
int oracle_svd_jacobi_sorted(double* A, int64_t n, int64_t m, int64_t lda,
                             double* S, double* V, int64_t ldv, int max_sweeps) {
  int sw = oracle_jacobi_svd(A, n, m, lda, S, V, ldv, max_sweeps);
  sort_normalise_sign(A, n, m, lda, S, V, ldv);
  return sw;
}

/* Energy truncation (Sec. 3.1 cumulative energy; truncate() of Alg. 3). */
int64_t oracle_truncation_rank(const double* S, int64_t m, double energy,
                               int64_t r_max) {
  if (r_max > m) r_max = m;
  if (energy <= 0.0) return r_max;
  double total = 0.0;
  for (int64_t i = 0; i < m; ++i) total += S[i] * S[i];
  if (total == 0.0) return r_max;
  double acc = 0.0;
  for (int64_t k = 0; k < m; ++k) {
    acc += S[k] * S[k];
    if (acc / total >= energy) return (k + 1 < r_max) ? k + 1 : r_max;
  }
  return r_max;
}

/* ------------------------------------------------------------------------
 * POD (Alg. 2 with tsqr_svd of Alg. 1 replaced by its exact result):
 *   Y_w = diag(sqrt w)(X - xbar 1^T);  Y_w = Q [R; 0];  R = U_r S V^T;
 *   U = Q [U_r; 0]  (Eqs. svdqr1-svdqr3).
 * Outputs: U (N x r, first r columns of ldu-strided storage), S (M),
 * VT (M x M, row i = v_i^T, the temporal coefficients of mode i), mean
 * (N, nullable), r.  mode_kind 0: U = left singular vectors of Y_w
 * (Euclidean-orthonormal); 1: physical modes Phi = diag(w)^(-1/2) U,
 * orthonormal in the w-weighted inner product.
 * Returns Jacobi sweeps, or -1 on non-convergence.
 * ------------------------------------------------------------------------ */
int oracle_pod(const double* X, int64_t N, int64_t M, int64_t ldx,
               const double* w, int remove_mean, double energy, int64_t r_max,
               int mode_kind, double* U, int64_t ldu, double* S, double* VT,
               int64_t ldvt, double* mean, int64_t* r_out, int max_sweeps) {
  double* Y = (double*)malloc(sizeof(double) * N * M);
  double* tau = (double*)malloc(sizeof(double) * M);
  double* R = (double*)malloc(sizeof(double) * M * M);
  double* V = (double*)malloc(sizeof(double) * M * M);
  oracle_center_weight(X, N, M, ldx, w, remove_mean, Y, N, mean);
  oracle_householder_qr(Y, N, M, N, tau);
  for (int64_t j = 0; j < M; ++j)
    for (int64_t i = 0; i < M; ++i) R[j * M + i] = (i <= j) ? Y[j * N + i] : 0.0;
  int sweeps = oracle_svd_jacobi_sorted(R, M, M, M, S, V, M, max_sweeps);
  int64_t r = oracle_truncation_rank(S, M, energy, r_max);
  *r_out = r;
  /* U = Q [U_r(:, 0:r); 0] */
  for (int64_t c = 0; c < r; ++c) {
    double* col = U + c * ldu;
    for (int64_t i = 0; i < N; ++i) col[i] = (i < M) ? R[c * M + i] : 0.0;
  }
  oracle_apply_q(Y, N, M, N, tau, U, r, ldu);
  if (mode_kind == 1 && w) {
    for (int64_t c = 0; c < r; ++c)
      for (int64_t i = 0; i < N; ++i) U[c * ldu + i] /= sqrt(w[i]);
  }
  for (int64_t i = 0; i < M; ++i)
    for (int64_t k = 0; k < M; ++k) VT[k * ldvt + i] = V[i * M + k];
  free(Y); free(tau); free(R); free(V);
  return sweeps;
}

/* ------------------------------------------------------------------------
 * TSQR result of Alg. 1 (Q_i and R) by its definition: the Householder QR
 * of the whole matrix.  R: M x M (upper), Q: N x M explicit (nullable).
 * R's rows are fixed only up to sign by the definition; callers compare
 * R^T R, |R_ii| or products such as Q R.
 * ------------------------------------------------------------------------ */
void oracle_tsqr(const double* A, int64_t N, int64_t M, int64_t lda, double* R,
                 int64_t ldr, double* Q, int64_t ldq) {
  double* Y = (double*)malloc(sizeof(double) * N * M);
  double* tau = (double*)malloc(sizeof(double) * M);
  for (int64_t j = 0; j < M; ++j) memcpy(Y + j * N, A + j * lda, sizeof(double) * N);
  oracle_householder_qr(Y, N, M, N, tau);
  for (int64_t j = 0; j < M; ++j)
    for (int64_t i = 0; i < M; ++i) R[j * ldr + i] = (i <= j) ? Y[j * N + i] : 0.0;
  if (Q) {
    for (int64_t j = 0; j < M; ++j)
      for (int64_t i = 0; i < N; ++i) Q[j * ldq + i] = (i == j) ? 1.0 : 0.0;
    oracle_apply_q(Y, N, M, N, tau, Q, M, ldq);
  }
  free(Y); free(tau);
}

/* ------------------------------------------------------------------------
 * Local product of Alg. 4 (matmul_paral) on one process: C = op(A) B,
 * op(A) = A (m x k) or A^T (A stored k x m).  All column-major.
 * ------------------------------------------------------------------------ */
void oracle_matmul(int transA, const double* A, const double* B, double* C,
                   int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                   int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t p = 0; p < k; ++p) {
        double a = transA ? A[i * lda + p] : A[p * lda + i];
        s += a * B[j * ldb + p];
      }
      C[j * ldc + i] = s;
    }
}

/* ------------------------------------------------------------------------
 * Truncated-POD reconstruction loss and its gradient.
 * L(X) = || (I - U_r U_r^T) Y_w ||_F^2 = sum_{i>r} s_i^2, with Y_w the
 * weighted (and optionally centred) snapshot matrix of Alg. 2 and U_r its
 * r leading left singular vectors (Eqs. svdqr1-svdqr3).  Where s_r > s_{r+1}
 * the derivative of sum_{i<=r} s_i^2 is 2 U_r U_r^T Y_w, so
 *   dL/dY_w = 2 (I - U_r U_r^T) Y_w,
 *   dL/dX   = diag(sqrt w) dL/dY_w (I - 1 1^T / M if the mean is removed).
 * Returns L; writes G (N x M, ldg) when G != NULL.
 * ------------------------------------------------------------------------ */
double oracle_pod_loss_grad(const double* X, int64_t N, int64_t M, int64_t ldx,
                            const double* w, int remove_mean, int64_t r, double* G,
                            int64_t ldg) {
  double* Y = (double*)malloc(sizeof(double) * N * M);
  double* U = (double*)malloc(sizeof(double) * N * (r > 0 ? r : 1));
  double* S = (double*)malloc(sizeof(double) * M);
  double* VT = (double*)malloc(sizeof(double) * M * M);
  double* C = (double*)malloc(sizeof(double) * (r > 0 ? r : 1) * M);
  int64_t rr = 0;
  oracle_center_weight(X, N, M, ldx, w, remove_mean, Y, N, NULL);
  oracle_pod(X, N, M, ldx, w, remove_mean, 0.0, r, 0, U, N, S, VT, M, NULL, &rr, 60);
  double L = 0.0;
  for (int64_t i = r; i < M; ++i) L += S[i] * S[i];
  if (G) {
    /* C = U_r^T Y_w (r x M), then G = 2 (Y_w - U_r C) */
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m)
      for (int64_t i = 0; i < r; ++i) {
        double s = 0.0;
        for (int64_t n = 0; n < N; ++n) s += U[i * N + n] * Y[m * N + n];
        C[m * r + i] = s;
      }
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
      double swn = w ? sqrt(w[n]) : 1.0;
      double rowsum = 0.0;
      for (int64_t m = 0; m < M; ++m) {
        double p = 0.0;
        for (int64_t i = 0; i < r; ++i) p += U[i * N + n] * C[m * r + i];
        double g = 2.0 * (Y[m * N + n] - p) * swn;
        G[m * ldg + n] = g;
        rowsum += g;
      }
      if (remove_mean) {
        double mu = rowsum / (double)M;
        for (int64_t m = 0; m < M; ++m) G[m * ldg + n] -= mu;
      }
    }
  }
  free(Y); free(U); free(S); free(VT); free(C);
  return L;
}

/* ========================================================================
 * Complex (binary64) SVD of a tall matrix, for the per-frequency SVDs of
 * SPOD (Sec. 2.3, Alg. 6: (1/sqrt(nBlks)) Q_f = U_f S_f V_f^H).  Same route
 * as the real POD: Householder QR, one-sided Jacobi on R, U = Q [U_r; 0].
 * ======================================================================== */
typedef double complex zc;
#define Z_(i, j) A[(int64_t)(j) * lda + (i)]

/* Householder QR with complex reflectors: H_j = I - tau_j v_j v_j^H,
 * H_j^H [alpha; x] = [beta; 0] with beta real, beta = -sign(Re alpha)|[alpha; x]|
 * (sign(0) = +1), tau_j = (beta - alpha) / beta, v_j = [1; x / (alpha - beta)];
 * A = Q [R; 0] with Q = H_0 H_1 ... H_{m-1}.  A column that is already
 * [real; 0] gets tau = 0. */
void oracle_zhouseholder_qr(zc* A, int64_t n, int64_t m, int64_t lda, zc* tau) {
  for (int64_t j = 0; j < m; ++j) {
    zc alpha = Z_(j, j);
    double xx = 0.0;
    for (int64_t i = j + 1; i < n; ++i) xx += creal(Z_(i, j) * conj(Z_(i, j)));
    if (xx == 0.0 && cimag(alpha) == 0.0) { tau[j] = 0.0; continue; }
    double nrm = sqrt(creal(alpha) * creal(alpha) + cimag(alpha) * cimag(alpha) + xx);
    double beta = (creal(alpha) >= 0.0) ? -nrm : nrm;
    tau[j] = (beta - alpha) / beta;
    zc scal = 1.0 / (alpha - beta);
    for (int64_t i = j + 1; i < n; ++i) Z_(i, j) *= scal;
    Z_(j, j) = beta;
    /* apply H_j^H = I - conj(tau) v v^H to the trailing columns */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < m; ++k) {
      zc s = Z_(j, k);
      for (int64_t i = j + 1; i < n; ++i) s += conj(Z_(i, j)) * Z_(i, k);
      s *= conj(tau[j]);
      Z_(j, k) -= s;
      for (int64_t i = j + 1; i < n; ++i) Z_(i, k) -= s * Z_(i, j);
    }
  }
}

/* C := Q C (C is n x k). */
void oracle_zapply_q(const zc* A, int64_t n, int64_t m, int64_t lda, const zc* tau, zc* C, int64_t k,
                     int64_t ldc) {
  for (int64_t j = m - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < k; ++c) {
      zc* col = C + c * ldc;
      zc s = col[j];
      for (int64_t i = j + 1; i < n; ++i) s += conj(Z_(i, j)) * col[i];
      s *= tau[j];
      col[j] -= s;
      for (int64_t i = j + 1; i < n; ++i) col[i] -= s * Z_(i, j);
    }
  }
}

/* One-sided complex Jacobi: for a pair with gamma = a_i^H a_j = |gamma| e^{i phi}
 * the real rotation of the real case (zeta = (beta - alpha) / (2|gamma|)) acts
 * on [a_i, e^{-i phi} a_j]:  a_i <- c a_i - s e^{-i phi} a_j,
 * a_j <- s a_i + c e^{-i phi} a_j, and the same on V.  Cyclic by row;
 * rotate while |gamma| > n 2^-53 sqrt(alpha beta).  Returns sweeps or -1. */
int oracle_zjacobi_svd(zc* A, int64_t n, int64_t m, int64_t lda, double* S, zc* V, int64_t ldv,
                       int max_sweeps) {
  const double tol = (double)n * ldexp(1.0, -53);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) V[j * ldv + i] = (i == j) ? 1.0 : 0.0;
  int sweep = 0, converged = 0;
  while (sweep < max_sweeps && !converged) {
    int rotated = 0;
    for (int64_t i = 0; i < m - 1; ++i) {
      for (int64_t j = i + 1; j < m; ++j) {
        double alpha = 0.0, beta = 0.0;
        zc gamma = 0.0;
        for (int64_t k = 0; k < n; ++k) {
          alpha += creal(conj(Z_(k, i)) * Z_(k, i));
          beta += creal(conj(Z_(k, j)) * Z_(k, j));
          gamma += conj(Z_(k, i)) * Z_(k, j);
        }
        double g = cabs(gamma);
        if (g == 0.0 || g <= tol * sqrt(alpha * beta)) continue;
        rotated = 1;
        zc eph = conj(gamma) / g; /* e^{-i phi} */
        double zeta = (beta - alpha) / (2.0 * g);
        double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t k = 0; k < n; ++k) {
          zc ai = Z_(k, i), aj = eph * Z_(k, j);
          Z_(k, i) = c * ai - s * aj;
          Z_(k, j) = s * ai + c * aj;
        }
        for (int64_t k = 0; k < m; ++k) {
          zc vi = V[i * ldv + k], vj = eph * V[j * ldv + k];
          V[i * ldv + k] = c * vi - s * vj;
          V[j * ldv + k] = s * vi + c * vj;
        }
      }
    }
    ++sweep;
    if (!rotated) converged = 1;
  }
  for (int64_t i = 0; i < m; ++i) {
    double ss = 0.0;
    for (int64_t k = 0; k < n; ++k) ss += creal(conj(Z_(k, i)) * Z_(k, i));
    S[i] = sqrt(ss);
  }
  return converged ? sweep : -1;
}

/* Complex SVD X = U diag(S) V^H of an N x M (N >= M) matrix by QR + Jacobi:
 * sorted descending (stable), each pair (u_i, v_i) multiplied by the unit
 * phase that makes the largest-magnitude entry of v_i real and positive
 * (lowest index on ties).  Outputs U (N x k, first k columns), S (M),
 * V (M x M).  Zero singular values are not completed (U columns left 0).
 * Returns Jacobi sweeps or -1. */
int oracle_zsvd(const zc* X, int64_t N, int64_t M, int64_t ldx, int64_t k, zc* U, int64_t ldu,
                double* S, zc* V, int64_t ldv, int max_sweeps) {
  zc* Y = (zc*)malloc(sizeof(zc) * N * M);
  zc* tau = (zc*)malloc(sizeof(zc) * M);
  zc* R = (zc*)malloc(sizeof(zc) * M * M);
  zc* Vw = (zc*)malloc(sizeof(zc) * M * M);
  double* Sw = (double*)malloc(sizeof(double) * M);
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * M);
  for (int64_t j = 0; j < M; ++j) memcpy(Y + j * N, X + j * ldx, sizeof(zc) * N);
  oracle_zhouseholder_qr(Y, N, M, N, tau);
  for (int64_t j = 0; j < M; ++j)
    for (int64_t i = 0; i < M; ++i) R[j * M + i] = (i <= j) ? Y[j * N + i] : 0.0;
  int sw = oracle_zjacobi_svd(R, M, M, M, Sw, Vw, M, max_sweeps);
  for (int64_t i = 0; i < M; ++i) perm[i] = i;
  for (int64_t i = 1; i < M; ++i) {
    int64_t p = perm[i], q = i;
    while (q > 0 && Sw[perm[q - 1]] < Sw[p]) { perm[q] = perm[q - 1]; --q; }
    perm[q] = p;
  }
  for (int64_t c = 0; c < M; ++c) {
    int64_t p = perm[c];
    S[c] = Sw[p];
    int64_t kmax = 0;
    double vmax = -1.0;
    for (int64_t q = 0; q < M; ++q) {
      double a = cabs(Vw[p * M + q]);
      if (a > vmax) { vmax = a; kmax = q; }
    }
    zc ph = (vmax > 0.0) ? conj(Vw[p * M + kmax]) / vmax : 1.0;
    for (int64_t q = 0; q < M; ++q) V[c * ldv + q] = Vw[p * M + q] * ph;
    if (c < k) {
      zc* col = U + c * ldu;
      for (int64_t i = 0; i < N; ++i) col[i] = (i < M && Sw[p] > 0.0) ? R[p * M + i] * ph / Sw[p] : 0.0;
    }
  }
  oracle_zapply_q(Y, N, M, N, tau, U, k, ldu);
  free(Y); free(tau); free(R); free(Vw); free(Sw); free(perm);
  return sw;
}

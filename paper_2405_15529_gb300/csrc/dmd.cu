// dmd.cu -- exact DMD with optimal amplitudes on one device (pyLOM, arXiv
// 2405.15529, Sec. 3.2, Alg. 3, Alg. 4's product, Alg. 5).
//
// One TSQR of the whole (centred) snapshot matrix Y = Q R (N x M) carries
// the method.  The QR of Y1 = Y[:, :M-1] is the leading part of it,
// Y1 = Q[:, :M-1] R[:M-1, :M-1], and Y2 = Y[:, 1:] = Q R[:, 1:], so with
// R[:M-1, :M-1] = U_R S V^T (U = Q [U_R; 0]):
//   A   = U^T Y2 V S^-1 = U_R^T R[:M-1, 1:] V S^-1           (r x r)
//   phi = Y2 V S^-1 w / mu = Q (R[:, 1:] V S^-1 w / mu)        (N x r)
// Everything between the leaf QR and the modes product works on matrices
// of at most M rows; the data is read once (leaf QR) and the reflectors
// once (modes), as for the POD.
//
// Small steps (one device, r = the truncation rank):
//   rank cap        r <= count of s_k > max(N, M-1) 2^-52 s_1 (the numerical
//                   rank of Y1; S^-1 must exist);
//   T1 = R[:, 1:] V S^-1 (M x r), A = U_R^T T1[:M-1] (r x r);
//   eigen(A)        Householder Hessenberg reduction, then Francis
//                   double-shift QR to the real Schur form T = Z^T A Z
//                   (one thread block), eigenvectors of T by back
//                   substitution, w = Z x, each normalised to unit norm with
//                   its (first) entry of largest modulus real and positive;
//   amplitudes      P = (w^H w) o conj(V_and V_and^H) with V_and[i, t] =
//                   mu_i^t (t < M-1), q = conj(diag(V_and V S w)), P = L L^H
//                   (Cholesky), b = L^-H L^-1 q  (Alg. 5; the conjugate in P
//                   is the one the least-squares objective requires);
//   order           by |b| descending, a conjugate pair sharing the larger
//                   |b| of its members, adjacent, positive imaginary part
//                   first;
//   modes           B = T1 w / mu packed real (a conjugate pair stores the
//                   real and imaginary parts of its first member, as in
//                   LAPACK's real eigenvector layout), then Q [B; 0] by the
//                   POD's top-down pass and leaf modes kernels.
#include <float.h>

#include "kernels.h"

namespace pylom {
namespace {

constexpr int kEigThreads = 256;
constexpr int kSmallThreads = 256;
constexpr double kEps = 2.220446049250313e-16;    // 2^-52
constexpr size_t kEigSmemCap = 190 * 1024;        // H (and Z) resident in shared memory up to this

struct DmdState {
  int64_t M, M1, rmax;
  double* UR;          // M1 x M1 left singular vectors of R[:M1, :M1] (ld M1)
  double* VT;          // M1 x M1 (ld M1), row k = v_k^T
  double* T1;          // M x rmax (ld M): R[:, 1:] V S^-1
  double* H;           // rmax x rmax (ld rmax): A, Hessenberg form, real Schur form
  double* Z;           // rmax x rmax (ld rmax): Schur vectors
  double *Xr, *Xi;     // rmax x rmax: eigenvectors of the Schur form
  double *Wr, *Wi;     // rmax x rmax: eigenvectors of A, normalised
  double *mur, *mui;   // rmax: eigenvalues in Schur order
  int* flag;           // rmax: 0 real, 1 / 2 first (Im > 0) / second member of a conjugate pair
  double *Pr, *Pi;     // rmax x rmax: P (lower triangle), then its Cholesky factor
  double *qr, *qi;     // rmax: q, then y, then b (Schur order)
  double* key;         // rmax: sort keys
  int* perm;           // rmax: sorted position -> Schur index
  double* Bp;          // M x rmax (ld M): packed small modes
};

size_t dmd_small_bytes(int64_t M, int64_t rmax) {
  const int64_t M1 = M - 1;
  const size_t d = sizeof(double);
  size_t b = 0;
  b += 2 * align256(d * (size_t)M1 * M1);                   // UR, VT
  b += 2 * align256(d * (size_t)M * rmax);                  // T1, Bp
  b += 8 * align256(d * (size_t)rmax * rmax);               // H, Z, Xr, Xi, Wr, Wi, Pr, Pi
  b += 5 * align256(d * (size_t)rmax);                      // mur, mui, qr, qi, key
  b += 2 * align256(sizeof(int) * (size_t)rmax);            // flag, perm
  return b;
}

void dmd_small_carve(DmdState& d, char* p, int64_t M, int64_t rmax) {
  d.M = M;
  d.M1 = M - 1;
  d.rmax = rmax;
  const size_t dd = sizeof(double);
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
  d.UR = (double*)take(dd * (size_t)d.M1 * d.M1);
  d.VT = (double*)take(dd * (size_t)d.M1 * d.M1);
  d.T1 = (double*)take(dd * (size_t)M * rmax);
  d.Bp = (double*)take(dd * (size_t)M * rmax);
  d.H = (double*)take(dd * (size_t)rmax * rmax);
  d.Z = (double*)take(dd * (size_t)rmax * rmax);
  d.Xr = (double*)take(dd * (size_t)rmax * rmax);
  d.Xi = (double*)take(dd * (size_t)rmax * rmax);
  d.Wr = (double*)take(dd * (size_t)rmax * rmax);
  d.Wi = (double*)take(dd * (size_t)rmax * rmax);
  d.Pr = (double*)take(dd * (size_t)rmax * rmax);
  d.Pi = (double*)take(dd * (size_t)rmax * rmax);
  d.mur = (double*)take(dd * (size_t)rmax);
  d.mui = (double*)take(dd * (size_t)rmax);
  d.qr = (double*)take(dd * (size_t)rmax);
  d.qi = (double*)take(dd * (size_t)rmax);
  d.key = (double*)take(dd * (size_t)rmax);
  d.flag = (int*)take(sizeof(int) * (size_t)rmax);
  d.perm = (int*)take(sizeof(int) * (size_t)rmax);
}

__device__ __forceinline__ int64_t dmd_rank(const WsHeader* h) { return *((volatile const long long*)&h->r); }

// complex helpers (re, im pairs)
struct cx {
  double re, im;
};
__device__ __forceinline__ cx cmul(cx a, cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cx csub(cx a, cx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ double cabs2(cx a) { return a.re * a.re + a.im * a.im; }
// a / b by Smith's scaling (no overflow of |b|^2 for large b)
__device__ __forceinline__ cx cdiv(cx a, cx b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  }
  const double r = b.re / b.im, den = b.im + b.re * r;
  return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}

template <int K>
__device__ __forceinline__ void block_sum_small(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = warp_sum(v[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) red[q * 32 + warp] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[q * 32 + w];
    v[q] = s;
  }
}

// ---------------------------------------------------------------------------
// rank cap, T1, A
// ---------------------------------------------------------------------------

__global__ void dmd_rank_kernel(WsHeader* hdr, const double* S, int64_t N, int64_t M1) {
  if (read_status(hdr) != 0) return;
  const double s0 = S[0];
  const double tol = (double)(N > M1 ? N : M1) * kEps * s0;
  long long cnt = 0;
  for (int64_t k = threadIdx.x; k < M1; k += 32) cnt += (s0 > 0.0 && S[k] > tol) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (threadIdx.x == 0 && cnt < hdr->r) hdr->r = cnt;
}

// T1[i, c] = sum_j R[i, j+1] V[j, c] / s_c over j >= i - 1 (R upper triangular, ld M)
__global__ void dmd_t1_kernel(DmdState d, const double* R, const double* S, const WsHeader* hdr) {
  const int64_t r = dmd_rank(hdr);
  if (read_status(hdr) != 0) return;
  const int64_t M = d.M, M1 = d.M1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * r;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, c = idx / M;
    double s = 0.0;
    for (int64_t j = (i > 0 ? i - 1 : 0); j < M1; ++j) s = fma(R[i + (j + 1) * M], d.VT[c + j * M1], s);
    d.T1[i + c * M] = s / S[c];
  }
}

// A[a, c] = sum_{i < M1} U_R[i, a] T1[i, c]
__global__ void dmd_a_kernel(DmdState d, const WsHeader* hdr) {
  const int64_t r = dmd_rank(hdr);
  if (read_status(hdr) != 0) return;
  const int64_t M = d.M, M1 = d.M1, ld = d.rmax;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < r * r;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = idx % r, c = idx / r;
    const double* u = d.UR + a * M1;
    const double* t = d.T1 + c * M;
    double s = 0.0;
    for (int64_t i = 0; i < M1; ++i) s = fma(u[i], t[i], s);
    d.H[a + c * ld] = s;
  }
}

// ---------------------------------------------------------------------------
// eigendecomposition of A (one thread block)
// ---------------------------------------------------------------------------

#define HH(i, j) H[(i) + (int64_t)(j) * ldh]
#define ZZ(i, j) Z[(i) + (int64_t)(j) * ldz]

// Householder reduction to upper Hessenberg form, H := P^T H P, Z := Z P.
// Reflector k maps H[k+1:, k] to beta e_1: P = I - tau v v^T, v[0] = 1.
__device__ void hessenberg_reduce(double* H, int64_t ldh, double* Z, int64_t ldz, int64_t n, double* sv,
                                  double* red, double* sc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int64_t k = 0; k + 2 < n; ++k) {
    double part[1] = {0.0};
    for (int64_t i = k + 2 + tid; i < n; i += blockDim.x) {
      const double v = HH(i, k);
      part[0] = fma(v, v, part[0]);
    }
    block_sum_small<1>(part, red);
    if (tid == 0) {
      const double sigma = part[0], alpha = HH(k + 1, k);
      double tau = 0.0, beta = alpha, scale = 0.0;
      if (sigma > 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sigma));
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      sc[0] = tau;
      sc[1] = beta;
      sc[2] = scale;
    }
    __syncthreads();
    const double tau = sc[0], beta = sc[1], scale = sc[2];
    if (tau == 0.0) continue;   // column already reduced (uniform branch)
    const int64_t m = n - k - 1;
    for (int64_t i = tid; i < m; i += blockDim.x) sv[i] = (i == 0) ? 1.0 : HH(k + 1 + i, k) * scale;
    __syncthreads();
    for (int64_t i = k + 1 + tid; i < n; i += blockDim.x) HH(i, k) = (i == k + 1) ? beta : 0.0;
    // H[k+1:, k+1:] := P H[k+1:, k+1:]   (a warp per column)
    for (int64_t j = k + 1 + warp; j < n; j += nw) {
      double s = 0.0;
      for (int64_t i = lane; i < m; i += 32) s = fma(sv[i], HH(k + 1 + i, j), s);
      s = warp_sum(s) * tau;
      for (int64_t i = lane; i < m; i += 32) HH(k + 1 + i, j) -= s * sv[i];
    }
    __syncthreads();
    // H[:, k+1:] := H[:, k+1:] P,  Z[:, k+1:] := Z[:, k+1:] P   (a thread per row)
    for (int64_t i = tid; i < n; i += blockDim.x) {
      double s = 0.0, t = 0.0;
      for (int64_t j = 0; j < m; ++j) {
        s = fma(HH(i, k + 1 + j), sv[j], s);
        t = fma(ZZ(i, k + 1 + j), sv[j], t);
      }
      s *= tau;
      t *= tau;
      for (int64_t j = 0; j < m; ++j) {
        HH(i, k + 1 + j) -= s * sv[j];
        ZZ(i, k + 1 + j) -= t * sv[j];
      }
    }
    __syncthreads();
  }
}

// P = I - tau v v^T with v = [1, v1, v2] mapping (x, y, z) to (beta, 0, 0)
__device__ __forceinline__ void reflector3(double x, double y, double z, double& tau, double& v1, double& v2) {
  const double sigma = fma(y, y, z * z);
  tau = 0.0;
  v1 = 0.0;
  v2 = 0.0;
  if (sigma > 0.0) {
    const double nrm = sqrt(fma(x, x, sigma));
    const double beta = x >= 0.0 ? -nrm : nrm;
    tau = (beta - x) / beta;
    const double inv = 1.0 / (x - beta);
    v1 = y * inv;
    v2 = z * inv;
  }
}

// One implicit double-shift (Francis) QR step on the active window [l, hi]
// of the full matrix: the first column of (H - s1 I)(H - s2 I) for the two
// eigenvalues s1, s2 of the window's trailing 2 x 2 block (or an ad hoc
// exceptional shift after 10 and 20 fruitless steps), a bulge introduced at
// the top of the window and chased to its bottom by 3 x 3 reflectors.  The
// reflectors are applied to whole rows (to column n-1) and whole columns
// (from row 0) so that H converges to the full real Schur form, and to Z.
__device__ void francis_step(double* H, int64_t ldh, double* Z, int64_t ldz, int64_t n, int64_t l, int64_t hi,
                             int its, double* sc) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    double s, t;
    if (its == 10 || its == 20) {
      const double w = fabs(HH(hi, hi - 1)) + fabs(HH(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      const double a = HH(hi - 1, hi - 1), b = HH(hi - 1, hi), c = HH(hi, hi - 1), dd = HH(hi, hi);
      s = a + dd;
      t = a * dd - b * c;
    }
    const double h00 = HH(l, l), h10 = HH(l + 1, l), h01 = HH(l, l + 1), h11 = HH(l + 1, l + 1);
    const double h21 = HH(l + 2, l + 1);
    sc[0] = h00 * h00 + h01 * h10 - s * h00 + t;
    sc[1] = h10 * (h00 + h11 - s);
    sc[2] = h10 * h21;
  }
  __syncthreads();
  for (int64_t k = l; k <= hi - 2; ++k) {
    if (tid == 0) {
      double tau, v1, v2;
      reflector3(sc[0], sc[1], sc[2], tau, v1, v2);
      sc[3] = tau;
      sc[4] = v1;
      sc[5] = v2;
    }
    __syncthreads();
    const double tau = sc[3], v1 = sc[4], v2 = sc[5];
    if (tau != 0.0) {
      const int64_t j0 = k > l ? k - 1 : l;
      for (int64_t j = j0 + tid; j < n; j += blockDim.x) {
        double* c = H + j * ldh;
        const double s = tau * (c[k] + v1 * c[k + 1] + v2 * c[k + 2]);
        c[k] -= s;
        c[k + 1] -= s * v1;
        c[k + 2] -= s * v2;
        if (j == k - 1) {   // the bulge's column: exactly reduced
          c[k + 1] = 0.0;
          c[k + 2] = 0.0;
        }
      }
    }
    __syncthreads();
    if (tau != 0.0) {
      const int64_t i1 = (k + 3 < hi) ? k + 3 : hi;
      for (int64_t i = tid; i <= i1; i += blockDim.x) {
        const double s = tau * (HH(i, k) + v1 * HH(i, k + 1) + v2 * HH(i, k + 2));
        HH(i, k) -= s;
        HH(i, k + 1) -= s * v1;
        HH(i, k + 2) -= s * v2;
      }
      for (int64_t i = tid; i < n; i += blockDim.x) {
        const double s = tau * (ZZ(i, k) + v1 * ZZ(i, k + 1) + v2 * ZZ(i, k + 2));
        ZZ(i, k) -= s;
        ZZ(i, k + 1) -= s * v1;
        ZZ(i, k + 2) -= s * v2;
      }
    }
    __syncthreads();
    if (tid == 0) {
      sc[0] = HH(k + 1, k);
      sc[1] = HH(k + 2, k);
      sc[2] = (k < hi - 2) ? HH(k + 3, k) : 0.0;
    }
    __syncthreads();
  }
  // last, 2 x 2 reflector on rows hi-1, hi
  if (tid == 0) {
    double tau, v1, v2;
    reflector3(sc[0], sc[1], 0.0, tau, v1, v2);
    sc[3] = tau;
    sc[4] = v1;
  }
  __syncthreads();
  const double tau = sc[3], v1 = sc[4];
  if (tau != 0.0) {
    for (int64_t j = hi - 2 + tid; j < n; j += blockDim.x) {
      double* c = H + j * ldh;
      const double s = tau * (c[hi - 1] + v1 * c[hi]);
      c[hi - 1] -= s;
      c[hi] -= s * v1;
      if (j == hi - 2) c[hi] = 0.0;
    }
  }
  __syncthreads();
  if (tau != 0.0) {
    for (int64_t i = tid; i <= hi; i += blockDim.x) {
      const double s = tau * (HH(i, hi - 1) + v1 * HH(i, hi));
      HH(i, hi - 1) -= s;
      HH(i, hi) -= s * v1;
    }
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const double s = tau * (ZZ(i, hi - 1) + v1 * ZZ(i, hi));
      ZZ(i, hi - 1) -= s;
      ZZ(i, hi) -= s * v1;
    }
  }
  __syncthreads();
}

// A converged 2 x 2 diagonal block at rows p, p+1: with real eigenvalues it
// is rotated to upper triangular form (first column of the rotation = the
// eigenvector of the eigenvalue farther from its (1,1)... computed without
// cancellation); with complex eigenvalues it stays, and the pair is
// recorded (Im > 0 first).
__device__ void settle_2x2(double* H, int64_t ldh, double* Z, int64_t ldz, int64_t n, int64_t p, double* mur,
                           double* mui, int* flag, double* sc, int* si) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    const double a = HH(p, p), b = HH(p, p + 1), c = HH(p + 1, p), dd = HH(p + 1, p + 1);
    double cs = 1.0, sn = 0.0, re = 0.0, im = 0.0;
    int cplx = 0;
    if (c != 0.0) {
      const double pp = 0.5 * (a - dd);
      const double disc = fma(pp, pp, b * c);
      if (disc >= 0.0) {
        const double x = pp + copysign(sqrt(disc), pp);   // lambda_1 - d
        const double nrm = hypot(x, c);
        cs = x / nrm;
        sn = c / nrm;
      } else {
        cplx = 1;
        re = dd + pp;
        im = sqrt(-disc);
      }
    }
    sc[0] = cs;
    sc[1] = sn;
    sc[2] = re;
    sc[3] = im;
    si[1] = cplx;
  }
  __syncthreads();
  const double cs = sc[0], sn = sc[1];
  const int cplx = si[1];
  if (!cplx && sn != 0.0) {
    for (int64_t j = p + tid; j < n; j += blockDim.x) {
      const double x = HH(p, j), y = HH(p + 1, j);
      HH(p, j) = cs * x + sn * y;
      HH(p + 1, j) = cs * y - sn * x;
    }
    __syncthreads();
    for (int64_t i = tid; i <= p + 1; i += blockDim.x) {
      const double x = HH(i, p), y = HH(i, p + 1);
      HH(i, p) = cs * x + sn * y;
      HH(i, p + 1) = cs * y - sn * x;
    }
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const double x = ZZ(i, p), y = ZZ(i, p + 1);
      ZZ(i, p) = cs * x + sn * y;
      ZZ(i, p + 1) = cs * y - sn * x;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (cplx) {
      mur[p] = sc[2];
      mui[p] = sc[3];
      mur[p + 1] = sc[2];
      mui[p + 1] = -sc[3];
      flag[p] = 1;
      flag[p + 1] = 2;
    } else {
      HH(p + 1, p) = 0.0;
      mur[p] = HH(p, p);
      mui[p] = 0.0;
      mur[p + 1] = HH(p + 1, p + 1);
      mui[p + 1] = 0.0;
      flag[p] = 0;
      flag[p + 1] = 0;
    }
  }
  __syncthreads();
}

// Eigenvectors of the quasi-triangular T by back substitution, one thread
// per eigenvalue: x[k] = 1 (real) or the 2 x 2 block's eigenvector (pair),
// zeros below, then rows upward (2 x 2 diagonal blocks as complex 2 x 2
// solves).  Near-zero pivots are raised to smin, as perturbed eigenvalues
// would be.  A pair's second column is the conjugate of its first.
__device__ void schur_eigvecs(const double* H, int64_t ldh, int64_t n, const double* mur, const double* mui,
                              const int* flag, double* Xr, double* Xi, int64_t ldx) {
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const int fk = flag[k];
    if (fk == 2) continue;
    double* xr = Xr + k * ldx;
    double* xi = Xi + k * ldx;
    for (int64_t i = 0; i < n; ++i) {
      xr[i] = 0.0;
      xi[i] = 0.0;
    }
    const cx lam = {mur[k], mui[k]};
    const double smin = fmax(kEps * (fabs(lam.re) + fabs(lam.im)), DBL_MIN / kEps);
    int64_t top;
    if (fk == 0) {
      xr[k] = 1.0;
      top = k;
    } else {
      const double a = HH(k, k), b = HH(k, k + 1), c = HH(k + 1, k), dd = HH(k + 1, k + 1);
      if (fabs(b) >= fabs(c)) {
        xr[k] = b;
        xr[k + 1] = lam.re - a;
        xi[k + 1] = lam.im;
      } else {
        xr[k] = lam.re - dd;
        xi[k] = lam.im;
        xr[k + 1] = c;
      }
      top = k + 1;
    }
    int64_t i = k - 1;
    while (i >= 0) {
      if (i > 0 && flag[i] == 2) {
        cx r0 = {0.0, 0.0}, r1 = {0.0, 0.0};
        for (int64_t j = i + 1; j <= top; ++j) {
          const double t0 = HH(i - 1, j), t1 = HH(i, j);
          r0.re -= t0 * xr[j];
          r0.im -= t0 * xi[j];
          r1.re -= t1 * xr[j];
          r1.im -= t1 * xi[j];
        }
        const cx a11 = {HH(i - 1, i - 1) - lam.re, -lam.im}, a22 = {HH(i, i) - lam.re, -lam.im};
        const double a12 = HH(i - 1, i), a21 = HH(i, i - 1);
        cx det = csub(cmul(a11, a22), cx{a12 * a21, 0.0});
        if (cabs2(det) < smin * smin) det = {smin, 0.0};
        const cx y0 = cdiv(csub(cmul(r0, a22), cx{a12 * r1.re, a12 * r1.im}), det);
        const cx y1 = cdiv(csub(cmul(a11, r1), cx{a21 * r0.re, a21 * r0.im}), det);
        xr[i - 1] = y0.re;
        xi[i - 1] = y0.im;
        xr[i] = y1.re;
        xi[i] = y1.im;
        i -= 2;
      } else {
        cx rr = {0.0, 0.0};
        for (int64_t j = i + 1; j <= top; ++j) {
          const double t = HH(i, j);
          rr.re -= t * xr[j];
          rr.im -= t * xi[j];
        }
        cx den = {HH(i, i) - lam.re, -lam.im};
        if (cabs2(den) < smin * smin) den = {smin, 0.0};
        const cx x = cdiv(rr, den);
        xr[i] = x.re;
        xi[i] = x.im;
        i -= 1;
      }
    }
    if (fk == 1) {
      double* yr = Xr + (k + 1) * ldx;
      double* yi = Xi + (k + 1) * ldx;
      for (int64_t q = 0; q < n; ++q) {
        yr[q] = xr[q];
        yi[q] = -xi[q];
      }
    }
  }
}

// smem_mode: 0 = H and Z in global memory, 1 = H in shared memory, 2 = both.
__global__ void __launch_bounds__(kEigThreads) dmd_eig_kernel(DmdState d, WsHeader* hdr, int smem_mode) {
  extern __shared__ double dyn[];
  __shared__ double red[32];
  __shared__ double sc[8];
  __shared__ int si[4];
  const int64_t n = dmd_rank(hdr);
  if (n == 0 || read_status(hdr) != 0) return;
  const int tid = threadIdx.x;
  const int64_t ldg = d.rmax;
  const int64_t lds = d.rmax | 1;   // odd stride: no bank conflicts along rows
  double* sv = dyn;                 // Householder vector, rmax doubles
  double* H = d.H;
  double* Z = d.Z;
  int64_t ldh = ldg, ldz = ldg;
  if (smem_mode >= 1) {
    H = dyn + d.rmax;
    ldh = lds;
    for (int64_t idx = tid; idx < n * n; idx += blockDim.x) H[idx % n + (idx / n) * ldh] = d.H[idx % n + (idx / n) * ldg];
  }
  if (smem_mode == 2) {
    Z = H + lds * d.rmax;
    ldz = lds;
  }
  for (int64_t idx = tid; idx < n * n; idx += blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    ZZ(i, j) = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  hessenberg_reduce(H, ldh, Z, ldz, n, sv, red, sc);
  // a scale for the deflation test where both neighbouring diagonals vanish
  double part[1] = {0.0};
  for (int64_t idx = tid; idx < n * n; idx += blockDim.x) part[0] = fmax(part[0], fabs(H[idx % n + (idx / n) * ldh]));
  {
    const int lane = tid & 31, warp = tid >> 5;
    double v = part[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      sc[7] = m > 0.0 ? m : 1.0;
    }
    __syncthreads();
  }
  const double hscale = sc[7];
  int64_t hi = n - 1;
  int its = 0, total = 0;
  const int max_total = 60 * (int)n + 100;
  bool ok = true;
  while (hi >= 0) {
    if (tid == 0) {
      int64_t l = hi;
      while (l > 0) {
        double s = fabs(HH(l - 1, l - 1)) + fabs(HH(l, l));
        if (s == 0.0) s = hscale;
        if (fabs(HH(l, l - 1)) <= kEps * s) break;
        --l;
      }
      if (l > 0) HH(l, l - 1) = 0.0;
      si[0] = (int)l;
    }
    __syncthreads();
    const int64_t l = si[0];
    __syncthreads();
    if (l == hi) {
      if (tid == 0) {
        d.mur[hi] = HH(hi, hi);
        d.mui[hi] = 0.0;
        d.flag[hi] = 0;
      }
      hi -= 1;
      its = 0;
      continue;
    }
    if (l == hi - 1) {
      settle_2x2(H, ldh, Z, ldz, n, hi - 1, d.mur, d.mui, d.flag, sc, si);
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > max_total) {
      ok = false;
      break;
    }
    ++its;
    francis_step(H, ldh, Z, ldz, n, l, hi, its, sc);
  }
  __syncthreads();
  if (!ok) {
    if (tid == 0) raise_status(hdr, PYLOM_ERR_NOCONV);
    return;
  }
  schur_eigvecs(H, ldh, n, d.mur, d.mui, d.flag, d.Xr, d.Xi, ldg);
  if (smem_mode == 2) {
    for (int64_t idx = tid; idx < n * n; idx += blockDim.x) d.Z[idx % n + (idx / n) * ldg] = ZZ(idx % n, idx / n);
  }
}

#undef HH
#undef ZZ

// W = Z X (real times complex)
__global__ void dmd_w_kernel(DmdState d, const WsHeader* hdr) {
  const int64_t n = dmd_rank(hdr);
  if (read_status(hdr) != 0) return;
  const int64_t ld = d.rmax;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, k = idx / n;
    // x_k has no entries below row k + 1
    const int64_t top = (d.flag[k] == 0) ? k : (d.flag[k] == 1 ? k + 1 : k);
    double sr = 0.0, si = 0.0;
    for (int64_t j = 0; j <= top; ++j) {
      const double z = d.Z[i + j * ld];
      sr = fma(z, d.Xr[j + k * ld], sr);
      si = fma(z, d.Xi[j + k * ld], si);
    }
    d.Wr[i + k * ld] = sr;
    d.Wi[i + k * ld] = si;
  }
}

// Column k of W to unit norm with its (first) entry of largest modulus real
// and positive.  One block per column.
__global__ void __launch_bounds__(kSmallThreads) dmd_wnorm_kernel(DmdState d, const WsHeader* hdr) {
  __shared__ double red[64];
  __shared__ double bm[32];
  __shared__ long long bi[32];
  const int64_t n = dmd_rank(hdr);
  const int64_t k = blockIdx.x;
  if (k >= n || read_status(hdr) != 0) return;
  const int64_t ld = d.rmax;
  double* wr = d.Wr + k * ld;
  double* wi = d.Wi + k * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double nrm2[1] = {0.0};
  double best = -1.0;
  long long besti = 0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double m2 = fma(wr[i], wr[i], wi[i] * wi[i]);
    nrm2[0] += m2;
    if (m2 > best) {
      best = m2;
      besti = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, besti, o);
    if (ob > best || (ob == best && oi < besti)) {
      best = ob;
      besti = oi;
    }
  }
  if (lane == 0) {
    bm[warp] = best;
    bi[warp] = besti;
  }
  block_sum_small<1>(nrm2, red);
  if (tid == 0) {
    for (int w = 1; w < nw; ++w)
      if (bm[w] > bm[0] || (bm[w] == bm[0] && bi[w] < bi[0])) {
        bm[0] = bm[w];
        bi[0] = bi[w];
      }
  }
  __syncthreads();
  const int64_t im = bi[0];
  const double nrm = sqrt(nrm2[0]);
  const double ar = wr[im], ai = wi[im];
  const double am = hypot(ar, ai);
  __syncthreads();
  // scale by conj(w_im) / (|w_im| nrm)
  const double cr = ar / (am * nrm), ci = -ai / (am * nrm);
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double xr = wr[i], xi = wi[i];
    wr[i] = xr * cr - xi * ci;
    wi[i] = xr * ci + xi * cr;
  }
  __syncthreads();
  if (tid == 0) {
    wr[im] = am / nrm;
    wi[im] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// amplitudes (Alg. 5)
// ---------------------------------------------------------------------------

// P[i, j] = (w^H w)_ij conj(sum_t (mu_i conj(mu_j))^t), lower triangle
__global__ void dmd_p_kernel(DmdState d, const WsHeader* hdr) {
  const int64_t n = dmd_rank(hdr);
  if (read_status(hdr) != 0) return;
  const int64_t ld = d.rmax, M1 = d.M1;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    if (i < j) continue;
    double gr = 0.0, gi = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double ar = d.Wr[k + i * ld], ai = d.Wi[k + i * ld];
      const double br = d.Wr[k + j * ld], bi = d.Wi[k + j * ld];
      gr = fma(ar, br, fma(ai, bi, gr));
      gi = fma(ar, bi, fma(-ai, br, gi));
    }
    const double zr = d.mur[i] * d.mur[j] + d.mui[i] * d.mui[j];
    const double zi = d.mui[i] * d.mur[j] - d.mur[i] * d.mui[j];
    double pr = 1.0, pi = 0.0, vr = 0.0, vi = 0.0;
    for (int64_t t = 0; t < M1; ++t) {
      vr += pr;
      vi += pi;
      const double nr = pr * zr - pi * zi;
      pi = pr * zi + pi * zr;
      pr = nr;
    }
    d.Pr[i + j * ld] = gr * vr + gi * vi;
    d.Pi[i + j * ld] = gi * vr - gr * vi;
  }
}

// q_i = conj(sum_k s_k w[k, i] sum_t mu_i^t V[t, k]), one block per i
__global__ void __launch_bounds__(kSmallThreads) dmd_q_kernel(DmdState d, const double* S, const WsHeader* hdr) {
  __shared__ double red[64];
  const int64_t n = dmd_rank(hdr);
  const int64_t i = blockIdx.x;
  if (i >= n || read_status(hdr) != 0) return;
  const int64_t ld = d.rmax, M1 = d.M1;
  const double mr = d.mur[i], mi = d.mui[i];
  double acc[2] = {0.0, 0.0};
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    double cr = 0.0, ci = 0.0, pr = 1.0, pi = 0.0;
    for (int64_t t = 0; t < M1; ++t) {
      const double v = d.VT[k + t * M1];
      cr = fma(pr, v, cr);
      ci = fma(pi, v, ci);
      const double nr = pr * mr - pi * mi;
      pi = pr * mi + pi * mr;
      pr = nr;
    }
    const double wr = d.Wr[k + i * ld] * S[k], wi = d.Wi[k + i * ld] * S[k];
    acc[0] += wr * cr - wi * ci;
    acc[1] += wr * ci + wi * cr;
  }
  block_sum_small<2>(acc, red);
  if (threadIdx.x == 0) {
    d.qr[i] = acc[0];
    d.qi[i] = -acc[1];
  }
}

// Cholesky P = L L^H, b = L^-H L^-1 q, the order of the modes, the sorted
// eigenvalues and amplitudes (interleaved re, im).  One block.
__global__ void __launch_bounds__(kSmallThreads) dmd_amp_kernel(DmdState d, WsHeader* hdr, double* mu_out,
                                                                double* b_out) {
  __shared__ double sc[4];
  const int64_t n = dmd_rank(hdr);
  if (n == 0 || read_status(hdr) != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int64_t ld = d.rmax;
  double* Pr = d.Pr;
  double* Pi = d.Pi;
  for (int64_t k = 0; k < n; ++k) {
    if (tid == 0) {
      const double dk = Pr[k + k * ld];
      sc[0] = (dk > 0.0) ? sqrt(dk) : -1.0;
      if (!(dk > 0.0)) raise_status(hdr, PYLOM_ERR_SINGULAR);
    }
    __syncthreads();
    const double dk = sc[0];
    if (dk < 0.0) return;
    const double inv = 1.0 / dk;
    for (int64_t i = k + 1 + tid; i < n; i += blockDim.x) {
      Pr[i + k * ld] *= inv;
      Pi[i + k * ld] *= inv;
    }
    if (tid == 0) {
      Pr[k + k * ld] = dk;
      Pi[k + k * ld] = 0.0;
    }
    __syncthreads();
    for (int64_t j = k + 1 + warp; j < n; j += nw) {
      const double ljr = Pr[j + k * ld], lji = -Pi[j + k * ld];   // conj(L[j, k])
      for (int64_t i = j + lane; i < n; i += 32) {
        const double lir = Pr[i + k * ld], lii = Pi[i + k * ld];
        Pr[i + j * ld] -= lir * ljr - lii * lji;
        Pi[i + j * ld] -= lir * lji + lii * ljr;
      }
    }
    __syncthreads();
  }
  // L y = q
  double* qr = d.qr;
  double* qi = d.qi;
  for (int64_t i = 0; i < n; ++i) {
    if (tid == 0) {
      const double inv = 1.0 / Pr[i + i * ld];
      qr[i] *= inv;
      qi[i] *= inv;
    }
    __syncthreads();
    const double yr = qr[i], yi = qi[i];
    for (int64_t j = i + 1 + tid; j < n; j += blockDim.x) {
      const double lr = Pr[j + i * ld], li = Pi[j + i * ld];
      qr[j] -= lr * yr - li * yi;
      qi[j] -= lr * yi + li * yr;
    }
    __syncthreads();
  }
  // L^H b = y
  for (int64_t i = n - 1; i >= 0; --i) {
    if (tid == 0) {
      const double inv = 1.0 / Pr[i + i * ld];
      qr[i] *= inv;
      qi[i] *= inv;
    }
    __syncthreads();
    const double br = qr[i], bi = qi[i];
    for (int64_t j = tid; j < i; j += blockDim.x) {
      const double lr = Pr[i + j * ld], li = -Pi[i + j * ld];   // conj(L[i, j])
      qr[j] -= lr * br - li * bi;
      qi[j] -= lr * bi + li * br;
    }
    __syncthreads();
  }
  // sort keys: |b|, a conjugate pair sharing the larger of its two
  for (int64_t i = tid; i < n; i += blockDim.x) {
    double kk = hypot(qr[i], qi[i]);
    if (d.flag[i] == 1) kk = fmax(kk, hypot(qr[i + 1], qi[i + 1]));
    if (d.flag[i] == 2) kk = fmax(kk, hypot(qr[i - 1], qi[i - 1]));
    d.key[i] = (kk >= 0.0) ? kk : -1.0;   // a NaN amplitude sorts last (ranks stay a permutation)
  }
  __syncthreads();
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double ki = d.key[i];
    const int64_t gi = (d.flag[i] == 2) ? i - 1 : i;
    int64_t rank = 0;
    for (int64_t j = 0; j < n; ++j) {
      const double kj = d.key[j];
      const int64_t gj = (d.flag[j] == 2) ? j - 1 : j;
      // ahead of i: larger key; equal key and an earlier group; same pair and Im > 0
      rank += (kj > ki || (kj == ki && (gj < gi || (gj == gi && d.flag[j] == 1 && d.flag[i] == 2)))) ? 1 : 0;
    }
    d.perm[rank] = (int)i;
  }
  __syncthreads();
  for (int64_t p = tid; p < n; p += blockDim.x) {
    const int64_t i = d.perm[p];
    mu_out[2 * p] = d.mur[i];
    mu_out[2 * p + 1] = d.mui[i];
    b_out[2 * p] = qr[i];
    b_out[2 * p + 1] = qi[i];
  }
}

// B[:, p] = T1 w_i / mu_i for the sorted position p (i = perm[p]); the
// second member of a pair stores the imaginary part of the first's.
__global__ void dmd_pack_kernel(DmdState d, const WsHeader* hdr) {
  const int64_t n = dmd_rank(hdr);
  if (read_status(hdr) != 0) return;
  const int64_t M = d.M, ld = d.rmax;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx % M, p = idx / M;
    int64_t i = d.perm[p];
    bool imag = false;
    if (i >= 0 && i < n && d.flag[i] == 2) {
      i = (p > 0) ? d.perm[p - 1] : -1;
      imag = true;
    }
    if (i < 0 || i >= n) {   // not reached for a valid order; keeps every index in range
      d.Bp[row + p * M] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    double cr = 0.0, ci = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double t = d.T1[row + k * M];
      cr = fma(t, d.Wr[k + i * ld], cr);
      ci = fma(t, d.Wi[k + i * ld], ci);
    }
    const cx c = cdiv(cx{cr, ci}, cx{d.mur[i], d.mui[i]});
    d.Bp[row + p * M] = imag ? c.im : c.re;
  }
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

size_t dmd_bytes(int64_t N, int64_t M, int64_t P, int64_t r_max) {
  return sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, true) + svd_state_bytes(M - 1) +
         dmd_small_bytes(M, r_max);
}

}  // namespace
}  // namespace pylom

using namespace pylom;

extern "C" size_t pylom_dmd_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max, int xtype) {
  if (M < 2 || !tall_shape_ok(N, M, leaf_rows) || r_max < 1 || r_max > M - 1) return 0;
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) return 0;
  return dmd_bytes(N, M, leaves_of(N, M, leaf_rows, PYLOM_PREC_FP64), r_max);
}

extern "C" pylom_status pylom_dmd(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype, int remove_mean,
                                  double energy, int64_t r_max, int64_t leaf_rows, double* mu, double* b,
                                  double* Phi, int64_t ldphi, double* S, double* mean, int64_t* r_out, void* ws,
                                  size_t ws_bytes, void* stream) {
  set_error_message("");
  if (!X || !mu || !b || !Phi || !S || !r_out || !ws) {
    set_error_message("pylom_dmd: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) {
    set_error_message("pylom_dmd: xtype must be PYLOM_F32 or PYLOM_F64");
    return PYLOM_ERR_ARG;
  }
  if (M < 2 || leaf_rows < 0 || !tall_shape_ok(N, M, leaf_rows) || r_max < 1 || r_max > M - 1) {
    set_error_message("pylom_dmd: bad shape (N=%lld M=%lld b=%lld r_max=%lld; need 2 <= M <= 4096, N >= M, "
                      "1 <= r_max <= M-1)",
                      (long long)N, (long long)M, (long long)leaf_rows, (long long)r_max);
    return PYLOM_ERR_SHAPE;
  }
  if (ldx < N || ldphi < N) {
    set_error_message("pylom_dmd: leading dimension too small");
    return PYLOM_ERR_ARG;
  }
  const int64_t P = leaves_of(N, M, leaf_rows, PYLOM_PREC_FP64);
  const size_t need = dmd_bytes(N, M, P, r_max);
  if (((uintptr_t)ws & 255) != 0 || ws_bytes < need) {
    set_error_message("pylom_dmd: workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  if (!device_readable(X, "pylom_dmd", "X", &X)) return PYLOM_ERR_ARG;
  const int64_t M1 = M - 1;
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  WsHeader* hdr = (WsHeader*)base;
  TsqrState ts;
  ts.hdr = hdr;
  tsqr_state_carve(ts, base + sizeof(WsHeader), N, M, P, r_max, true);
  char* p2 = base + sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, true);
  SvdState ss;
  ss.hdr = hdr;
  svd_state_carve(ss, p2, M1);
  DmdState d;
  dmd_small_carve(d, p2 + svd_state_bytes(M1), M, r_max);

  // eigensolver residency: H (and Z) in shared memory when they fit
  const size_t hbytes = sizeof(double) * (size_t)(r_max | 1) * r_max;
  const size_t svbytes = sizeof(double) * (size_t)r_max;
  int smem_mode = 0;
  if (2 * hbytes <= kEigSmemCap) smem_mode = 2;
  else if (hbytes <= kEigSmemCap) smem_mode = 1;
  const size_t eig_smem = svbytes + (smem_mode == 2 ? 2 * hbytes : smem_mode == 1 ? hbytes : 0);
  cudaError_t e = ensure_dyn_smem((const void*)dmd_eig_kernel, kEigSmemCap + sizeof(double) * 4096);
  if (e != cudaSuccess) {
    set_error_message("pylom_dmd: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  auto fail = [&](const char* what) {
    set_error_message("pylom_dmd: %s: %s", what, cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  };
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st)) != cudaSuccess) return fail("header clear");
  if ((e = cudaMemsetAsync(ts.arrive, 0, sizeof(unsigned) * (size_t)P, st)) != cudaSuccess)
    return fail("counter clear");
  // Y = D - mean (over all M snapshots) = Q R
  if ((e = launch_tsqr_fp64(ts, X, ldx, xtype, nullptr, remove_mean, mean, st)) != cudaSuccess)
    return fail("leaf QR / tree");
  // SVD of Y1 = Q[:, :M-1] R[:M-1, :M-1]; truncation by energy and r_max
  if ((e = launch_svd_fp64(ss, ts.Rs, M, d.UR, M1, S, d.VT, M1, 60, energy, r_max, st)) != cudaSuccess)
    return fail("small SVD");
  dmd_rank_kernel<<<1, 32, 0, st>>>(hdr, S, N, M1);
  dmd_t1_kernel<<<grid_for(M * r_max, kSmallThreads), kSmallThreads, 0, st>>>(d, ts.Rs, S, hdr);
  dmd_a_kernel<<<grid_for(r_max * r_max, kSmallThreads), kSmallThreads, 0, st>>>(d, hdr);
  dmd_eig_kernel<<<1, kEigThreads, eig_smem, st>>>(d, hdr, smem_mode);
  dmd_w_kernel<<<grid_for(r_max * r_max, kSmallThreads), kSmallThreads, 0, st>>>(d, hdr);
  dmd_wnorm_kernel<<<(unsigned)r_max, kSmallThreads, 0, st>>>(d, hdr);
  dmd_p_kernel<<<grid_for(r_max * r_max, kSmallThreads), kSmallThreads, 0, st>>>(d, hdr);
  dmd_q_kernel<<<(unsigned)r_max, kSmallThreads, 0, st>>>(d, S, hdr);
  dmd_amp_kernel<<<1, kSmallThreads, 0, st>>>(d, hdr, mu, b);
  dmd_pack_kernel<<<grid_for(M * r_max, kSmallThreads), kSmallThreads, 0, st>>>(d, hdr);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("small DMD kernels");
  // phi = Q [B; 0]: the POD's top-down pass and leaf modes product, r read on the device
  if ((e = launch_modes_fp64(ts, d.Bp, M, -1, nullptr, 0, Phi, ldphi, r_out, st)) != cudaSuccess)
    return fail("modes");
  return PYLOM_OK;
}

// svd_batched.cu -- batched complex SVDs of many tall matrices in one
// persistent launch: the per-frequency SVDs of SPOD (pyLOM, arXiv
// 2405.15529, Sec. 2.3 and Alg. 6: (1/sqrt(nBlks)) Q_f = U_f S_f V_f^H for
// every frequency bin f).  Each bin goes through the same route as the POD:
// a TSQR of its rows (complex Householder leaves, last-arriver binary tree,
// Alg. 1), a one-sided Jacobi SVD of its small R (Eq. svdqr2) and the modes
// U = Q U_r (Eq. svdqr3).
//
// One cooperative persistent launch runs all bins.  Blocks take
//   phase A items (bin, leaf) from a queue ordered by cost: leaf QR, then
//     the tree climb; the block that completes a bin's root runs that bin's
//     Jacobi SVD and publishes the bin's modes items to a ready list;
//   phase D items from the ready list (bounded wait for publication): the
//     leaf's block of U, by walking the tree from the root to the leaf and
//     applying the leaf's reflectors.
// No block waits on a block that waits, so progress is guaranteed while all
// blocks are resident (cooperative launch); every wait is time-bounded.
//
// Precision: the leaf working copy is complex64 (TC = float, the "mixed"
// path: FP32 storage and updates, compensated FP32 sums reduced in FP64) or
// complex128 (TC = double); tree, Jacobi and all reflector scalars are FP64.
#include <type_traits>

#include "kernels.h"

namespace pylom {

// ---------------------------------------------------------------------------
// complex helpers (FP64 arithmetic on double2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 warp_csum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// complex arithmetic in the working precision TC (inner loops)
template <typename TC> struct TCx { TC x, y; };
template <typename TC> __device__ __forceinline__ TCx<TC> tc_of(double2 a) { return {(TC)a.x, (TC)a.y}; }
// conj(a) * b
template <typename TC> __device__ __forceinline__ TCx<TC> tc_mulc(TCx<TC> a, TCx<TC> b) {
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename TC> __device__ __forceinline__ TCx<TC> tc_mul(TCx<TC> a, TCx<TC> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename TC> __device__ __forceinline__ TCx<TC> tc_sub(TCx<TC> a, TCx<TC> b) {
  return {a.x - b.x, a.y - b.y};
}

template <typename TC> struct CT;
template <> struct CT<float> {
  using V = float2;
  __device__ static double2 ld(const float2* p) { const float2 v = *p; return make_double2(v.x, v.y); }
  __device__ static void st(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }
  __device__ static TCx<float> ldt(const float2* p) { const float2 v = *p; return {v.x, v.y}; }
  __device__ static void stt(float2* p, TCx<float> v) { *p = make_float2(v.x, v.y); }
};
template <> struct CT<double> {
  using V = double2;
  __device__ static double2 ld(const double2* p) { return *p; }
  __device__ static void st(double2* p, double2 v) { *p = v; }
  __device__ static TCx<double> ldt(const double2* p) { const double2 v = *p; return {v.x, v.y}; }
  __device__ static void stt(double2* p, TCx<double> v) { *p = make_double2(v.x, v.y); }
};

// Compensated (Kahan) running sum of complex terms computed in TC precision;
// for TC = double the compensation is exact bookkeeping of the same sum.
template <typename TC>
struct KSum {
  TC sx = 0, sy = 0, cx = 0, cy = 0;
  __device__ __forceinline__ void add(TC x, TC y) {
    TC yx = x - cx, tx = sx + yx;
    cx = (tx - sx) - yx;
    sx = tx;
    TC yy = y - cy, ty = sy + yy;
    cy = (ty - sy) - yy;
    sy = ty;
  }
  __device__ __forceinline__ double2 get() const {
    return make_double2((double)sx - (double)cx, (double)sy - (double)cy);
  }
};

// Warp total of a compensated complex sum times a complex FP64 factor, in
// the working precision.  TC = float: the lanes combine their (sum,
// compensation) pairs by TwoSum in FP32 and lane 0 alone forms factor *
// total in FP64 and broadcasts it (FP64 arithmetic runs at a small fraction
// of the FP32 rate on this part, so per-lane FP64 reductions dominated the
// complex64 leaves).  TC = double: the plain FP64 reduction.
__device__ __forceinline__ void two_sum_f(float& s, float& c, float os, float oc) {
  const float t = s + os;
  const float bb = t - s;
  const float e = (s - (t - bb)) + (os - bb);
  s = t;
  c = c + oc + e;
}
template <typename TC>
__device__ __forceinline__ TCx<TC> warp_ksum_scaled(const KSum<TC>& k, double2 factor);
template <>
__device__ __forceinline__ TCx<float> warp_ksum_scaled<float>(const KSum<float>& k, double2 factor) {
  float sx = k.sx, cx = -k.cx, sy = k.sy, cy = -k.cy;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float osx = __shfl_xor_sync(0xffffffffu, sx, o), ocx = __shfl_xor_sync(0xffffffffu, cx, o);
    const float osy = __shfl_xor_sync(0xffffffffu, sy, o), ocy = __shfl_xor_sync(0xffffffffu, cy, o);
    two_sum_f(sx, cx, osx, ocx);
    two_sum_f(sy, cy, osy, ocy);
  }
  float fx = 0.f, fy = 0.f;
  if ((threadIdx.x & 31) == 0) {
    const double2 f = cmul(factor, make_double2((double)sx + (double)cx, (double)sy + (double)cy));
    fx = (float)f.x;
    fy = (float)f.y;
  }
  return {__shfl_sync(0xffffffffu, fx, 0), __shfl_sync(0xffffffffu, fy, 0)};
}
template <>
__device__ __forceinline__ TCx<double> warp_ksum_scaled<double>(const KSum<double>& k, double2 factor) {
  const double2 f = cmul(factor, warp_csum(k.get()));
  return {f.x, f.y};
}

// Warp total of the real part of a compensated sum as (sum, compensation),
// valid in lane 0.
template <typename TC>
__device__ __forceinline__ double2 warp_ksum_pair(const KSum<TC>& k) {
  if constexpr (sizeof(TC) == 4) {
    float s = (float)k.sx, c = -(float)k.cx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
      two_sum_f(s, c, os, oc);
    }
    double2 r = make_double2(0.0, 0.0);
    if ((threadIdx.x & 31) == 0) r = make_double2((double)s, (double)c);
    return r;
  } else {
    double v = (double)k.sx - (double)k.cx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return make_double2(v, 0.0);
  }
}

// Block total of the real part of a compensated sum, valid in thread 0
// (scratch: one double2 per warp).
template <typename TC>
__device__ __forceinline__ double block_real_sum0(const KSum<TC>& k, double2* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (sizeof(TC) == 4) {
    float s = (float)k.sx, c = -(float)k.cx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
      two_sum_f(s, c, os, oc);
    }
    __syncthreads();
    if (lane == 0) scratch[warp] = make_double2((double)s, (double)c);
  } else {
    double v = (double)k.sx - (double)k.cx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) scratch[warp] = make_double2(v, 0.0);
  }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nwarps; ++w) t += scratch[w].x + scratch[w].y;
  return t;
}

// ---------------------------------------------------------------------------
// per-bin description and workspace tables (built by the host plan)
// ---------------------------------------------------------------------------
struct BinDesc {
  const float2* X;   // input, N x Nb complex64, ld ldx (kind 0)
  int64_t ldx;
  // kind 0: a complex64 matrix (a SPOD frequency bin); kind 1 / 2: a real
  // float32 / float64 snapshot window (N points x Nb snapshots) whose POD is
  // taken: temporal mean removal and sqrt(w) weights in the leaf load,
  // real modes and right vectors out
  int kind, remove_mean, physical, pad_;
  const void* Xr;    // real input (kinds 1, 2), ld ldx
  const double* w;   // N cell volumes or null (kinds 1, 2)
  double* mean;      // N means out or null (kinds 1, 2)
  void* Ureal;       // N x k real modes, element TC (kinds 1, 2), ld ldu
  double* VT;        // Nb x Nb right vectors out (row i = v_i^T) or null (kinds 1, 2)
  int64_t ldvt;
  int64_t N, Nb, P, k;
  int64_t y_off;     // working copy (TC complex elements), N x Nb, ld N
  int64_t tau_off;   // double2: P x Nb leaf tau
  int64_t rs_off;    // double2: P x Nb x Nb R slots
  int64_t taut_off;  // double2: P x Nb tree tau
  int64_t arr_off;   // unsigned: P arrival counters
  int64_t jac_off;   // double2: 2 x Np x Np, Np = Nb rounded up to even (Jacobi A = R^H, V)
  int64_t ur_off;    // double2: Nb x Nb left vectors of R (sorted, phased)
  int64_t rf_off;    // float2: P x Nb x Nb complex64 copies of the node reflectors (complex64 leaves only)
  int64_t s_off;     // S output offset
  float2* U;         // output modes, N x k complex64
  int64_t ldu;
};

struct BatchCounters {
  unsigned a_next, d_next, d_tail, pad[61];
};

struct BatchArgs {
  WsHeader* hdr;
  BatchCounters* cnt;
  const BinDesc* bins;
  const int2* itemsA;   // (bin, leaf), cost-ordered
  int nA;
  int3* ready;          // (bin, leaf, valid), nD slots
  int nD;
  void* ybase;          // TC complex working copies
  double2* zbase;       // FP64 complex tables
  float2* fbase;        // complex64 copies of the node reflectors (complex64 leaves only)
  unsigned* ubase;      // counters
  double* S;            // packed singular values
  double2* scratch;     // per block: 2 x kMaxNb x kMaxK
  int max_sweeps;
};

constexpr int kBThreads = 256;
constexpr int kMaxNb = 128;
constexpr int kMaxK = 32;
// Leaves hold at most 32 rows per lane (complex64) or 16 (complex128), so a
// warp keeps a whole leaf column in registers between its dot product with
// the current reflector and its update.
constexpr int64_t kLeafMaxRowsF = 1024;
constexpr int64_t kLeafMaxRowsD = 512;
template <typename TC> struct LeafCap;
template <> struct LeafCap<float> { static constexpr int EL = 32; };
template <> struct LeafCap<double> { static constexpr int EL = 16; };

__device__ __forceinline__ int64_t bin_leaf_begin(const BinDesc& b, int64_t leaf) {
  return (leaf * b.N) / b.P;
}

// sum of one double2 per warp lane group into smem slot q (nwarps x K scratch)
__device__ __forceinline__ double2 block_csum(double2 v, double2* sred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  v = warp_csum(v);
  __syncthreads();
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < nwarps; ++w) s = cadd(s, sred[w]);
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// phase A: leaf complex Householder QR, then the bin's tree
// ---------------------------------------------------------------------------
template <typename TC>
__device__ void leaf_qr_complex(const BatchArgs& a, const BinDesc& b, int64_t leaf, double2* sd,
                                double2* sred, typename CT<TC>::V* sv) {
  using V = typename CT<TC>::V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int64_t r0 = bin_leaf_begin(b, leaf), h = bin_leaf_begin(b, leaf + 1) - r0;
  const int64_t Nb = b.Nb, ldy = b.N;
  V* Y = (V*)a.ybase + b.y_off + r0;
  double2* tau = a.zbase + b.tau_off + leaf * Nb;
  // load the leaf (complex64 input -> TC working copy); flag non-finite input
  int bad = 0;
  if (b.kind == 0) {
    for (int64_t j = 0; j < Nb; ++j)
      for (int64_t i = tid; i < h; i += nthr) {
        const float2 x = b.X[r0 + i + j * b.ldx];
        if (!isfinite(x.x) || !isfinite(x.y)) bad = 1;
        CT<TC>::st(Y + i + j * ldy, make_double2(x.x, x.y));
      }
  } else {
    // a real snapshot window (Alg. 2 on each window): per point, its mean
    // over the window's snapshots (binary64) and sqrt of its cell volume;
    // the working copy holds sqrt(w) (x - mean) with a zero imaginary part
    const float* Xf = (const float*)b.Xr;
    const double* Xd = (const double*)b.Xr;
    for (int64_t i = tid; i < h; i += nthr) {
      const int64_t n = r0 + i;
      double xbar = 0.0;
      if (b.remove_mean) {
        double sum = 0.0;
        for (int64_t j = 0; j < Nb; ++j) sum += (b.kind == 1) ? (double)Xf[n + j * b.ldx] : Xd[n + j * b.ldx];
        xbar = sum / (double)Nb;
      }
      if (b.mean) b.mean[n] = xbar;
      double sw = 1.0;
      if (b.w) {
        const double wn = b.w[n];
        if (!(wn > 0.0) || !isfinite(wn)) bad = 1;
        sw = sqrt(wn);
      }
      for (int64_t j = 0; j < Nb; ++j) {
        const double x = (b.kind == 1) ? (double)Xf[n + j * b.ldx] : Xd[n + j * b.ldx];
        if (!isfinite(x)) bad = 1;
        CT<TC>::st(Y + i + j * ldy, make_double2(sw * (x - xbar), 0.0));
      }
    }
  }
  if (bad) raise_status(a.hdr, PYLOM_ERR_NONFINITE);
  __syncthreads();
  // sd[3]: squared norm below the diagonal of the next column, left there by
  // the warp that updated that column (x = sum + compensation); sd[4].x = 1
  // when it is valid
  if (tid == 0) sd[4] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int64_t j = 0; j < Nb; ++j) {
    double xx0 = 0.0;
    // every thread reads the flag before thread 0 resets it below, so the
    // branch (which holds block barriers) is taken by all threads alike
    const bool have_norm = sd[4].x != 0.0;
    __syncthreads();
    if (!have_norm) {
      // squared norm below the diagonal of column j, by a block pass
      KSum<TC> ks;
      for (int64_t i = j + 1 + tid; i < h; i += nthr) {
        const TCx<TC> y = CT<TC>::ldt(Y + i + j * ldy);
        ks.add(y.x * y.x + y.y * y.y, (TC)0);
      }
      xx0 = block_real_sum0<TC>(ks, sred);
    } else if (tid == 0) {
      xx0 = sd[3].x + sd[3].y;
    }
    // thread 0 forms the reflector's scalars and broadcasts them
    if (tid == 0) {
      sd[4] = make_double2(0.0, 0.0);
      const double2 alpha = CT<TC>::ld(Y + j + j * ldy);
      double2 t0 = make_double2(0.0, 0.0), scale0 = make_double2(0.0, 0.0);
      double beta0 = alpha.x;
      if (!(xx0 == 0.0 && alpha.y == 0.0)) {
        const double nrm = sqrt(cabs2(alpha) + xx0);
        beta0 = (alpha.x >= 0.0) ? -nrm : nrm;
        t0 = make_double2((beta0 - alpha.x) / beta0, -alpha.y / beta0);
        scale0 = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta0, alpha.y));
      }
      sd[0] = t0;
      sd[1] = scale0;
      sd[2] = make_double2(beta0, 0.0);
    }
    __syncthreads();
    const double2 t = sd[0], scale = sd[1];
    const double beta = sd[2].x;
    const TCx<TC> sc = tc_of<TC>(scale);
    // scaled reflector v_j (one on the diagonal) into the leaf and the stage
    for (int64_t i = j + tid; i < h; i += nthr) {
      TCx<TC> v = {(TC)1, (TC)0};
      if (i > j) {
        v = tc_mul(CT<TC>::ldt(Y + i + j * ldy), sc);
        CT<TC>::stt(Y + i + j * ldy, v);
      }
      CT<TC>::stt(sv + i, v);
    }
    __syncthreads();
    if (tid == 0) {
      CT<TC>::st(Y + j + j * ldy, make_double2(beta, 0.0));
      tau[j] = t;
    }
    if (j + 1 < Nb && (t.x != 0.0 || t.y != 0.0)) {
      // a warp per column c > j, held in registers: d_c = v_j^H y_c, then
      // y_c -= conj(tau) d_c v_j
      constexpr int EL = LeafCap<TC>::EL;
      for (int64_t c = j + 1 + warp; c < Nb; c += nwarps) {
        V* yc = Y + c * ldy;
        TCx<TC> x[EL];
        KSum<TC> kd;
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const int64_t i = j + lane + 32 * e;
          x[e] = (i < h) ? CT<TC>::ldt(yc + i) : TCx<TC>{(TC)0, (TC)0};
        }
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const int64_t i = j + lane + 32 * e;
          if (i < h) {
            const TCx<TC> p = tc_mulc(CT<TC>::ldt(sv + i), x[e]);
            kd.add(p.x, p.y);
          }
        }
        const TCx<TC> f = warp_ksum_scaled<TC>(kd, cconj(t));
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const int64_t i = j + lane + 32 * e;
          if (i < h) CT<TC>::stt(yc + i, tc_sub(x[e], tc_mul(f, CT<TC>::ldt(sv + i))));
        }
        if (c == j + 1) {
          // the next column's squared norm below its diagonal, re-read by the
          // lanes that just wrote it
          __syncwarp();
          KSum<TC> kn;
          for (int64_t i = j + lane; i < h; i += 32) {   // the rows this lane stored
            if (i <= j + 1) continue;
            const TCx<TC> y = CT<TC>::ldt(yc + i);
            kn.add(y.x * y.x + y.y * y.y, (TC)0);
          }
          const double2 nn = warp_ksum_pair<TC>(kn);
          if (lane == 0) {
            sd[3] = nn;
            sd[4] = make_double2(1.0, 0.0);
          }
        }
      }
    }
    __syncthreads();
  }
  // leaf R (FP64) into the slot
  double2* Rl = a.zbase + b.rs_off + leaf * Nb * Nb;
  for (int64_t idx = tid; idx < Nb * Nb; idx += nthr) {
    const int64_t i = idx % Nb, c = idx / Nb;
    Rl[idx] = (i <= c) ? CT<TC>::ld(Y + i + c * ldy) : make_double2(0.0, 0.0);
  }
}

// QR of [Rt; Rb] (two upper-triangular Nb x Nb, FP64 complex): reflector c
// is [e_c; u_c] with u_c in column c of Rb (rows 0..c), H_c = I - t_c v v^H;
// H_c^H is applied to the trailing columns.  Blocked by panels of kMP
// columns: within a panel one reflector at a time (a warp per later panel
// column); the trailing columns then take the panel's block reflector
// Q = I - V T V^H (T by the forward recurrence) as W = V^H C, W' = T^H W,
// C -= V W' with one thread per entry, so the dot products need no
// cross-lane reductions (FP64 runs at a small fraction of the FP32 rate on
// this part).  sm: shared scratch of kMergeSmem double2.
constexpr int kMP = 8;
constexpr int kMergeSmem = kMaxNb * kMP + kMP * kMaxNb + kMP * kMP;
__device__ void tree_merge_complex(double2* Rt, double2* Rb, double2* tau, int64_t Nb, double2* sd,
                                   float2* Rbf, double2* sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5, nthr = blockDim.x;
  double2* sU = sm;                       // [i][p]: u of the panel's reflector p, rows 0..Nb-1
  double2* sW = sU + kMaxNb * kMP;        // [p][column]
  double2* sT = sW + kMP * kMaxNb;        // [q][p], upper
  for (int64_t k = 0; k < Nb; k += kMP) {
    const int nbk = (int)((Nb - k) < kMP ? (Nb - k) : kMP);
    for (int idx = tid; idx < kMaxNb * kMP; idx += nthr) sU[idx] = make_double2(0.0, 0.0);
    for (int idx = tid; idx < kMP * kMP; idx += nthr) sT[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int jj = 0; jj < nbk; ++jj) {
      const int64_t c = k + jj;
      if (warp == 0) {
        double xx = 0.0;
        for (int64_t i = lane; i <= c; i += 32) xx += cabs2(__ldcg(Rb + i + c * Nb));
        xx = warp_sum(xx);
        if (lane == 0) {
          const double2 alpha = __ldcg(Rt + c + c * Nb);
          double2 t = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
          double beta = alpha.x;
          if (!(xx == 0.0 && alpha.y == 0.0)) {
            const double nrm = sqrt(cabs2(alpha) + xx);
            beta = (alpha.x >= 0.0) ? -nrm : nrm;
            t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
            scale = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta, alpha.y));
          }
          sd[0] = t;
          sd[1] = scale;
          Rt[c + c * Nb] = make_double2(beta, 0.0);
          tau[c] = t;
          sT[jj * kMP + jj] = t;
        }
      }
      __syncthreads();
      const double2 t = sd[0], scale = sd[1];
      for (int64_t i = tid; i <= c; i += nthr) {
        const double2 u = cmul(__ldcg(Rb + i + c * Nb), scale);
        Rb[i + c * Nb] = u;
        sU[i * kMP + jj] = u;
      }
      __syncthreads();
      if (t.x != 0.0 || t.y != 0.0) {
        // the later columns of this panel, one reflector at a time
        for (int64_t cc = c + 1 + warp; cc < k + nbk; cc += nwarps) {
          double2 s = make_double2(0.0, 0.0);
          for (int64_t i = lane; i <= c; i += 32) s = cadd(s, cmulc(sU[i * kMP + jj], __ldcg(Rb + i + cc * Nb)));
          s = cadd(warp_csum(s), __ldcg(Rt + c + cc * Nb));
          const double2 f = cmul(cconj(t), s);
          for (int64_t i = lane; i <= c; i += 32)
            Rb[i + cc * Nb] = csub(__ldcg(Rb + i + cc * Nb), cmul(f, sU[i * kMP + jj]));
          __syncwarp();
          if (lane == 0) Rt[c + cc * Nb] = csub(__ldcg(Rt + c + cc * Nb), f);
        }
      }
      __syncthreads();
    }
    const int64_t c1 = k + nbk;   // first trailing column
    if (c1 >= Nb) break;
    // T[0:j, j] = -t_j T[0:j, 0:j] (V^H v_j)[0:j]; v_q^H v_j = u_q^H u_j (the
    // e parts are disjoint); a warp per pair (q, j), then warp 0 forms T
    for (int pr = warp; pr < nbk * nbk; pr += nwarps) {
      const int q = pr % nbk, j = pr / nbk;
      if (q >= j) continue;
      double2 s = make_double2(0.0, 0.0);
      for (int64_t i = lane; i <= k + q; i += 32) s = cadd(s, cmulc(sU[i * kMP + q], sU[i * kMP + j]));
      s = warp_csum(s);
      if (lane == 0) sW[q * kMaxNb + j] = s;   // staging (sW is free until the trailing update)
    }
    __syncthreads();
    if (tid == 0) {
      for (int j = 1; j < nbk; ++j) {
        const double2 tj = sT[j * kMP + j];
        for (int p = 0; p < j; ++p) {
          double2 acc = make_double2(0.0, 0.0);
          for (int q = p; q < j; ++q) acc = cadd(acc, cmul(sT[p * kMP + q], sW[q * kMaxNb + j]));
          sT[p * kMP + j] = cmul(make_double2(-tj.x, -tj.y), acc);
        }
      }
    }
    __syncthreads();
    // W[p][cc] = Rt[k+p][cc] + sum_{i <= k+p} conj(u_p[i]) Rb[i][cc]
    const int64_t ncols = Nb - c1;
    for (int64_t idx = tid; idx < nbk * ncols; idx += nthr) {
      const int p = (int)(idx % nbk);
      const int64_t cc = c1 + idx / nbk;
      double2 s = __ldcg(Rt + (k + p) + cc * Nb);
      for (int64_t i = 0; i <= k + p; ++i) s = cadd(s, cmulc(sU[i * kMP + p], __ldcg(Rb + i + cc * Nb)));
      sW[p * kMaxNb + (cc - c1)] = s;
    }
    __syncthreads();
    // W' = T^H W, in place column by column (row p needs rows q <= p)
    for (int64_t cc = tid; cc < ncols; cc += nthr) {
      double2 w[kMP];
#pragma unroll
      for (int q = 0; q < kMP; ++q) w[q] = (q < nbk) ? sW[q * kMaxNb + cc] : make_double2(0.0, 0.0);
#pragma unroll
      for (int p = 0; p < kMP; ++p) {
        if (p >= nbk) break;
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q <= p; ++q) acc = cadd(acc, cmul(cconj(sT[q * kMP + p]), w[q]));
        sW[p * kMaxNb + cc] = acc;
      }
    }
    __syncthreads();
    // C -= V W': top rows k..k+nbk-1 of Rt, rows 0..k+nbk-1 of Rb
    for (int64_t idx = tid; idx < nbk * ncols; idx += nthr) {
      const int p = (int)(idx % nbk);
      const int64_t cc = c1 + idx / nbk;
      double2* rt = Rt + (k + p) + cc * Nb;
      *rt = csub(__ldcg(rt), sW[p * kMaxNb + (cc - c1)]);
    }
    for (int64_t idx = tid; idx < c1 * ncols; idx += nthr) {
      const int64_t i = idx % c1, cc = c1 + idx / c1;
      double2 acc = make_double2(0.0, 0.0);
      for (int p = 0; p < nbk; ++p) acc = cadd(acc, cmul(sU[i * kMP + p], sW[p * kMaxNb + (cc - c1)]));
      double2* rb = Rb + i + cc * Nb;
      *rb = csub(__ldcg(rb), acc);
    }
    __syncthreads();
  }
  // complex64 copy of the node reflectors (rows 0..c of column c) for the
  // leaves' single-precision walk down the tree
  if (Rbf) {
    for (int64_t idx = threadIdx.x; idx < Nb * Nb; idx += blockDim.x) {
      const int64_t i = idx % Nb, c = idx / Nb;
      if (i <= c) {
        const double2 v = __ldcg(Rb + idx);
        Rbf[idx] = make_float2((float)v.x, (float)v.y);
      }
    }
  }
}

// One-block complex Jacobi SVD of the bin's R (Nb x Nb, FP64), rotating the
// columns of R^H: R^H J = A, so J holds R's left vectors and the normalised
// columns of A its right vectors.  Round-robin pairs, a warp per pair.
// Then sort, the phase rule (largest |v| entry real and positive), S and the
// sorted left vectors UR.
__device__ void bin_jacobi(const BatchArgs& a, const BinDesc& b, double2* sd, int* si) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t Nb = b.Nb, Np = Nb + (Nb & 1);
  const double2* R = a.zbase + b.rs_off;   // root slot (leaf 0)
  double2* A = a.zbase + b.jac_off;        // Nb x Np
  double2* Vm = A + Nb * Np;               // Np x Np
  double2* UR = a.zbase + b.ur_off;        // Nb x Nb
  for (int64_t idx = tid; idx < Nb * Np; idx += blockDim.x) {
    const int64_t i = idx % Nb, j = idx / Nb;
    // A = R^H: A(i, j) = conj(R(j, i)); R is upper triangular; column Nb pads odd Nb
    A[idx] = (j < Nb && j <= i) ? cconj(__ldcg(R + j + i * Nb)) : make_double2(0.0, 0.0);
  }
  for (int64_t idx = tid; idx < Np * Np; idx += blockDim.x)
    Vm[idx] = (idx % Np == idx / Np) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
  __syncthreads();
  const double tol = (double)Nb * 1.1102230246251565e-16;
  int sweep = 0;
  bool converged = false;
  while (sweep < a.max_sweeps) {
    if (tid == 0) si[0] = 0;
    __syncthreads();
    for (int64_t step = 0; step < Np - 1; ++step) {
      for (int64_t pr = warp; pr < Np / 2; pr += nwarps) {
        const int64_t p = (pr == 0) ? 0 : ((pr - 1 + step) % (Np - 1)) + 1;
        const int64_t q = ((Np - 2 - pr + step) % (Np - 1)) + 1;
        const int64_t i = p < q ? p : q, j = p < q ? q : p;
        double al = 0.0, be = 0.0;
        double2 ga = make_double2(0.0, 0.0);
        for (int64_t r = lane; r < Nb; r += 32) {
          const double2 x = A[r + i * Nb], y = A[r + j * Nb];
          al += cabs2(x);
          be += cabs2(y);
          ga = cadd(ga, cmulc(x, y));
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_csum(ga);
        // every lane holds the same sums; lane 0 alone forms the rotation
        // (FP64 square roots and divisions are slow on this part)
        int rot = 0;
        double c = 0.0, s = 0.0;
        double2 eph = make_double2(0.0, 0.0);   // e^{-i phi}
        if (lane == 0) {
          const double g = sqrt(cabs2(ga));
          if (g != 0.0 && g > tol * sqrt(al * be)) {
            eph = cscale(cconj(ga), 1.0 / g);
            const double zeta = (be - al) / (2.0 * g);
            const double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = c * t;
            rot = 1;
          }
        }
        rot = __shfl_sync(0xffffffffu, rot, 0);
        if (rot) {
          c = __shfl_sync(0xffffffffu, c, 0);
          s = __shfl_sync(0xffffffffu, s, 0);
          eph.x = __shfl_sync(0xffffffffu, eph.x, 0);
          eph.y = __shfl_sync(0xffffffffu, eph.y, 0);
          for (int64_t r = lane; r < Nb; r += 32) {
            const double2 x = A[r + i * Nb], y = cmul(eph, A[r + j * Nb]);
            A[r + i * Nb] = csub(cscale(x, c), cscale(y, s));
            A[r + j * Nb] = cadd(cscale(x, s), cscale(y, c));
          }
          for (int64_t r = lane; r < Np; r += 32) {
            const double2 x = Vm[r + i * Np], y = cmul(eph, Vm[r + j * Np]);
            Vm[r + i * Np] = csub(cscale(x, c), cscale(y, s));
            Vm[r + j * Np] = cadd(cscale(x, s), cscale(y, c));
          }
          if (lane == 0) atomicAdd(si, 1);
        }
      }
      __syncthreads();
    }
    ++sweep;
    const int rot = si[0];
    __syncthreads();
    if (rot == 0) { converged = true; break; }
  }
  if (!converged) raise_status(a.hdr, PYLOM_ERR_NOCONV);
  // singular values, ranks (NaN last), phase, outputs
  double* sig = (double*)(sd + 8);        // Nb doubles
  int* perm = si + 4;                     // Nb ints
  for (int64_t j = warp; j < Nb; j += nwarps) {
    double s2 = 0.0;
    for (int64_t r = lane; r < Nb; r += 32) s2 += cabs2(A[r + j * Nb]);
    s2 = warp_sum(s2);
    if (lane == 0) sig[j] = sqrt(s2);
  }
  __syncthreads();
  for (int64_t j = tid; j < Nb; j += blockDim.x) {
    const double sj = (sig[j] == sig[j]) ? sig[j] : -1.0;
    int rank = 0;
    for (int64_t q = 0; q < Nb; ++q) {
      const double sq = (sig[q] == sig[q]) ? sig[q] : -1.0;
      rank += (sq > sj) || (sq == sj && q < j);
    }
    perm[rank] = (int)j;
  }
  __syncthreads();
  for (int64_t c = warp; c < Nb; c += nwarps) {
    const int64_t j = perm[c];
    // right vector a_j / sigma_j: phase from its largest-magnitude entry
    double best = -1.0;
    int64_t kb = 0;
    for (int64_t r = lane; r < Nb; r += 32) {
      const double m2 = cabs2(A[r + j * Nb]);
      if (m2 > best) { best = m2; kb = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t ok = __shfl_xor_sync(0xffffffffu, kb, o);
      if (ob > best || (ob == best && ok < kb)) { best = ob; kb = ok; }
    }
    const double2 vk = A[kb + j * Nb];
    const double mag = sqrt(cabs2(vk));
    const double2 ph = (mag > 0.0) ? cscale(cconj(vk), 1.0 / mag) : make_double2(1.0, 0.0);
    for (int64_t r = lane; r < Nb; r += 32) UR[r + c * Nb] = cmul(Vm[r + j * Np], ph);
    if (lane == 0) a.S[b.s_off + c] = sig[j];
    if (b.kind != 0 && b.VT) {
      // real window: v_c = a_j ph / sigma_j is real (its largest entry is
      // real and positive); rows of exactly zero sigma are left zero
      const double inv = (sig[j] > 0.0) ? 1.0 / sig[j] : 0.0;
      for (int64_t r = lane; r < Nb; r += 32) b.VT[c + r * b.ldvt] = cmul(A[r + j * Nb], ph).x * inv;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase D: modes of one leaf
// ---------------------------------------------------------------------------
template <typename TC>
__device__ void leaf_modes_complex(const BatchArgs& a, const BinDesc& b, int64_t leaf, double2* scratch,
                                   typename CT<TC>::V* sv) {
  using V = typename CT<TC>::V;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t Nb = b.Nb, k = b.k, P = b.P;
  const double2* UR = a.zbase + b.ur_off;
  int64_t top = 1;
  while (top * 2 < P) top *= 2;
  int64_t node = 0;
  // B at the leaf (Nb x k, complex TC): the first k columns of U_R pushed
  // down the tree from the root to this leaf
  using TB = typename std::conditional<sizeof(TC) == 4, float2, double2>::type;
  TB* Bt = (TB*)scratch;
  TB* Bb = Bt + kMaxNb * kMaxK;
  for (int64_t idx = tid; idx < Nb * k; idx += blockDim.x) {
    const double2 v = UR[(idx % Nb) + (idx / Nb) * Nb];
    if constexpr (sizeof(TC) == 4) Bt[idx] = make_float2((float)v.x, (float)v.y);
    else Bt[idx] = v;
  }
  __syncthreads();
  for (int64_t step = (P > 1 ? top : 0); step >= 1; step >>= 1) {
    const int64_t right = node + step;
    if (right >= P) continue;
    const bool go_right = leaf >= right;
    const double2* tau = a.zbase + b.taut_off + right * Nb;
    for (int64_t idx = tid; idx < Nb * k; idx += blockDim.x) {
      if constexpr (sizeof(TC) == 4) Bb[idx] = make_float2(0.f, 0.f);
      else Bb[idx] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int64_t col = warp; col < k; col += nwarps) {
      TB* bt = Bt + col * Nb;
      TB* bb = Bb + col * Nb;
      for (int64_t c = Nb - 1; c >= 0; --c) {
        const double2 t = tau[c];
        if (t.x == 0.0 && t.y == 0.0) continue;
        if constexpr (sizeof(TC) == 4) {
          // single precision with compensated sums; lane 0 forms
          // t (u_c^H b + b_c) in FP64 and broadcasts it
          const float2* Uf = a.fbase + b.rf_off + right * Nb * Nb + c * Nb;
          KSum<float> ks;
          for (int64_t i = lane; i <= c; i += 32) {
            const float2 u = Uf[i], x = bb[i];
            ks.add(u.x * x.x + u.y * x.y, u.x * x.y - u.y * x.x);
          }
          const float2 btc = bt[c];
          ks.add(lane == 0 ? btc.x : 0.f, lane == 0 ? btc.y : 0.f);
          const TCx<float> f = warp_ksum_scaled<float>(ks, t);
          __syncwarp();
          if (lane == 0) bt[c] = make_float2(btc.x - f.x, btc.y - f.y);
          for (int64_t i = lane; i <= c; i += 32) {
            const float2 u = Uf[i], x = bb[i];
            bb[i] = make_float2(x.x - (f.x * u.x - f.y * u.y), x.y - (f.x * u.y + f.y * u.x));
          }
        } else {
          const double2* Uu = a.zbase + b.rs_off + right * Nb * Nb;
          double2 s = make_double2(0.0, 0.0);
          for (int64_t i = lane; i <= c; i += 32) s = cadd(s, cmulc(Uu[i + c * Nb], bb[i]));
          s = cadd(warp_csum(s), bt[c]);
          const double2 f = cmul(t, s);
          __syncwarp();
          if (lane == 0) bt[c] = csub(bt[c], f);
          for (int64_t i = lane; i <= c; i += 32) bb[i] = csub(bb[i], cmul(f, Uu[i + c * Nb]));
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (go_right) {
      for (int64_t idx = tid; idx < Nb * k; idx += blockDim.x) Bt[idx] = Bb[idx];
      node = right;
    }
    __syncthreads();
  }
  // U_leaf = Q_leaf [B; 0]: reflectors in reverse order; a warp per mode
  // column, held in registers; each reflector staged once in shared memory
  const int64_t r0 = bin_leaf_begin(b, leaf), h = bin_leaf_begin(b, leaf + 1) - r0;
  const V* Y = (const V*)a.ybase + b.y_off + r0;
  const double2* tl = a.zbase + b.tau_off + leaf * Nb;
  float2* Uo = b.U + r0;
  constexpr int EL = LeafCap<TC>::EL;
  for (int64_t c0 = 0; c0 < k; c0 += nwarps) {
    const int64_t col = c0 + warp;
    const bool live = col < k;
    TCx<TC> x[EL];
#pragma unroll
    for (int e = 0; e < EL; ++e) {
      const int64_t i = lane + 32 * e;
      TB v{};
      if (live && i < Nb) v = Bt[i + col * Nb];
      x[e] = {(TC)v.x, (TC)v.y};
    }
    for (int64_t j = Nb - 1; j >= 0; --j) {
      const double2 t = tl[j];
      if (t.x == 0.0 && t.y == 0.0) continue;   // uniform across the block
      __syncthreads();
      for (int64_t i = j + tid; i < h; i += blockDim.x)
        CT<TC>::stt(sv + i, (i == j) ? TCx<TC>{(TC)1, (TC)0} : CT<TC>::ldt(Y + i + j * b.N));
      __syncthreads();
      KSum<TC> ks;
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int64_t i = lane + 32 * e;
        if (i >= j && i < h) {
          const TCx<TC> p = tc_mulc(CT<TC>::ldt(sv + i), x[e]);
          ks.add(p.x, p.y);
        }
      }
      const TCx<TC> f = warp_ksum_scaled<TC>(ks, t);
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int64_t i = lane + 32 * e;
        if (i >= j && i < h) x[e] = tc_sub(x[e], tc_mul(f, CT<TC>::ldt(sv + i)));
      }
    }
    if (live && b.kind == 0) {
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int64_t i = lane + 32 * e;
        if (i < h) Uo[i + col * b.ldu] = make_float2((float)x[e].x, (float)x[e].y);
      }
    } else if (live) {
      // real window: the mode is the real part (its imaginary part is
      // rounding only), divided by sqrt(w) for physical modes
      TC* Ur = (TC*)b.Ureal + r0;
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int64_t i = lane + 32 * e;
        if (i < h) {
          TC v = x[e].x;
          if (b.physical && b.w) v = (TC)((double)v / sqrt(b.w[r0 + i]));
          Ur[i + col * b.ldu] = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename TC>
__global__ void __launch_bounds__(kBThreads, 2) svd_batched_kernel(BatchArgs a) {
  __shared__ double2 sd[8 + kMaxNb / 2 + 4];
  __shared__ double2 sred[kBThreads / 32];
  __shared__ int si[4 + kMaxNb];
  __shared__ int s_item, s_prev;
  // the current reflector of a leaf (at most 1024 complex64 or 512 complex128 rows)
  __shared__ __align__(16) unsigned char svraw[8192];
  __shared__ double2 smerge[kMergeSmem];
  using V = typename CT<TC>::V;
  V* sv = (V*)svraw;
  static_assert(kLeafMaxRowsF * 8 <= 8192 && kLeafMaxRowsD * 16 <= 8192, "reflector stage too small");
  const int tid = threadIdx.x;
  double2* scratch = a.scratch + (int64_t)blockIdx.x * 2 * kMaxNb * kMaxK;
  // phase A
  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(&a.cnt->a_next, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.nA) break;
    if (read_status(a.hdr) == PYLOM_ERR_TIMEOUT) return;
    const int f = a.itemsA[item].x;
    const int64_t leaf = a.itemsA[item].y;
    const BinDesc b = a.bins[f];
    leaf_qr_complex<TC>(a, b, leaf, sd, sred, sv);
    __threadfence();
    __syncthreads();
    int64_t node = leaf;
    bool root = true;
    unsigned* arr = a.ubase + b.arr_off;
    for (int64_t step = 1; step < b.P; step <<= 1) {
      int64_t left, right;
      if (node & step) { left = node - step; right = node; }
      else {
        right = node + step;
        if (right >= b.P) continue;
        left = node;
      }
      if (tid == 0) s_prev = (int)atomicAdd(&arr[right], 1u);
      __syncthreads();
      const int prev = s_prev;
      __syncthreads();
      if (prev == 0) { root = false; break; }
      __threadfence();
      tree_merge_complex(a.zbase + b.rs_off + left * b.Nb * b.Nb, a.zbase + b.rs_off + right * b.Nb * b.Nb,
                         a.zbase + b.taut_off + right * b.Nb, b.Nb, sd,
                         sizeof(TC) == 4 ? a.fbase + b.rf_off + right * b.Nb * b.Nb : nullptr, smerge);
      __threadfence();
      __syncthreads();
      node = left;
    }
    if (!root) continue;
    // this block completed the bin's root: SVD of R, then publish modes items
    bin_jacobi(a, b, sd, si);
    __threadfence();
    __syncthreads();
    if (b.k > 0) {
      if (tid == 0) s_prev = (int)atomicAdd(&a.cnt->d_tail, (unsigned)b.P);
      __syncthreads();
      const int pos = s_prev;
      for (int64_t l = tid; l < b.P; l += blockDim.x) {
        a.ready[pos + l].x = f;
        a.ready[pos + l].y = (int)l;
      }
      __threadfence();
      __syncthreads();
      for (int64_t l = tid; l < b.P; l += blockDim.x) atomicExch(&a.ready[pos + l].z, 1);
      __syncthreads();
    }
  }
  // phase D
  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(&a.cnt->d_next, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.nD) break;
    if (tid == 0) {
      const unsigned long long t0 = global_ns();
      int ok = 1;
      while (atomicAdd(&a.ready[item].z, 0) == 0) {
        if (global_ns() - t0 > kWaitLimitNs || read_status(a.hdr) == PYLOM_ERR_TIMEOUT) {
          raise_status(a.hdr, PYLOM_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
      s_prev = ok;
    }
    __syncthreads();
    if (!s_prev) return;
    __threadfence();
    const int f = __ldcg(&a.ready[item].x);
    const int64_t leaf = __ldcg(&a.ready[item].y);
    const BinDesc b = a.bins[f];
    leaf_modes_complex<TC>(a, b, leaf, scratch, sv);
    __syncthreads();
  }
}

}  // namespace pylom

// ---------------------------------------------------------------------------
// host side: plan, bind, run
// ---------------------------------------------------------------------------
#include <algorithm>
#include <cstring>
#include <vector>

struct pylom_batched_plan {
  int nbins = 0, prec = 0;
  int64_t kmodes = 0;
  std::vector<int64_t> N, Nb, P, h;
  std::vector<pylom::BinDesc> bins;   // offsets filled by the plan, pointers by bind
  std::vector<int2> itemsA;
  int nA = 0, nD = 0;
  size_t off_f = 0;   // complex64 node-reflector copies
  size_t off_cnt = 0, off_bins = 0, off_items = 0, off_ready = 0, off_u = 0, off_z = 0, off_y = 0,
         off_scr = 0, bytes = 0;
  int64_t total_u = 0, total_z = 0, total_y = 0, total_s = 0;
  int grid = 0;
  bool bound = false;
};

namespace pylom {

constexpr int64_t kBatchedMaxNb = kMaxNb;
constexpr int64_t kBatchedMaxK = kMaxK;

// Longest leaf a bin may have: a warp holds a leaf column in registers.
int64_t batched_max_leaf_rows(int prec) { return prec == PYLOM_PREC_FP64 ? kLeafMaxRowsD : kLeafMaxRowsF; }

int64_t batched_default_leaf_rows(int64_t N, int64_t Nb, int prec) {
  int64_t h = batched_max_leaf_rows(prec);
  if (h < Nb) h = Nb;
  if (h > N) h = N;
  return h;
}

template <typename TC>
static cudaError_t batched_grid(int* grid) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, svd_batched_kernel<TC>, kBThreads, 0);
  if (e != cudaSuccess) return e;
  *grid = nsm * (per > 0 ? per : 1);
  return cudaSuccess;
}

}  // namespace pylom

using namespace pylom;

extern "C" pylom_status pylom_svd_batched_plan(int nbins, const int64_t* N, const int64_t* Nb,
                                               const int64_t* leaf_rows, int64_t kmodes, int prec,
                                               pylom_batched_plan** plan_out, size_t* ws_bytes) {
  set_error_message("");
  if (!N || !Nb || !plan_out || !ws_bytes || nbins < 1) {
    set_error_message("pylom_svd_batched_plan: null pointer or nbins < 1");
    return PYLOM_ERR_ARG;
  }
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) {
    set_error_message("pylom_svd_batched_plan: bad prec %d", prec);
    return PYLOM_ERR_ARG;
  }
  if (kmodes < 0 || kmodes > kBatchedMaxK) {
    set_error_message("pylom_svd_batched_plan: kmodes must be in [0, %lld]", (long long)kBatchedMaxK);
    return PYLOM_ERR_SHAPE;
  }
  auto* p = new pylom_batched_plan();
  p->nbins = nbins;
  p->prec = prec;
  p->kmodes = kmodes;
  const size_t ye = (prec == PYLOM_PREC_FP64) ? 16 : 8;
  int64_t y = 0, z = 0, u = 0, sacc = 0, fz = 0;
  for (int f = 0; f < nbins; ++f) {
    const int64_t n = N[f], nb = Nb[f];
    if (nb < 1 || nb > kBatchedMaxNb || n < nb) {
      set_error_message("pylom_svd_batched_plan: bin %d has N = %lld, Nb = %lld (need 1 <= Nb <= %lld, N >= Nb)",
                        f, (long long)n, (long long)nb, (long long)kBatchedMaxNb);
      delete p;
      return PYLOM_ERR_SHAPE;
    }
    int64_t h = (leaf_rows && leaf_rows[f] > 0) ? leaf_rows[f] : batched_default_leaf_rows(n, nb, prec);
    if (h < nb) {
      set_error_message("pylom_svd_batched_plan: bin %d leaf height %lld < Nb", f, (long long)h);
      delete p;
      return PYLOM_ERR_SHAPE;
    }
    int64_t P = n / h;
    // no leaf longer than the register-resident limit (with the floor
    // partition the longest leaf has ceil(n / P) rows; the shortest keeps
    // >= Nb rows because the limit is at least 2 Nb)
    const int64_t hmax = batched_max_leaf_rows(prec);
    if (P < (n + hmax - 1) / hmax) P = (n + hmax - 1) / hmax;
    if (P < 1) P = 1;
    const int64_t np = nb + (nb & 1);
    BinDesc b{};
    b.N = n; b.Nb = nb; b.P = P; b.k = kmodes < nb ? kmodes : nb;
    b.y_off = y;                 y += n * nb;
    b.tau_off = z;               z += P * nb;
    b.rs_off = z;                z += P * nb * nb;
    b.taut_off = z;              z += P * nb;
    b.jac_off = z;               z += 2 * np * np;
    b.ur_off = z;                z += nb * nb;
    b.rf_off = fz;               fz += (prec == PYLOM_PREC_FP64) ? 0 : P * nb * nb;
    b.arr_off = u;               u += P;
    b.s_off = sacc;              sacc += nb;
    p->N.push_back(n); p->Nb.push_back(nb); p->P.push_back(P); p->h.push_back(h);
    p->bins.push_back(b);
    for (int64_t l = 0; l < P; ++l) p->itemsA.push_back(make_int2(f, (int)l));
    if (b.k > 0) p->nD += (int)P;
  }
  // cost order: leaves of the widest bins first (their roots need the longest Jacobi)
  std::stable_sort(p->itemsA.begin(), p->itemsA.end(), [&](const int2& x, const int2& yv) {
    const int64_t cx = p->Nb[x.x] * p->Nb[x.x] * (p->N[x.x] / p->P[x.x]);
    const int64_t cy = p->Nb[yv.x] * p->Nb[yv.x] * (p->N[yv.x] / p->P[yv.x]);
    if (p->Nb[x.x] != p->Nb[yv.x]) return p->Nb[x.x] > p->Nb[yv.x];
    return cx > cy;
  });
  p->nA = (int)p->itemsA.size();
  p->total_y = y; p->total_z = z; p->total_u = u; p->total_s = sacc;
  cudaError_t e = (prec == PYLOM_PREC_FP64) ? batched_grid<double>(&p->grid) : batched_grid<float>(&p->grid);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_batched_plan: %s", cudaGetErrorString(e));
    delete p;
    return PYLOM_ERR_CUDA;
  }
  size_t off = sizeof(WsHeader);
  p->off_cnt = off;   off += align256(sizeof(BatchCounters));
  p->off_bins = off;  off += align256(sizeof(BinDesc) * (size_t)nbins);
  p->off_items = off; off += align256(sizeof(int2) * (size_t)p->nA);
  p->off_ready = off; off += align256(sizeof(int3) * (size_t)(p->nD > 0 ? p->nD : 1));
  p->off_u = off;     off += align256(sizeof(unsigned) * (size_t)u);
  p->off_z = off;     off += align256(sizeof(double2) * (size_t)z);
  p->off_f = off;     off += align256(sizeof(float2) * (size_t)(fz > 0 ? fz : 1));
  p->off_y = off;     off += align256(ye * (size_t)y);
  p->off_scr = off;   off += align256(sizeof(double2) * (size_t)p->grid * 2 * kMaxNb * kMaxK);
  p->bytes = off;
  *plan_out = p;
  *ws_bytes = off;
  return PYLOM_OK;
}

extern "C" void pylom_svd_batched_plan_destroy(pylom_batched_plan* plan) { delete plan; }

extern "C" int64_t pylom_svd_batched_max_leaf_rows(int prec) {
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) return -1;
  return batched_max_leaf_rows(prec);
}

extern "C" int64_t pylom_svd_batched_plan_info(const pylom_batched_plan* plan, int bin, int what) {
  if (!plan || bin < 0 || bin >= plan->nbins) return -1;
  switch (what) {
    case 0: return plan->h[bin];
    case 1: return plan->P[bin];
    case 2: return plan->bins[bin].s_off;
    case 3: return plan->grid;
    case 4: return plan->nA;
    default: return -1;
  }
}

static pylom_status batched_upload_tables(pylom_batched_plan* plan, void* ws, void* stream, const char* who);

extern "C" pylom_status pylom_svd_batched_bind(pylom_batched_plan* plan, const void* const* Q, const int64_t* ldq,
                                               void* const* U, const int64_t* ldu, void* ws, size_t ws_bytes,
                                               void* stream) {
  set_error_message("");
  if (!plan || !Q || !ldq || !ws) {
    set_error_message("pylom_svd_batched_bind: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (((uintptr_t)ws & 255u) != 0 || ws_bytes < plan->bytes) {
    set_error_message("pylom_svd_batched_bind: workspace needs %zu bytes, 256-byte aligned", plan->bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  for (int f = 0; f < plan->nbins; ++f) {
    BinDesc& b = plan->bins[f];
    if (!Q[f] || ldq[f] < b.N) {
      set_error_message("pylom_svd_batched_bind: bin %d input pointer or leading dimension invalid", f);
      return PYLOM_ERR_ARG;
    }
    b.kind = 0;
    b.Xr = nullptr;
    b.w = nullptr;
    b.mean = nullptr;
    b.Ureal = nullptr;
    b.VT = nullptr;
    b.X = (const float2*)Q[f];
    b.ldx = ldq[f];
    if (b.k > 0) {
      if (!U || !U[f] || !ldu || ldu[f] < b.N) {
        set_error_message("pylom_svd_batched_bind: bin %d output pointer or leading dimension invalid", f);
        return PYLOM_ERR_ARG;
      }
      b.U = (float2*)U[f];
      b.ldu = ldu[f];
    } else {
      b.U = nullptr;
      b.ldu = b.N;
    }
  }
  return batched_upload_tables(plan, ws, stream, "pylom_svd_batched_bind");
}

extern "C" pylom_status pylom_svd_batched_bind_items(pylom_batched_plan* plan, const pylom_batched_item* items,
                                                     void* ws, size_t ws_bytes, void* stream) {
  set_error_message("");
  if (!plan || !items || !ws) {
    set_error_message("pylom_svd_batched_bind_items: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (((uintptr_t)ws & 255u) != 0 || ws_bytes < plan->bytes) {
    set_error_message("pylom_svd_batched_bind_items: workspace needs %zu bytes, 256-byte aligned", plan->bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  for (int f = 0; f < plan->nbins; ++f) {
    BinDesc& b = plan->bins[f];
    const pylom_batched_item& it = items[f];
    if (it.xtype != PYLOM_C64 && it.xtype != PYLOM_F32 && it.xtype != PYLOM_F64) {
      set_error_message("pylom_svd_batched_bind_items: item %d: xtype must be PYLOM_C64, PYLOM_F32 or PYLOM_F64", f);
      return PYLOM_ERR_ARG;
    }
    if (!it.X || it.ldx < b.N) {
      set_error_message("pylom_svd_batched_bind_items: item %d input pointer or leading dimension invalid", f);
      return PYLOM_ERR_ARG;
    }
    if (b.k > 0 && (!it.U || it.ldu < b.N)) {
      set_error_message("pylom_svd_batched_bind_items: item %d output pointer or leading dimension invalid", f);
      return PYLOM_ERR_ARG;
    }
    const bool real = it.xtype != PYLOM_C64;
    if (real && it.mode_kind != PYLOM_MODES_ORTHONORMAL && it.mode_kind != PYLOM_MODES_PHYSICAL) {
      set_error_message("pylom_svd_batched_bind_items: item %d: bad mode_kind %d", f, it.mode_kind);
      return PYLOM_ERR_ARG;
    }
    if (real && it.VT && it.ldvt < b.Nb) {
      set_error_message("pylom_svd_batched_bind_items: item %d: ldvt < Nb", f);
      return PYLOM_ERR_ARG;
    }
    b.kind = real ? (it.xtype == PYLOM_F32 ? 1 : 2) : 0;
    b.ldx = it.ldx;
    b.X = real ? nullptr : (const float2*)it.X;
    b.Xr = real ? it.X : nullptr;
    b.remove_mean = real ? (it.remove_mean != 0) : 0;
    b.physical = real ? (it.mode_kind == PYLOM_MODES_PHYSICAL) : 0;
    b.w = real ? it.w : nullptr;
    b.mean = real ? it.mean : nullptr;
    b.VT = real ? it.VT : nullptr;
    b.ldvt = real ? it.ldvt : 0;
    b.U = (b.k > 0 && !real) ? (float2*)it.U : nullptr;
    b.Ureal = (b.k > 0 && real) ? it.U : nullptr;
    b.ldu = b.k > 0 ? it.ldu : b.N;
  }
  return batched_upload_tables(plan, ws, stream, "pylom_svd_batched_bind_items");
}

static pylom_status batched_upload_tables(pylom_batched_plan* plan, void* ws, void* stream, const char* who) {
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  cudaError_t e = cudaMemcpyAsync(base + plan->off_bins, plan->bins.data(), sizeof(BinDesc) * plan->bins.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + plan->off_items, plan->itemsA.data(), sizeof(int2) * plan->itemsA.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error_message("%s: %s", who, cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  plan->bound = true;
  return PYLOM_OK;
}

extern "C" pylom_status pylom_svd_batched_run(const pylom_batched_plan* plan, void* ws, double* S,
                                              int max_sweeps, void* stream) {
  set_error_message("");
  if (!plan || !ws || !S || !plan->bound) {
    set_error_message("pylom_svd_batched_run: plan not bound, or null pointer");
    return PYLOM_ERR_ARG;
  }
  if (max_sweeps < 1 || max_sweeps > kMaxSweeps) {
    set_error_message("pylom_svd_batched_run: max_sweeps must be in [1, %d]", kMaxSweeps);
    return PYLOM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  cudaError_t e = cudaMemsetAsync(base, 0, plan->off_bins, st);   // header + counters
  if (e == cudaSuccess)
    e = cudaMemsetAsync(base + plan->off_ready, 0, sizeof(int3) * (size_t)(plan->nD > 0 ? plan->nD : 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + plan->off_u, 0, sizeof(unsigned) * (size_t)plan->total_u, st);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_batched_run: clear: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  BatchArgs a;
  a.hdr = (WsHeader*)base;
  a.cnt = (BatchCounters*)(base + plan->off_cnt);
  a.bins = (const BinDesc*)(base + plan->off_bins);
  a.itemsA = (const int2*)(base + plan->off_items);
  a.nA = plan->nA;
  a.ready = (int3*)(base + plan->off_ready);
  a.nD = plan->nD;
  a.ybase = base + plan->off_y;
  a.zbase = (double2*)(base + plan->off_z);
  a.fbase = (float2*)(base + plan->off_f);
  a.ubase = (unsigned*)(base + plan->off_u);
  a.S = S;
  a.scratch = (double2*)(base + plan->off_scr);
  a.max_sweeps = max_sweeps;
  void* args[] = {(void*)&a};
  if (plan->prec == PYLOM_PREC_FP64)
    e = cudaLaunchCooperativeKernel((const void*)svd_batched_kernel<double>, dim3(plan->grid), dim3(kBThreads),
                                    args, 0, st);
  else
    e = cudaLaunchCooperativeKernel((const void*)svd_batched_kernel<float>, dim3(plan->grid), dim3(kBThreads),
                                    args, 0, st);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_batched_run: launch: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

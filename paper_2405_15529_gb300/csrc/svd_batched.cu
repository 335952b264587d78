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

// ---------------------------------------------------------------------------
// per-bin description and workspace tables (built by the host plan)
// ---------------------------------------------------------------------------
struct BinDesc {
  const float2* X;   // input, N x Nb complex64, ld ldx
  int64_t ldx;
  int64_t N, Nb, P, k;
  int64_t y_off;     // working copy (TC complex elements), N x Nb, ld N
  int64_t tau_off;   // double2: P x Nb leaf tau
  int64_t rs_off;    // double2: P x Nb x Nb R slots
  int64_t taut_off;  // double2: P x Nb tree tau
  int64_t arr_off;   // unsigned: P arrival counters
  int64_t jac_off;   // double2: 2 x Np x Np, Np = Nb rounded up to even (Jacobi A = R^H, V)
  int64_t ur_off;    // double2: Nb x Nb left vectors of R (sorted, phased)
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
  unsigned* ubase;      // counters
  double* S;            // packed singular values
  double2* scratch;     // per block: 2 x kMaxNb x kMaxK
  int max_sweeps;
};

constexpr int kBThreads = 256;
constexpr int kMaxNb = 128;
constexpr int kMaxK = 32;

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
                                double2* sred) {
  using V = typename CT<TC>::V;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const int64_t r0 = bin_leaf_begin(b, leaf), h = bin_leaf_begin(b, leaf + 1) - r0;
  const int64_t Nb = b.Nb, ldy = b.N;
  V* Y = (V*)a.ybase + b.y_off + r0;
  double2* tau = a.zbase + b.tau_off + leaf * Nb;
  // load the leaf (complex64 input -> TC working copy); flag non-finite input
  int bad = 0;
  for (int64_t j = 0; j < Nb; ++j)
    for (int64_t i = tid; i < h; i += nthr) {
      const float2 x = b.X[r0 + i + j * b.ldx];
      if (!isfinite(x.x) || !isfinite(x.y)) bad = 1;
      CT<TC>::st(Y + i + j * ldy, make_double2(x.x, x.y));
    }
  if (bad) raise_status(a.hdr, PYLOM_ERR_NONFINITE);
  __syncthreads();
  for (int64_t j = 0; j < Nb; ++j) {
    // squared norm below the diagonal of column j
    KSum<TC> ks;
    for (int64_t i = j + 1 + tid; i < h; i += nthr) {
      const TCx<TC> y = CT<TC>::ldt(Y + i + j * ldy);
      ks.add(y.x * y.x + y.y * y.y, (TC)0);
    }
    const double xx = block_csum(ks.get(), sred).x;
    const double2 alpha = CT<TC>::ld(Y + j + j * ldy);
    double2 t = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
    double beta = alpha.x;
    if (!(xx == 0.0 && alpha.y == 0.0)) {
      const double nrm = sqrt(cabs2(alpha) + xx);
      beta = (alpha.x >= 0.0) ? -nrm : nrm;
      t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
      scale = cdiv(make_double2(1.0, 0.0), make_double2(alpha.x - beta, alpha.y));
    }
    const TCx<TC> sc = tc_of<TC>(scale);
    for (int64_t i = j + 1 + tid; i < h; i += nthr)
      CT<TC>::stt(Y + i + j * ldy, tc_mul(CT<TC>::ldt(Y + i + j * ldy), sc));
    __syncthreads();
    if (tid == 0) {
      CT<TC>::st(Y + j + j * ldy, make_double2(beta, 0.0));
      tau[j] = t;
    }
    if (j + 1 < Nb && (t.x != 0.0 || t.y != 0.0)) {
      // d_c = v_j^H y_c for c > j (a warp per column), then
      // y_c -= conj(tau) d_c v_j
      const TCx<TC> one = {(TC)1, (TC)0};
      for (int64_t c = j + 1 + warp; c < Nb; c += nwarps) {
        KSum<TC> kd;
        for (int64_t i = j + lane; i < h; i += 32) {
          const TCx<TC> v = (i == j) ? one : CT<TC>::ldt(Y + i + j * ldy);
          const TCx<TC> p = tc_mulc(v, CT<TC>::ldt(Y + i + c * ldy));
          kd.add(p.x, p.y);
        }
        const double2 d = warp_csum(kd.get());
        const TCx<TC> f = tc_of<TC>(cmul(cconj(t), d));
        for (int64_t i = j + lane; i < h; i += 32) {
          const TCx<TC> v = (i == j) ? one : CT<TC>::ldt(Y + i + j * ldy);
          CT<TC>::stt(Y + i + c * ldy, tc_sub(CT<TC>::ldt(Y + i + c * ldy), tc_mul(f, v)));
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
  (void)sd;
}

// QR of [Rt; Rb] (two upper-triangular Nb x Nb, FP64 complex): reflector c
// is [e_c; u_c] with u_c in column c of Rb (rows 0..c); H_c^H applied to the
// trailing columns.  A warp per trailing column.
__device__ void tree_merge_complex(double2* Rt, double2* Rb, double2* tau, int64_t Nb, double2* sd) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int64_t c = 0; c < Nb; ++c) {
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
      }
    }
    __syncthreads();
    const double2 t = sd[0], scale = sd[1];
    for (int64_t i = tid; i <= c; i += blockDim.x) Rb[i + c * Nb] = cmul(__ldcg(Rb + i + c * Nb), scale);
    __syncthreads();
    if (t.x != 0.0 || t.y != 0.0) {
      for (int64_t cc = c + 1 + warp; cc < Nb; cc += nwarps) {
        double2 s = make_double2(0.0, 0.0);
        for (int64_t i = lane; i <= c; i += 32) s = cadd(s, cmulc(__ldcg(Rb + i + c * Nb), __ldcg(Rb + i + cc * Nb)));
        s = cadd(warp_csum(s), __ldcg(Rt + c + cc * Nb));
        const double2 f = cmul(cconj(t), s);
        for (int64_t i = lane; i <= c; i += 32)
          Rb[i + cc * Nb] = csub(__ldcg(Rb + i + cc * Nb), cmul(f, __ldcg(Rb + i + c * Nb)));
        __syncwarp();
        if (lane == 0) Rt[c + cc * Nb] = csub(__ldcg(Rt + c + cc * Nb), f);
      }
    }
    __syncthreads();
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
        const double g = sqrt(cabs2(ga));
        if (g != 0.0 && g > tol * sqrt(al * be)) {
          const double2 eph = cscale(cconj(ga), 1.0 / g);   // e^{-i phi}
          const double zeta = (be - al) / (2.0 * g);
          const double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
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
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase D: modes of one leaf
// ---------------------------------------------------------------------------
template <typename TC>
__device__ void leaf_modes_complex(const BatchArgs& a, const BinDesc& b, int64_t leaf, double2* scratch) {
  using V = typename CT<TC>::V;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t Nb = b.Nb, k = b.k, P = b.P;
  double2* Bt = scratch;                 // Nb x k
  double2* Bb = scratch + kMaxNb * kMaxK;
  const double2* UR = a.zbase + b.ur_off;
  for (int64_t idx = tid; idx < Nb * k; idx += blockDim.x) Bt[idx] = UR[(idx % Nb) + (idx / Nb) * Nb];
  __syncthreads();
  // walk the tree from the root to this leaf
  int64_t top = 1;
  while (top * 2 < P) top *= 2;
  int64_t node = 0;
  for (int64_t step = (P > 1 ? top : 0); step >= 1; step >>= 1) {
    const int64_t right = node + step;
    if (right >= P) continue;
    const bool go_right = leaf >= right;
    const double2* Uu = a.zbase + b.rs_off + right * Nb * Nb;
    const double2* tau = a.zbase + b.taut_off + right * Nb;
    for (int64_t idx = tid; idx < Nb * k; idx += blockDim.x) Bb[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int64_t col = warp; col < k; col += nwarps) {
      double2* bt = Bt + col * Nb;
      double2* bb = Bb + col * Nb;
      for (int64_t c = Nb - 1; c >= 0; --c) {
        const double2 t = tau[c];
        if (t.x == 0.0 && t.y == 0.0) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int64_t i = lane; i <= c; i += 32) s = cadd(s, cmulc(Uu[i + c * Nb], bb[i]));
        s = cadd(warp_csum(s), bt[c]);
        const double2 f = cmul(t, s);
        __syncwarp();
        if (lane == 0) bt[c] = csub(bt[c], f);
        for (int64_t i = lane; i <= c; i += 32) bb[i] = csub(bb[i], cmul(f, Uu[i + c * Nb]));
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
  // U_leaf = Q_leaf [B; 0]: reflectors in reverse order, a warp per column
  const int64_t r0 = bin_leaf_begin(b, leaf), h = bin_leaf_begin(b, leaf + 1) - r0;
  const V* Y = (const V*)a.ybase + b.y_off + r0;
  const double2* tl = a.zbase + b.tau_off + leaf * Nb;
  float2* Uo = b.U + r0;
  for (int64_t col = warp; col < k; col += nwarps) {
    for (int64_t i = lane; i < h; i += 32) {
      const double2 v = (i < Nb) ? Bt[i + col * Nb] : make_double2(0.0, 0.0);
      Uo[i + col * b.ldu] = make_float2((float)v.x, (float)v.y);
    }
  }
  __syncthreads();
  for (int64_t col = warp; col < k; col += nwarps) {
    float2* u = Uo + col * b.ldu;
    for (int64_t j = Nb - 1; j >= 0; --j) {
      const double2 t = tl[j];
      if (t.x == 0.0 && t.y == 0.0) continue;
      const TCx<TC> one = {(TC)1, (TC)0};
      KSum<TC> ks;
      for (int64_t i = j + lane; i < h; i += 32) {
        const TCx<TC> v = (i == j) ? one : CT<TC>::ldt(Y + i + j * b.N);
        const float2 x = u[i];
        const TCx<TC> p = tc_mulc(v, TCx<TC>{(TC)x.x, (TC)x.y});
        ks.add(p.x, p.y);
      }
      const double2 d = warp_csum(ks.get());
      const TCx<TC> f = tc_of<TC>(cmul(t, d));
      __syncwarp();
      for (int64_t i = j + lane; i < h; i += 32) {
        const TCx<TC> v = (i == j) ? one : CT<TC>::ldt(Y + i + j * b.N);
        const float2 x = u[i];
        const TCx<TC> nv = tc_sub(TCx<TC>{(TC)x.x, (TC)x.y}, tc_mul(f, v));
        u[i] = make_float2((float)nv.x, (float)nv.y);
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename TC>
__global__ void __launch_bounds__(kBThreads) svd_batched_kernel(BatchArgs a) {
  __shared__ double2 sd[8 + kMaxNb / 2 + 4];
  __shared__ double2 sred[kBThreads / 32];
  __shared__ int si[4 + kMaxNb];
  __shared__ int s_item, s_prev;
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
    leaf_qr_complex<TC>(a, b, leaf, sd, sred);
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
                         a.zbase + b.taut_off + right * b.Nb, b.Nb, sd);
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
    leaf_modes_complex<TC>(a, b, leaf, scratch);
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
  size_t off_cnt = 0, off_bins = 0, off_items = 0, off_ready = 0, off_u = 0, off_z = 0, off_y = 0,
         off_scr = 0, bytes = 0;
  int64_t total_u = 0, total_z = 0, total_y = 0, total_s = 0;
  int grid = 0;
  bool bound = false;
};

namespace pylom {

constexpr int64_t kBatchedMaxNb = kMaxNb;
constexpr int64_t kBatchedMaxK = kMaxK;

int64_t batched_default_leaf_rows(int64_t N, int64_t Nb, int prec) {
  // about 1 MiB of working copy per leaf (L2-friendly with ~300 leaves in flight)
  const int64_t elem = (prec == PYLOM_PREC_FP64) ? 16 : 8;
  int64_t h = (int64_t)(1 << 20) / (Nb * elem);
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
  int64_t y = 0, z = 0, u = 0, sacc = 0;
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
  p->off_y = off;     off += align256(ye * (size_t)y);
  p->off_scr = off;   off += align256(sizeof(double2) * (size_t)p->grid * 2 * kMaxNb * kMaxK);
  p->bytes = off;
  *plan_out = p;
  *ws_bytes = off;
  return PYLOM_OK;
}

extern "C" void pylom_svd_batched_plan_destroy(pylom_batched_plan* plan) { delete plan; }

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
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  cudaError_t e = cudaMemcpyAsync(base + plan->off_bins, plan->bins.data(), sizeof(BinDesc) * plan->bins.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + plan->off_items, plan->itemsA.data(), sizeof(int2) * plan->itemsA.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error_message("pylom_svd_batched_bind: %s", cudaGetErrorString(e));
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

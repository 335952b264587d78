// svd_jacobi.cu -- binary64 SVD of the small M x M factor R (Eq. svdqr2 of
// pyLOM, arXiv 2405.15529): parallel one-sided (Hestenes) Jacobi across
// thread blocks, then sort / sign / cumulative-energy truncation (Sec. 3.1).
//
// The rotations act on the columns of R^T (the rows of R): if R^T J = A has
// orthogonal columns, R = J diag(|a_j|) (A diag(1/|a_j|))^T, so the
// accumulated rotations J are R's left singular vectors and the normalised
// columns of A its right singular vectors.  On the triangular, graded R of a
// QR factorisation this needs about a third of the sweeps that rotating the
// columns of R does (10 vs 27 on the 256-column six-decade workload).
//
// Pairs follow the round-robin ("tournament") ordering: in each of the
// Mp - 1 steps of a sweep the Mp/2 column pairs are disjoint, one pair per
// block, so a step needs no locking; steps are separated by a bounded grid
// barrier of a cooperative launch.  Odd M is padded with one zero column,
// which never rotates.
#include "kernels.h"

namespace pylom {

constexpr int kJacThreads = 256;
constexpr int kFinThreads = 1024;

size_t svd_state_bytes(int64_t M, bool precond) {
  const int64_t Mp = M + (M & 1);
  return align256(sizeof(double) * (size_t)M * Mp) + align256(sizeof(double) * (size_t)Mp * Mp) +
         (precond ? jacobi32_extra_bytes(M) : 0);
}

void svd_state_carve(SvdState& s, char* base, int64_t M, bool precond) {
  s.M = M;
  s.Mp = M + (M & 1);
  s.A = (double*)base;
  s.V = (double*)(base + align256(sizeof(double) * (size_t)M * s.Mp));
  s.Mb = 0;
  s.A32 = s.V32 = nullptr;
  s.G = s.Tm = s.mmws = nullptr;
  s.rot32 = nullptr;
  if (precond && M >= kJac32MinM)
    jacobi32_carve(s, (char*)s.V + align256(sizeof(double) * (size_t)s.Mp * s.Mp));
}

__global__ void jacobi_init_kernel(SvdState s, const double* R, int64_t ldr) {
  const int64_t M = s.M, Mp = s.Mp;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * Mp; idx += stride) {
    const int64_t i = idx % M, j = idx / M;
    s.A[idx] = (j < M) ? R[j + i * ldr] : 0.0;   // A = R^T
  }
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < Mp * Mp; idx += stride)
    s.V[idx] = (idx % Mp == idx / Mp) ? 1.0 : 0.0;
}

// EL = elements of a column per thread (M <= EL * kJacThreads): the pair's
// two columns stay in registers between the dot products and the rotation,
// so each step reads them from L2 once.
template <int EL>
__global__ void __launch_bounds__(kJacThreads) jacobi_kernel(SvdState s, int max_sweeps) {
  __shared__ double sred[3 * (kJacThreads / 32)];
  __shared__ double sout[4];
  const int tid = threadIdx.x;
  constexpr int nthr = kJacThreads;
  const int64_t M = s.M, Mp = s.Mp, npairs = Mp / 2;
  const double tol = (double)M * 1.1102230246251565e-16;  // M * 2^-53
  int sweep = 0;
  bool converged = false;
  while (sweep < max_sweeps) {
    unsigned local_rot = 0;
    for (int64_t step = 0; step < Mp - 1; ++step) {
      for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const int64_t p = (pr == 0) ? 0 : ((pr - 1 + step) % (Mp - 1)) + 1;
        const int64_t q = ((Mp - 2 - pr + step) % (Mp - 1)) + 1;
        const int64_t i = p < q ? p : q, j = p < q ? q : p;
        double* ai = s.A + i * M;
        double* aj = s.A + j * M;
        double x[EL], y[EL];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const int64_t r = tid + (int64_t)e * nthr;
          x[e] = (r < M) ? ldcg(ai + r) : 0.0;
          y[e] = (r < M) ? ldcg(aj + r) : 0.0;
        }
        double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          v[0] += x[e] * x[e];
          v[1] += y[e] * y[e];
          v[2] += x[e] * y[e];
        }
        // block reduction (fixed order); thread 0 alone forms the rotation
        // (FP64 square roots and divisions are slow on this part) and
        // broadcasts it: sout = {c, s, rotate?}
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = warp_sum(v[k]);
        if ((tid & 31) == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) sred[k * (nthr / 32) + (tid >> 5)] = v[k];
        }
        __syncthreads();
        if (tid == 0) {
          double tot[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            double a = 0.0;
            for (int w = 0; w < nthr / 32; ++w) a += sred[k * (nthr / 32) + w];
            tot[k] = a;
          }
          const double alpha = tot[0], beta = tot[1], gamma = tot[2];
          sout[2] = 0.0;
          if (gamma != 0.0 && fabs(gamma) > tol * sqrt(alpha * beta)) {
            const double zeta = (beta - alpha) / (2.0 * gamma);
            const double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            sout[0] = c;
            sout[1] = c * t;
            sout[2] = 1.0;
          }
        }
        __syncthreads();
        if (sout[2] != 0.0) {
          const double c = sout[0], sn = sout[1];
#pragma unroll
          for (int e = 0; e < EL; ++e) {
            const int64_t r = tid + (int64_t)e * nthr;
            if (r < M) {
              ai[r] = c * x[e] - sn * y[e];
              aj[r] = sn * x[e] + c * y[e];
            }
          }
          double* vi = s.V + i * Mp;
          double* vj = s.V + j * Mp;
#pragma unroll
          for (int e = 0; e < EL; ++e) {
            const int64_t r = tid + (int64_t)e * nthr;
            x[e] = (r < Mp) ? ldcg(vi + r) : 0.0;
            y[e] = (r < Mp) ? ldcg(vj + r) : 0.0;
          }
#pragma unroll
          for (int e = 0; e < EL; ++e) {
            const int64_t r = tid + (int64_t)e * nthr;
            if (r < Mp) {
              vi[r] = c * x[e] - sn * y[e];
              vj[r] = sn * x[e] + c * y[e];
            }
          }
          ++local_rot;
        }
      }
      if (!grid_barrier(s.hdr, gridDim.x)) return;
    }
    if (tid == 0 && local_rot) atomicAdd(&s.hdr->rot[sweep], local_rot);
    if (!grid_barrier(s.hdr, gridDim.x)) return;
    const unsigned total = ld_acquire_u32(&s.hdr->rot[sweep]);
    ++sweep;
    if (total == 0) {
      converged = true;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    s.hdr->sweeps = sweep;
    if (!converged) raise_status(s.hdr, PYLOM_ERR_NOCONV);
  }
}

// One block.  sigma_j = |a_j|; sort descending (ties by index); left vectors
// = columns of the rotations J, right vectors = a_j / sigma_j (orthonormal
// completion where sigma_j == 0); sign so the largest |v| entry is positive
// (lowest index on ties); cumulative-energy rank.
__global__ void __launch_bounds__(kFinThreads) svd_finalize_kernel(SvdState s, double* U, int64_t ldu,
                                                                   double* S, double* VT,
                                                                   int64_t ldvt, double energy,
                                                                   int64_t r_max) {
  extern __shared__ double fsm[];
  const int64_t M = s.M, Mp = s.Mp;
  double* sig = fsm;                    // M
  double* sgn = sig + M;                // M (by output column)
  int* perm = (int*)(sgn + M);          // M
  __shared__ double sred[kFinThreads / 32];
  __shared__ double sout[2];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  for (int64_t j = warp; j < M; j += nwarps) {
    double a = 0.0;
    for (int64_t i = lane; i < M; i += 32) {
      const double x = s.A[i + j * M];
      a += x * x;
    }
    a = warp_sum(a);
    if (lane == 0) sig[j] = sqrt(a);
  }
  __syncthreads();
  // NaN (from non-finite input) sorts last as key -1, so ranks stay a
  // permutation and every perm entry is written.
  for (int64_t j = tid; j < M; j += nthr) {
    const double sj = (sig[j] == sig[j]) ? sig[j] : -1.0;
    int rank = 0;
    for (int64_t q = 0; q < M; ++q) {
      const double sq = (sig[q] == sig[q]) ? sig[q] : -1.0;
      rank += (sq > sj) || (sq == sj && q < j);
    }
    perm[rank] = (int)j;
  }
  __syncthreads();
  for (int64_t idx = tid; idx < M * M; idx += nthr) {
    const int64_t i = idx % M, c = idx / M;
    const int64_t j = perm[c];
    const double sj = sig[j];
    U[i + c * ldu] = s.V[i + j * Mp];
    VT[c + i * ldvt] = (sj > 0.0) ? s.A[i + j * M] / sj : 0.0;
  }
  for (int64_t c = tid; c < M; c += nthr) S[c] = sig[perm[c]];
  __syncthreads();
  // orthonormal completion of the right vectors for exactly-zero singular
  // values (sorted last): Gram-Schmidt of unit vectors, twice
  int64_t next_e = 0;
  for (int64_t c = 0; c < M; ++c) {
    if (!(sig[perm[c]] == 0.0)) continue;
    for (; next_e < M; ++next_e) {
      for (int64_t i = tid; i < M; i += nthr) VT[c + i * ldvt] = (i == next_e) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t q = 0; q < c; ++q) {
          double v[1] = {0.0};
          for (int64_t i = tid; i < M; i += nthr) v[0] += VT[q + i * ldvt] * VT[c + i * ldvt];
          block_sum<1>(v, sred, sout);
          const double d = sout[0];
          for (int64_t i = tid; i < M; i += nthr) VT[c + i * ldvt] -= d * VT[q + i * ldvt];
          __syncthreads();
        }
      }
      double v[1] = {0.0};
      for (int64_t i = tid; i < M; i += nthr) v[0] += VT[c + i * ldvt] * VT[c + i * ldvt];
      block_sum<1>(v, sred, sout);
      const double nn = sqrt(sout[0]);
      if (nn > 0.5) {
        for (int64_t i = tid; i < M; i += nthr) VT[c + i * ldvt] /= nn;
        __syncthreads();
        ++next_e;
        break;
      }
    }
  }
  __syncthreads();
  // sign of each pair from its right vector
  for (int64_t c = warp; c < M; c += nwarps) {
    double best = -1.0;
    int64_t kbest = 0;
    for (int64_t k = lane; k < M; k += 32) {
      const double a = fabs(VT[c + k * ldvt]);
      if (a > best) { best = a; kbest = k; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t ok = __shfl_xor_sync(0xffffffffu, kbest, o);
      if (ob > best || (ob == best && ok < kbest)) { best = ob; kbest = ok; }
    }
    if (lane == 0) sgn[c] = (VT[c + kbest * ldvt] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  for (int64_t idx = tid; idx < M * M; idx += nthr) {
    const int64_t i = idx % M, c = idx / M;
    if (sgn[c] < 0.0) {
      U[i + c * ldu] = -U[i + c * ldu];
      VT[c + i * ldvt] = -VT[c + i * ldvt];
    }
  }
  if (tid == 0) {
    int64_t rm = r_max < M ? r_max : M;
    int64_t r = rm;
    if (energy > 0.0) {
      double total = 0.0;
      for (int64_t i = 0; i < M; ++i) total += sig[perm[i]] * sig[perm[i]];
      if (total > 0.0) {
        double acc = 0.0;
        for (int64_t k = 0; k < M; ++k) {
          acc += sig[perm[k]] * sig[perm[k]];
          if (acc / total >= energy) {
            r = (k + 1 < rm) ? k + 1 : rm;
            break;
          }
        }
      }
    }
    s.hdr->r = r;
  }
}

cudaError_t launch_svd_fp64(const SvdState& s, const double* R, int64_t ldr, double* U, int64_t ldu,
                            double* S, double* VT, int64_t ldvt, int max_sweeps, double energy,
                            int64_t r_max, cudaStream_t st) {
  cudaError_t e;
  if (s.A32) {
    e = launch_jacobi32_precondition(s, R, ldr, st);
  } else {
    jacobi_init_kernel<<<64, 256, 0, st>>>(s, R, ldr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // smallest register footprint that holds a column (Mp <= EL * kJacThreads)
  const void* kern;
  if (s.Mp <= 1 * kJacThreads) kern = (const void*)jacobi_kernel<1>;
  else if (s.Mp <= 2 * kJacThreads) kern = (const void*)jacobi_kernel<2>;
  else if (s.Mp <= 4 * kJacThreads) kern = (const void*)jacobi_kernel<4>;
  else if (s.Mp <= 8 * kJacThreads) kern = (const void*)jacobi_kernel<8>;
  else kern = (const void*)jacobi_kernel<16>;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kJacThreads, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = s.Mp / 2;
  const int64_t cap = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  SvdState sa = s;
  int ms = max_sweeps;
  void* args[] = {(void*)&sa, (void*)&ms};
  e = cudaLaunchCooperativeKernel(kern, dim3((unsigned)grid), dim3(kJacThreads),
                                  args, 0, st);
  if (e != cudaSuccess) return e;
  const size_t fsm = sizeof(double) * 2 * (size_t)s.M + sizeof(int) * (size_t)s.M;
  if (fsm > 48 * 1024 && (e = ensure_dyn_smem((const void*)svd_finalize_kernel, fsm)) != cudaSuccess) return e;
  svd_finalize_kernel<<<1, kFinThreads, fsm, st>>>(s, U, ldu, S, VT, ldvt, energy, r_max);
  return cudaGetLastError();
}

}  // namespace pylom

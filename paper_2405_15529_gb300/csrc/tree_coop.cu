// tree_coop.cu -- the binary-tree reduction of the stacked leaf R factors
// (Sec. 3.1, the reduce loop of Alg. 1) with every merge spread over many
// thread blocks.  One merge of two M x M triangles costs (2/3) M^3 FP64
// flops (second term of the paper's cost model); at M in the thousands that
// is seconds for the single block of a last-arriver merge, and the top of
// the tree is a chain of log2(P) such merges.
//
// One cooperative persistent launch walks the levels.  Within a level all
// merges advance panel by panel (kNB columns): the trailing columns of each
// merge are cut into chunks, one block per (merge, chunk) applies the
// panel's block reflector, and the block holding a merge's first chunk --
// exactly the next panel's columns, so that block's update is short -- then
// factors that panel and publishes its T factor (double-buffered), so a
// single bounded grid barrier separates consecutive panels.  The pairing (left child's R on top), the
// merged R in the left slot and the node reflectors in the right slot are
// those of the last-arriver tree, so the top-down pass and the adjoint read
// them unchanged.
#include <atomic>

#include "kernels.h"
#include "reflectors.cuh"

namespace pylom {

// Factor panel [k, k+nbk) of merge j at tree step `step`; publish T to Tt
// when trailing columns remain.
static __device__ void coop_factor(const TsqrState& s, double* Tt, int64_t j, int64_t step, int64_t k, int nbk,
                                   double* sT, double* sred, double* sout, double* sP) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t M = s.M;
  const int64_t left = j * 2 * step, right = left + step;
  for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = 0.0;
  __syncthreads();
  if (merge_panel_staged(M))
    merge_panel_factor_staged(s.Rs + left * M * M, s.Rs + right * M * M, M, k, nbk, s.tau_tree + right * M + k, sT,
                              sP);
  else
    merge_panel_factor(s.Rs + left * M * M, s.Rs + right * M * M, M, k, nbk, s.tau_tree + right * M + k, sT, sred,
                       sout);
  __syncthreads();
  if (k + nbk < M) {
    for (int idx = tid; idx < kSmT; idx += nthr) Tt[idx] = sT[idx];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kLeafThreads, 2) tree_coop_kernel(TsqrState s) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sred = sT + kSmT;
  double* sout = sred + kSmRed;
  double* sW = sout + kSmOut;
  double* sWp = sW + kSmW;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t M = s.M, P = s.P, G = gridDim.x;
  const int64_t half = (P + 1) / 2;   // most merges a level can have
  for (int64_t step = 1; step < P; step <<= 1) {
    const int64_t m = (P - step + 2 * step - 1) / (2 * step);
    {
      const int nbk = (int)(M < kNB ? M : kNB);
      for (int64_t j = blockIdx.x; j < m; j += G) coop_factor(s, s.Tt + j * kSmT, j, step, 0, nbk, sT, sred, sout, sW);
    }
    if (!grid_barrier(s.hdr, (unsigned)G)) return;
    // panel k is full width whenever trailing columns follow it.  Chunk 0
    // of a merge is exactly the next panel's columns: its block updates them
    // and factors that panel at once (the critical path of a grid step),
    // while the other blocks update the remaining columns in chunks.
    for (int64_t k = 0; k + kNB < M; k += kNB) {
      const int64_t c_begin = k + kNB, rem = M - c_begin;
      const int64_t w0 = rem < kNB ? rem : kNB;       // chunk 0: the next panel
      const int64_t rem2 = rem - w0;                   // the rest
      const int64_t per_merge = (G + m - 1) / m;
      const int64_t helpers = per_merge > 1 ? per_merge - 1 : 1;
      int64_t cw = (rem2 + helpers - 1) / helpers;
      cw = (cw + 7) & ~int64_t(7);
      cw = cw < 2 * kNB ? 2 * kNB : (cw > kCW ? kCW : cw);
      const int64_t nch = 1 + (rem2 + cw - 1) / cw;
      const int64_t buf = (k / kNB) & 1;
      for (int64_t item = blockIdx.x; item < m * nch; item += G) {
        const int64_t j = item / nch, ch = item - j * nch;
        const int64_t left = j * 2 * step, right = left + step;
        double* Rt = s.Rs + left * M * M;
        double* Rb = s.Rs + right * M * M;
        const double* Tg = s.Tt + (buf * half + j) * kSmT;
        for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = ldcg(Tg + idx);
        __syncthreads();
        const int64_t c0 = (ch == 0) ? c_begin : c_begin + w0 + (ch - 1) * cw;
        const int64_t cwi = (ch == 0) ? w0 : cw;
        const int wc = (int)((M - c0) < cwi ? (M - c0) : cwi);
        MergeV V{Rb, M, k, kNB};
        block_reflector<true, true>(V, kNB, 0, k + kNB, Rb + c0 * M, M, wc, Rt + k + c0 * M, M, sT, sW, sWp);
        __syncthreads();
        if (ch == 0)
          coop_factor(s, s.Tt + ((buf ^ 1) * half + j) * kSmT, j, step, c_begin, (int)w0, sT, sred, sout, sW);
      }
      if (!grid_barrier(s.hdr, (unsigned)G)) return;
    }
  }
}

cudaError_t launch_tree_coop(const TsqrState& s, cudaStream_t st) {
  if (s.P <= 1) return cudaSuccess;
  // co-resident grid, per device (occupancy after the shared-memory limit is raised)
  // (atomic: calls may come from several host threads)
  static std::atomic<int> grid_of[64];
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = ensure_dyn_smem((const void*)tree_coop_kernel, kLeafSmemBytes)) != cudaSuccess) return e;
  int grid = (dev >= 0 && dev < 64) ? grid_of[dev].load(std::memory_order_relaxed) : 0;
  if (grid == 0) {
    int sms = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_coop_kernel, kLeafThreads, kLeafSmemBytes);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = per * sms;
    if (dev >= 0 && dev < 64) grid_of[dev].store(grid, std::memory_order_relaxed);
  }
  TsqrState a = s;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)tree_coop_kernel, dim3((unsigned)grid), dim3(kLeafThreads), args,
                                     kLeafSmemBytes, st);
}

}  // namespace pylom

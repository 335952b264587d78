// tree_pipe.cu -- the binary-tree reduction of the stacked leaf R factors
// (Sec. 3.1, the reduce loop of Alg. 1) as a dataflow pipeline over column
// blocks, for M below a few hundred columns.
//
// There a merge is small ((2/3) M^3 = 1.1e7 flops at M = 256) and the
// level-by-level schedule of tree_coop_kernel is bound by its critical path:
// log2(P) levels x M / kNB panel steps, each a grid barrier plus one panel
// factorisation.  Column block q of a merged R depends only on column block
// q of its two children, so here the column blocks of a merge are worked
// left-looking by kPipeSub thread blocks in turn: for block q the owner
// waits until both children have published block q, applies the merge's
// panels 0 .. q-1 to it (block reflector on the FP64 tensor pipe), factors
// panel q and publishes the block.  A parent then runs one column block
// behind its children, and the tree costs about one merge plus one block
// step per level instead of levels x merges' panel steps.
//
// Storage is that of the other two trees (left child's R on top, merged R in
// the left slot, node reflectors in the right slot, tau by right child), so
// the top-down pass and the adjoint read it unchanged.  The panel T factors
// of a merge are kept in Tn (indexed by its right child) for its later
// column blocks.  Progress: arrive[right] = column blocks of that merge that
// are final.  Merges are numbered level by level, a merge's kPipeSub units
// consecutively; a block takes units in increasing number and waits only on
// lower-numbered merges or on a sibling unit of its own merge, which the
// grid stride (a multiple of kPipeSub) puts in the same round; the launch is
// cooperative (all blocks resident), so the lowest unfinished unit can
// always proceed.  Every wait is bounded (PYLOM_ERR_TIMEOUT).
#include <atomic>

#include "kernels.h"
#include "reflectors.cuh"

namespace pylom {

static __device__ __forceinline__ int64_t merges_at(int64_t P, int64_t step) {
  return (P - step + 2 * step - 1) / (2 * step);
}

// wait until *flag >= target (acquire); gives up after kWaitLimitNs, or at
// once when another block has recorded a timeout
static __device__ bool wait_at_least(const WsHeader* h, const unsigned* flag, unsigned target) {
  if (!flag) return true;
  const unsigned long long t0 = global_ns();
  unsigned polls = 0;
  while (ld_acquire_u32(flag) < target) {
    if ((++polls & 63u) == 0) {
      if (global_ns() - t0 > kWaitLimitNs) return false;
      if (read_status(h) == PYLOM_ERR_TIMEOUT) return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Blocks per merge: the column blocks of a merge are dealt round-robin to
// kPipeSub thread blocks, so while one factors panel q the next applies the
// earlier panels to block q + 1 and waits only for panel q itself.
constexpr int kPipeSub = 2;

__global__ void __launch_bounds__(kLeafThreads, 2) tree_pipe_kernel(TsqrState s) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sred = sT + kSmT;
  double* sout = sred + kSmRed;
  double* sW = sout + kSmOut;
  double* sWp = sW + kSmW;
  __shared__ int s_ok;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t M = s.M, P = s.P, G = gridDim.x;
  const int64_t nblk = (M + kNB - 1) / kNB;
  int64_t step = 1, base = 0, m = merges_at(P, 1);
  // work unit u = merge u / kPipeSub, column blocks q = u % kPipeSub (mod
  // kPipeSub); G is a multiple of kPipeSub, so the units of one merge run at
  // the same time
  for (int64_t ui = blockIdx.x;; ui += G) {
    const int64_t mi = ui / kPipeSub;
    const int sub = (int)(ui % kPipeSub);
    while (step < P && mi >= base + m) {
      base += m;
      step <<= 1;
      m = step < P ? merges_at(P, step) : 0;
    }
    if (step >= P) break;
    const int64_t j = mi - base, left = j * 2 * step, right = left + step;
    // producers: the top child is merge (step / 2, left); the bottom one is
    // the last merge into slot `right`, or its leaf
    const unsigned* top = step > 1 ? s.arrive + left + step / 2 : nullptr;
    const unsigned* bot = nullptr;
    for (int64_t st = step / 2; st >= 1; st >>= 1)
      if (right % (2 * st) == 0 && right + st < P) {
        bot = s.arrive + right + st;
        break;
      }
    double* Rt = s.Rs + left * M * M;
    double* Rb = s.Rs + right * M * M;
    double* Tm = s.Tn + right * nblk * kSmT;
    const unsigned* own = s.arrive + right;   // panels of this merge factored so far
    for (int64_t q = sub; q < nblk; q += kPipeSub) {
      const int64_t c0 = q * kNB;
      const int wc = (int)((M - c0) < kNB ? (M - c0) : kNB);
      if (tid == 0)
        s_ok = wait_at_least(s.hdr, top, (unsigned)(q + 1)) && wait_at_least(s.hdr, bot, (unsigned)(q + 1));
      __syncthreads();
      if (!s_ok) {
        if (tid == 0) raise_status(s.hdr, PYLOM_ERR_TIMEOUT);
        return;
      }
      // left-looking update of column block q by this merge's panels 0 .. q-1
      // (panel p factored by the unit that owns block p)
      for (int64_t p = 0; p < q; ++p) {
        if (tid == 0) s_ok = wait_at_least(s.hdr, own, (unsigned)(p + 1));
        __syncthreads();
        if (!s_ok) {
          if (tid == 0) raise_status(s.hdr, PYLOM_ERR_TIMEOUT);
          return;
        }
        for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = ldcg(Tm + p * kSmT + idx);
        __syncthreads();
        const int64_t k = p * kNB;
        MergeV V{Rb, M, k, kNB};
        block_reflector<true, true>(V, kNB, 0, k + kNB, Rb + c0 * M, M, wc, Rt + k + c0 * M, M, sT, sW, sWp);
        __syncthreads();
      }
      for (int idx = tid; idx < kSmT; idx += nthr) sT[idx] = 0.0;
      __syncthreads();
      if (merge_panel_staged(M))
        merge_panel_factor_staged(Rt, Rb, M, c0, wc, s.tau_tree + right * M + c0, sT, sW);
      else
        merge_panel_factor(Rt, Rb, M, c0, wc, s.tau_tree + right * M + c0, sT, sred, sout);
      __syncthreads();
      if (q + 1 < nblk)
        for (int idx = tid; idx < kSmT; idx += nthr) Tm[q * kSmT + idx] = sT[idx];
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_u32(s.arrive + right, (unsigned)(q + 1));
      }
    }
  }
}

cudaError_t launch_tree_pipe(const TsqrState& s, cudaStream_t st) {
  if (s.P <= 1) return cudaSuccess;
  // (atomic: calls may come from several host threads)
  static std::atomic<int> per_sm_of[64];
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = ensure_dyn_smem((const void*)tree_pipe_kernel, kLeafSmemBytes)) != cudaSuccess) return e;
  int per = (dev >= 0 && dev < 64) ? per_sm_of[dev].load(std::memory_order_relaxed) : 0;
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tree_pipe_kernel, kLeafThreads, kLeafSmemBytes);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (dev >= 0 && dev < 64) per_sm_of[dev].store(per, std::memory_order_relaxed);
  }
  // the arrival counters double as progress counters (zeroed by the caller
  // before the leaf kernel, which leaves them untouched when the tree runs
  // separately)
  int64_t grid = (int64_t)per * sms;
  if (grid > (s.P - 1) * kPipeSub) grid = (s.P - 1) * kPipeSub;
  grid -= grid % kPipeSub;
  TsqrState a = s;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)tree_pipe_kernel, dim3((unsigned)grid), dim3(kLeafThreads), args,
                                     kLeafSmemBytes, st);
}

}  // namespace pylom

// pod_sharded.cu -- the POD of a snapshot matrix whose rows are split over
// several devices (or several calls on one device): the paper's own parallel
// form (Sec. 3.1, Alg. 1), with the processes' row blocks as shards.
//
//   1. pylom_pod_shard_factor, per shard g: the mean / weight prologue, the
//      leaf QR and the tree of the shard's own leaves (a1-a3), down to the
//      shard's M x M factor R_g.  The reflectors stay in the shard's
//      workspace.
//   2. the caller gathers the G factors R_0 .. R_{G-1} (an all-gather across
//      devices; the G * M^2 doubles are the only data exchanged).
//   3. pylom_pod_rstack, replicated on every shard: the top of the tree over
//      the stacked factors (Alg. 1's XOR pairing with the shards in place of
//      the processes), the SVD of the root R and the truncation (a4-a5), and
//      the top-down pass down to every shard: B_g, the shard's M x r block of
//      Q_top [U_r; 0] (the broadcast loop of Alg. 1, computed redundantly
//      instead of sent).
//   4. pylom_pod_shard_modes, per shard: the top-down pass through the
//      shard's own tree from B_g and the leaf modes (a6-a7).
// The shard's workspace carries everything between steps 1 and 4 and must
// not be touched in between.
#include "kernels.h"
#include "reflectors.cuh"

namespace pylom {
namespace {

// Tree over P leaves whose R factors already sit in the Rs slots: the block
// of leaf i climbs from leaf i (the last-arriver merges of the leaf kernel).
__global__ void __launch_bounds__(kLeafThreads) tree_only_kernel(TsqrState s) {
  extern __shared__ double smem[];
  double* sT = smem;
  double* sred = sT + kSmT;
  double* sout = sred + kSmRed;
  double* sW = sout + kSmOut;
  double* sWp = sW + kSmW;
  tree_climb(s, (int64_t)blockIdx.x, sT, sred, sout, sW, sWp);
}

// Rs slot g := upper triangle of R_g (zeros below), from the stack (ld M).
__global__ void load_rstack_kernel(TsqrState s, const double* Rstack) {
  const int64_t M = s.M, total = s.P * M * M;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, j = (idx / M) % M;
    s.Rs[idx] = (i <= j) ? Rstack[idx] : 0.0;
  }
}

// The chosen rank (device int64) into the shard's header, for its kernels.
__global__ void set_rank_kernel(WsHeader* h, const int64_t* r) { h->r = *r; }

struct ShardLayout {
  TsqrState ts;
  char* extra;
};

// Workspace of a shard: header | TSQR state (as pylom_pod's) | mixed extra.
size_t shard_bytes(int64_t N, int64_t M, int64_t P, int64_t r_max, int prec) {
  const bool mixed = prec == PYLOM_PREC_MIXED_3XTF32;
  return sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, !mixed) + (mixed ? mixed_extra_bytes(N, M, P) : 0);
}

ShardLayout shard_carve(void* ws, int64_t N, int64_t M, int64_t P, int64_t r_max, int prec) {
  const bool mixed = prec == PYLOM_PREC_MIXED_3XTF32;
  ShardLayout L;
  char* base = (char*)ws;
  L.ts.hdr = (WsHeader*)base;
  tsqr_state_carve(L.ts, base + sizeof(WsHeader), N, M, P, r_max, !mixed);
  L.extra = mixed ? base + sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, false) : nullptr;
  return L;
}

// Workspace of the replicated top: header | TSQR state over G "leaves"
// (no working matrix; B slots unused, the caller's B is used) | SVD | U_R.
size_t rstack_bytes(int64_t G, int64_t M, int64_t r_max) {
  return sizeof(WsHeader) + tsqr_state_bytes(0, M, G, r_max, false) + svd_state_bytes(M) +
         align256(sizeof(double) * (size_t)M * M);
}

bool aligned(const void* p) { return ((uintptr_t)p & 255u) == 0; }

bool shard_args_ok(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max, int xtype, int prec,
                   const char* who) {
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) {
    set_error_message("%s: xtype must be PYLOM_F32 or PYLOM_F64", who);
    return false;
  }
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) {
    set_error_message("%s: bad prec %d", who, prec);
    return false;
  }
  if (leaf_rows < 0 || !tall_shape_ok(N, M, leaf_rows) || r_max < 1 || r_max > M) {
    set_error_message("%s: need 1 <= M <= 4096, N_local >= M, leaf_rows 0 or >= M, 1 <= r_max <= M "
                      "(N_local=%lld M=%lld b=%lld r_max=%lld)",
                      who, (long long)N, (long long)M, (long long)leaf_rows, (long long)r_max);
    return false;
  }
  return true;
}

}  // namespace
}  // namespace pylom

using namespace pylom;

extern "C" size_t pylom_pod_shard_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max, int xtype,
                                                 int prec) {
  if (!shard_args_ok(N, M, leaf_rows, r_max, xtype, prec, "pylom_pod_shard_workspace_size")) return 0;
  return shard_bytes(N, M, leaves_of(N, M, leaf_rows, prec), r_max, prec);
}

extern "C" pylom_status pylom_pod_shard_factor(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype,
                                               const double* w, int remove_mean, int64_t leaf_rows, int64_t r_max,
                                               double* mean, double* R, int64_t ldr, int prec, void* ws,
                                               size_t ws_bytes, void* stream) {
  set_error_message("");
  if (!X || !R || !ws) {
    set_error_message("pylom_pod_shard_factor: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (!shard_args_ok(N, M, leaf_rows, r_max, xtype, prec, "pylom_pod_shard_factor")) {
    return (xtype != PYLOM_F32 && xtype != PYLOM_F64) || (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32)
               ? PYLOM_ERR_ARG
               : PYLOM_ERR_SHAPE;
  }
  if (ldx < N || ldr < M) {
    set_error_message("pylom_pod_shard_factor: leading dimension too small");
    return PYLOM_ERR_ARG;
  }
  const int64_t P = leaves_of(N, M, leaf_rows, prec);
  const size_t need = shard_bytes(N, M, P, r_max, prec);
  if (!aligned(ws) || ws_bytes < need) {
    set_error_message("pylom_pod_shard_factor: workspace needs %zu bytes, 256-byte aligned (got %zu)", need,
                      ws_bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  if (!device_readable(X, "pylom_pod_shard_factor", "X", &X)) return PYLOM_ERR_ARG;
  if (w) {
    const void* wd = nullptr;
    if (!device_readable(w, "pylom_pod_shard_factor", "w", &wd)) return PYLOM_ERR_ARG;
    w = (const double*)wd;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ShardLayout L = shard_carve(ws, N, M, P, r_max, prec);
  cudaError_t e = cudaMemsetAsync(L.ts.hdr, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.ts.arrive, 0, sizeof(unsigned) * (size_t)P, st);
  if (e == cudaSuccess)
    e = (prec == PYLOM_PREC_MIXED_3XTF32) ? launch_tsqr_mixed(L.ts, L.extra, X, ldx, xtype, w, remove_mean, mean, st)
                                          : launch_tsqr_fp64(L.ts, X, ldx, xtype, w, remove_mean, mean, st);
  if (e == cudaSuccess) e = launch_copy_root_r(L.ts, R, ldr, st);
  if (e != cudaSuccess) {
    set_error_message("pylom_pod_shard_factor: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

extern "C" size_t pylom_pod_rstack_workspace_size(int64_t G, int64_t M, int64_t r_max) {
  if (G < 1 || M < 1 || M > 4096 || r_max < 1 || r_max > M) return 0;
  return rstack_bytes(G, M, r_max);
}

extern "C" pylom_status pylom_pod_rstack(const double* Rstack, int64_t G, int64_t M, double energy, int64_t r_max,
                                         double* S, double* VT, int64_t ldvt, double* B, int64_t* r_out, void* ws,
                                         size_t ws_bytes, void* stream) {
  set_error_message("");
  if (!Rstack || !S || !VT || !B || !ws) {
    set_error_message("pylom_pod_rstack: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (G < 1 || M < 1 || M > 4096 || r_max < 1 || r_max > M) {
    set_error_message("pylom_pod_rstack: need G >= 1, 1 <= M <= 4096, 1 <= r_max <= M (G=%lld M=%lld r_max=%lld)",
                      (long long)G, (long long)M, (long long)r_max);
    return PYLOM_ERR_SHAPE;
  }
  if (ldvt < M) {
    set_error_message("pylom_pod_rstack: ldvt < M");
    return PYLOM_ERR_ARG;
  }
  const size_t need = rstack_bytes(G, M, r_max);
  if (!aligned(ws) || ws_bytes < need) {
    set_error_message("pylom_pod_rstack: workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)ws;
  TsqrState ts;
  ts.hdr = (WsHeader*)base;
  tsqr_state_carve(ts, base + sizeof(WsHeader), 0, M, G, r_max, false);
  ts.B = B;   // the top-down pass writes each shard's block straight to the caller's B
  char* p2 = base + sizeof(WsHeader) + tsqr_state_bytes(0, M, G, r_max, false);
  SvdState ss;
  ss.hdr = ts.hdr;
  svd_state_carve(ss, p2, M);
  double* UR = (double*)(p2 + svd_state_bytes(M));
  cudaError_t e = cudaMemsetAsync(ts.hdr, 0, sizeof(WsHeader), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ts.arrive, 0, sizeof(unsigned) * (size_t)G, st);
  if (e == cudaSuccess) {
    load_rstack_kernel<<<64, 256, 0, st>>>(ts, Rstack);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && G > 1) {
    if (ts.climb) {
      e = ensure_dyn_smem((const void*)tree_only_kernel, kLeafSmemBytes);
      if (e == cudaSuccess) {
        tree_only_kernel<<<(unsigned)G, kLeafThreads, kLeafSmemBytes, st>>>(ts);
        e = cudaGetLastError();
      }
    } else {
      e = launch_tree(ts, st);
    }
  }
  if (e == cudaSuccess) e = launch_svd_fp64(ss, ts.Rs, M, UR, M, S, VT, ldvt, 60, energy, r_max, st);
  if (e == cudaSuccess) e = launch_down_pass_fp64(ts, UR, M, -1, st);
  if (e == cudaSuccess && r_out) e = cudaMemcpyAsync(r_out, &ts.hdr->r, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    set_error_message("pylom_pod_rstack: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

extern "C" pylom_status pylom_pod_shard_modes(const double* Bg, const int64_t* r, int64_t N, int64_t M,
                                              int64_t leaf_rows, int64_t r_max, const double* w, int mode_kind,
                                              void* U, int64_t ldu, int prec, void* ws, size_t ws_bytes,
                                              void* stream) {
  set_error_message("");
  if (!Bg || !r || !U || !ws) {
    set_error_message("pylom_pod_shard_modes: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (mode_kind != PYLOM_MODES_ORTHONORMAL && mode_kind != PYLOM_MODES_PHYSICAL) {
    set_error_message("pylom_pod_shard_modes: bad mode_kind %d", mode_kind);
    return PYLOM_ERR_ARG;
  }
  if (!shard_args_ok(N, M, leaf_rows, r_max, PYLOM_F64, prec, "pylom_pod_shard_modes"))
    return (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) ? PYLOM_ERR_ARG : PYLOM_ERR_SHAPE;
  if (ldu < N) {
    set_error_message("pylom_pod_shard_modes: ldu < N");
    return PYLOM_ERR_ARG;
  }
  const int64_t P = leaves_of(N, M, leaf_rows, prec);
  const size_t need = shard_bytes(N, M, P, r_max, prec);
  if (!aligned(ws) || ws_bytes < need) {
    set_error_message("pylom_pod_shard_modes: workspace needs %zu bytes, 256-byte aligned (got %zu)", need,
                      ws_bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  ShardLayout L = shard_carve(ws, N, M, P, r_max, prec);
  set_rank_kernel<<<1, 1, 0, st>>>(L.ts.hdr, r);
  cudaError_t e = cudaGetLastError();
  const int phys = mode_kind == PYLOM_MODES_PHYSICAL;
  if (e == cudaSuccess)
    e = (prec == PYLOM_PREC_MIXED_3XTF32)
            ? launch_modes_mixed(L.ts, L.extra, Bg, M, -1, w, phys, (float*)U, ldu, nullptr, st, nullptr)
            : launch_modes_fp64(L.ts, Bg, M, -1, w, phys, (double*)U, ldu, nullptr, st, nullptr);
  if (e != cudaSuccess) {
    set_error_message("pylom_pod_shard_modes: %s", cudaGetErrorString(e));
    return PYLOM_ERR_CUDA;
  }
  return PYLOM_OK;
}

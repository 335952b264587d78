// api.cu -- the extern "C" entry points declared in include/pylom.h:
// argument validation, workspace layout and the launch sequence of each call.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"

using namespace pylom;

namespace {

thread_local char g_err[512] = "";

pylom_status fail(pylom_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

pylom_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return PYLOM_ERR_CUDA;
}

constexpr int64_t kMaxM = 4096;        // shared-memory bound of the tree merge and finalize
constexpr int64_t kAutoLeaves = 304;       // FP64 path: two leaves per SM of a 152-SM GB300
constexpr int64_t kAutoLeavesMixed = 152;  // mixed path: one leaf (512 tensor-memory columns) per SM
constexpr int64_t kMinAutoLeafRows = 1024;

// P = max(1, floor(N / b)) for a given leaf height b; automatic choice:
// P = min(304, floor(N / max(M, 1024))) (152 for the mixed path), at least 1.
}  // namespace

int64_t pylom::leaves_of(int64_t N, int64_t M, int64_t leaf_rows, int prec) {
  int64_t P;
  if (leaf_rows > 0) {
    P = N / leaf_rows;
  } else {
    const int64_t b = M > kMinAutoLeafRows ? M : kMinAutoLeafRows;
    const int64_t cap = (prec == PYLOM_PREC_MIXED_3XTF32) ? kAutoLeavesMixed : kAutoLeaves;
    P = N / b;
    if (P > cap) P = cap;
  }
  return P < 1 ? 1 : P;
}

bool pylom::tall_shape_ok(int64_t N, int64_t M, int64_t leaf_rows) {
  return M >= 1 && M <= kMaxM && N >= M && (leaf_rows == 0 || leaf_rows >= M);
}

namespace {

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Phase profiler: while active, each pylom_pod call records one event at
// every phase boundary on its own stream (leaf QR + tree | small SVD | down
// pass | leaf modes product).
struct PhaseProfiler {
  bool on = false;
  int cap = 0, n = 0;
  std::vector<cudaEvent_t> ev;  // cap x (PYLOM_PROFILE_PHASES + 1)
  cudaEvent_t at(int call, int k) { return ev[(size_t)call * (PYLOM_PROFILE_PHASES + 1) + k]; }
};
PhaseProfiler g_prof;

bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

}  // namespace

cudaError_t pylom::ensure_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[std::make_pair(dev, func)];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

void pylom::set_error_message(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

bool pylom::device_readable(const void* p, const char* who, const char* what, const void** dev) {
  cudaPointerAttributes at;
  memset(&at, 0, sizeof(at));
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_message("%s: %s: cudaPointerGetAttributes: %s", who, what, cudaGetErrorString(e));
    return false;
  }
  int cur = 0;
  if ((e = cudaGetDevice(&cur)) != cudaSuccess) {
    set_error_message("%s: cudaGetDevice: %s", who, cudaGetErrorString(e));
    return false;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
      if (at.device != cur) {
        set_error_message("%s: %s is memory of device %d, not of the current device %d", who, what, at.device, cur);
        return false;
      }
      *dev = p;
      return true;
    case cudaMemoryTypeManaged:
      *dev = p;
      return true;
    case cudaMemoryTypeHost:
      if (!at.devicePointer) {
        set_error_message("%s: %s is page-locked host memory not mapped into the device's address space", who,
                          what);
        return false;
      }
      *dev = at.devicePointer;
      return true;
    default:
      set_error_message("%s: %s must be device memory or page-locked host memory (cudaHostAlloc, "
                        "cudaHostRegister), not pageable host memory", who, what);
      return false;
  }
}

extern "C" const char* pylom_version(void) { return "pylom-gb300 0.1.0 (sm_103a, FP64 TSQR-SVD)"; }

extern "C" const char* pylom_last_error(void) { return g_err; }

extern "C" int64_t pylom_leaf_count(int64_t N, int64_t M, int64_t leaf_rows) {
  if (leaf_rows < 0 || !tall_shape_ok(N, M, leaf_rows)) return -1;
  return leaves_of(N, M, leaf_rows);
}

extern "C" pylom_status pylom_workspace_status(const void* ws, void* stream, int64_t* r, int* sweeps) {
  g_err[0] = 0;
  if (!ws) return fail(PYLOM_ERR_ARG, "pylom_workspace_status: null workspace");
  cudaError_t e = cudaStreamSynchronize(as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pylom_workspace_status: stream sync");
  WsHeader h;
  e = cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_workspace_status: copy");
  if (r) *r = h.r;
  if (sweeps) *sweeps = h.sweeps;
  if (h.status != PYLOM_OK)
    return fail((pylom_status)h.status, "device reported status %d", h.status);
  return PYLOM_OK;
}

// ---------------------------------------------------------------------------
// POD (Alg. 2 + Alg. 1 + Eqs. svdqr1-svdqr3)
// ---------------------------------------------------------------------------

// Workspace of pylom_pod: header | TSQR state | Jacobi state | U_R |
// (mixed only) FP32 working copy and 32-column panel factors.
static size_t pod_bytes(int64_t N, int64_t M, int64_t P, int64_t r_max, int prec = PYLOM_PREC_FP64) {
  const bool mixed = prec == PYLOM_PREC_MIXED_3XTF32;
  return sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, !mixed) + svd_state_bytes(M) +
         align256(sizeof(double) * (size_t)M * M) + (mixed ? mixed_extra_bytes(N, M, P) : 0);
}

extern "C" size_t pylom_pod_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max,
                                           int xtype, int prec) {
  if (!tall_shape_ok(N, M, leaf_rows) || r_max < 1 || r_max > M) return 0;
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) return 0;
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) return 0;
  return pod_bytes(N, M, leaves_of(N, M, leaf_rows, prec), r_max, prec);
}

extern "C" pylom_status pylom_pod(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype,
                                  const double* w, int remove_mean, double energy, int64_t r_max,
                                  int mode_kind, int64_t leaf_rows, void* U, int64_t ldu,
                                  double* S, double* VT, int64_t ldvt, double* mean,
                                  int64_t* r_out, int prec, void* ws, size_t ws_bytes,
                                  void* stream) {
  g_err[0] = 0;
  if (!X || !U || !S || !VT || !ws) return fail(PYLOM_ERR_ARG, "pylom_pod: null pointer argument");
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64)
    return fail(PYLOM_ERR_ARG, "pylom_pod: xtype must be PYLOM_F32 or PYLOM_F64");
  if (mode_kind != PYLOM_MODES_ORTHONORMAL && mode_kind != PYLOM_MODES_PHYSICAL)
    return fail(PYLOM_ERR_ARG, "pylom_pod: bad mode_kind %d", mode_kind);
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32)
    return fail(PYLOM_ERR_ARG, "pylom_pod: bad prec %d", prec);
  if (leaf_rows < 0) return fail(PYLOM_ERR_ARG, "pylom_pod: leaf_rows < 0");
  if (!tall_shape_ok(N, M, leaf_rows))
    return fail(PYLOM_ERR_SHAPE,
                "pylom_pod: need 1 <= M <= %lld, N >= M and leaf_rows 0 or >= M (N=%lld M=%lld b=%lld)",
                (long long)kMaxM, (long long)N, (long long)M, (long long)leaf_rows);
  if (r_max < 1 || r_max > M) return fail(PYLOM_ERR_SHAPE, "pylom_pod: r_max must be in [1, M]");
  if (ldx < N || ldu < N || ldvt < M) return fail(PYLOM_ERR_ARG, "pylom_pod: leading dimension too small");
  const bool mixed = prec == PYLOM_PREC_MIXED_3XTF32;
  const int64_t P = leaves_of(N, M, leaf_rows, prec);
  const size_t need = pod_bytes(N, M, P, r_max, prec);
  if (!aligned256(ws) || ws_bytes < need)
    return fail(PYLOM_ERR_WORKSPACE, "pylom_pod: workspace needs %zu bytes, 256-byte aligned (got %zu)",
                need, ws_bytes);
  if (!device_readable(X, "pylom_pod", "X", &X)) return PYLOM_ERR_ARG;
  if (w) {
    const void* wd = nullptr;
    if (!device_readable(w, "pylom_pod", "w", &wd)) return PYLOM_ERR_ARG;
    w = (const double*)wd;
  }
  cudaStream_t st = as_stream(stream);
  char* base = (char*)ws;
  WsHeader* hdr = (WsHeader*)base;
  TsqrState ts;
  ts.hdr = hdr;
  tsqr_state_carve(ts, base + sizeof(WsHeader), N, M, P, r_max, !mixed);
  char* p2 = base + sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, !mixed);
  SvdState ss;
  ss.hdr = hdr;
  svd_state_carve(ss, p2, M);
  double* UR = (double*)(p2 + svd_state_bytes(M));
  char* extra = p2 + svd_state_bytes(M) + align256(sizeof(double) * (size_t)M * M);

  const bool prof = g_prof.on && g_prof.n < g_prof.cap;
  const int call = g_prof.n;
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod: header clear");
  e = cudaMemsetAsync(ts.arrive, 0, sizeof(unsigned) * (size_t)P, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod: counter clear");
  if (prof && (e = cudaEventRecord(g_prof.at(call, 0), st)) != cudaSuccess) return cuda_fail(e, "profile");
  e = mixed ? launch_tsqr_mixed(ts, extra, X, ldx, xtype, w, remove_mean, mean, st, prof ? g_prof.at(call, 1) : nullptr)
            : launch_tsqr_fp64(ts, X, ldx, xtype, w, remove_mean, mean, st, prof ? g_prof.at(call, 1) : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod: leaf QR / tree");
  if (prof && (e = cudaEventRecord(g_prof.at(call, 2), st)) != cudaSuccess) return cuda_fail(e, "profile");
  e = launch_svd_fp64(ss, ts.Rs, M, UR, M, S, VT, ldvt, 60, energy, r_max, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod: small SVD");
  if (prof && (e = cudaEventRecord(g_prof.at(call, 3), st)) != cudaSuccess) return cuda_fail(e, "profile");
  if (mixed)
    e = launch_modes_mixed(ts, extra, UR, M, -1, w, mode_kind == PYLOM_MODES_PHYSICAL, (float*)U, ldu, r_out, st,
                           prof ? g_prof.at(call, 4) : nullptr);
  else
    e = launch_modes_fp64(ts, UR, M, -1, w, mode_kind == PYLOM_MODES_PHYSICAL, (double*)U, ldu, r_out, st,
                          prof ? g_prof.at(call, 4) : nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod: modes");
  if (prof) {
    if ((e = cudaEventRecord(g_prof.at(call, 5), st)) != cudaSuccess) return cuda_fail(e, "profile");
    ++g_prof.n;
  }
  return PYLOM_OK;
}

extern "C" pylom_status pylom_profile_begin(int max_calls) {
  g_err[0] = 0;
  if (g_prof.on) return fail(PYLOM_ERR_ARG, "pylom_profile_begin: already active");
  if (max_calls < 1 || max_calls > 100000) return fail(PYLOM_ERR_ARG, "pylom_profile_begin: bad max_calls");
  g_prof.ev.assign((size_t)max_calls * (PYLOM_PROFILE_PHASES + 1), nullptr);
  for (auto& ev : g_prof.ev) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(e, "pylom_profile_begin: event create");
  }
  g_prof.cap = max_calls;
  g_prof.n = 0;
  g_prof.on = true;
  return PYLOM_OK;
}

extern "C" pylom_status pylom_profile_end(double* phase_ms, int* calls) {
  g_err[0] = 0;
  if (!g_prof.on) return fail(PYLOM_ERR_ARG, "pylom_profile_end: not active");
  pylom_status st = PYLOM_OK;
  double acc[PYLOM_PROFILE_PHASES] = {0};
  for (int c = 0; c < g_prof.n && st == PYLOM_OK; ++c) {
    cudaError_t e = cudaEventSynchronize(g_prof.at(c, PYLOM_PROFILE_PHASES));
    if (e != cudaSuccess) { st = cuda_fail(e, "pylom_profile_end: sync"); break; }
    for (int k = 0; k < PYLOM_PROFILE_PHASES; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, g_prof.at(c, k), g_prof.at(c, k + 1));
      if (e != cudaSuccess) { st = cuda_fail(e, "pylom_profile_end: elapsed"); break; }
      acc[k] += ms;
    }
  }
  if (phase_ms)
    for (int k = 0; k < PYLOM_PROFILE_PHASES; ++k) phase_ms[k] = acc[k];
  if (calls) *calls = g_prof.n;
  for (auto& ev : g_prof.ev) if (ev) cudaEventDestroy(ev);
  g_prof.ev.clear();
  g_prof.on = false;
  g_prof.cap = g_prof.n = 0;
  return st;
}

// ---------------------------------------------------------------------------
// adjoint of the POD path
// ---------------------------------------------------------------------------

extern "C" size_t pylom_pod_backward_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r, int prec) {
  if (!tall_shape_ok(N, M, leaf_rows) || r < 0 || r > M) return 0;
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32) return 0;
  return pod_backward_bytes(N, M, leaves_of(N, M, leaf_rows, prec), r);
}

extern "C" pylom_status pylom_pod_backward(const void* fwd_ws, size_t fwd_ws_bytes, int64_t N, int64_t M,
                                           int64_t leaf_rows, int64_t r_max, int64_t r, const double* w,
                                           int remove_mean, int mode_kind, int prec, const double* S,
                                           const double* VT, int64_t ldvt, const double* dU,
                                           int64_t lddu, const double* dS, const double* dVT,
                                           int64_t lddvt, void* dX, int64_t lddx, int dxtype,
                                           void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!fwd_ws || !S || !VT || !dX || !ws) return fail(PYLOM_ERR_ARG, "pylom_pod_backward: null pointer argument");
  if (dxtype != PYLOM_F32 && dxtype != PYLOM_F64)
    return fail(PYLOM_ERR_ARG, "pylom_pod_backward: dxtype must be PYLOM_F32 or PYLOM_F64");
  if (mode_kind != PYLOM_MODES_ORTHONORMAL && mode_kind != PYLOM_MODES_PHYSICAL)
    return fail(PYLOM_ERR_ARG, "pylom_pod_backward: bad mode_kind %d", mode_kind);
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32)
    return fail(PYLOM_ERR_ARG, "pylom_pod_backward: bad prec %d", prec);
  const bool mixed = prec == PYLOM_PREC_MIXED_3XTF32;
  if (leaf_rows < 0 || !tall_shape_ok(N, M, leaf_rows))
    return fail(PYLOM_ERR_SHAPE, "pylom_pod_backward: bad shape (N=%lld M=%lld b=%lld)", (long long)N,
                (long long)M, (long long)leaf_rows);
  if (r_max < 1 || r_max > M || r < 0 || r > r_max)
    return fail(PYLOM_ERR_SHAPE, "pylom_pod_backward: need 1 <= r_max <= M and 0 <= r <= r_max");
  if (ldvt < M || (dU && lddu < N) || (dVT && lddvt < M) || lddx < N)
    return fail(PYLOM_ERR_ARG, "pylom_pod_backward: leading dimension too small");
  const int64_t P = leaves_of(N, M, leaf_rows, prec);
  if (!aligned256(fwd_ws) || fwd_ws_bytes < pod_bytes(N, M, P, r_max, prec))
    return fail(PYLOM_ERR_WORKSPACE, "pylom_pod_backward: forward workspace does not match N, M, b, r_max");
  const size_t need = pod_backward_bytes(N, M, P, r);
  if (!aligned256(ws) || ws_bytes < need)
    return fail(PYLOM_ERR_WORKSPACE, "pylom_pod_backward: workspace needs %zu bytes, 256-byte aligned", need);
  cudaStream_t st = as_stream(stream);
  char* fbase = (char*)fwd_ws;
  TsqrState fs;
  fs.hdr = (WsHeader*)fbase;
  tsqr_state_carve(fs, fbase + sizeof(WsHeader), N, M, P, r_max, !mixed);
  char* p2 = fbase + sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, !mixed);
  const double* UR = (const double*)(p2 + svd_state_bytes(M));
  char* extra = mixed ? p2 + svd_state_bytes(M) + align256(sizeof(double) * (size_t)M * M) : nullptr;
  cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod_backward: header clear");
  e = launch_pod_backward(fs, UR, S, VT, ldvt, dU, lddu, dS, dVT, lddvt, w, remove_mean,
                          mode_kind == PYLOM_MODES_PHYSICAL, r, dX, lddx, dxtype, (char*)ws, extra, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_pod_backward");
  return PYLOM_OK;
}

// ---------------------------------------------------------------------------
// TSQR (Alg. 1)
// ---------------------------------------------------------------------------

static size_t tsqr_bytes(int64_t N, int64_t M, int64_t P, int want_q) {
  return sizeof(WsHeader) + tsqr_state_bytes(N, M, P, want_q ? M : 0);
}

extern "C" size_t pylom_tsqr_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int want_q,
                                            int xtype, int prec) {
  if (!tall_shape_ok(N, M, leaf_rows)) return 0;
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) return 0;
  if (prec != PYLOM_PREC_FP64) return 0;
  return tsqr_bytes(N, M, leaves_of(N, M, leaf_rows), want_q);
}

extern "C" pylom_status pylom_tsqr(const void* A, int64_t N, int64_t M, int64_t lda, int xtype,
                                   int64_t leaf_rows, double* R, int64_t ldr, double* Q, int64_t ldq,
                                   int prec, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!A || !R || !ws) return fail(PYLOM_ERR_ARG, "pylom_tsqr: null pointer argument");
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64)
    return fail(PYLOM_ERR_ARG, "pylom_tsqr: xtype must be PYLOM_F32 or PYLOM_F64");
  if (prec != PYLOM_PREC_FP64 && prec != PYLOM_PREC_MIXED_3XTF32)
    return fail(PYLOM_ERR_ARG, "pylom_tsqr: bad prec %d", prec);
  if (leaf_rows < 0) return fail(PYLOM_ERR_ARG, "pylom_tsqr: leaf_rows < 0");
  if (!tall_shape_ok(N, M, leaf_rows))
    return fail(PYLOM_ERR_SHAPE, "pylom_tsqr: need 1 <= M <= %lld, N >= M, leaf_rows 0 or >= M",
                (long long)kMaxM);
  if (lda < N || ldr < M || (Q && ldq < N))
    return fail(PYLOM_ERR_ARG, "pylom_tsqr: leading dimension too small");
  if (prec != PYLOM_PREC_FP64)
    return fail(PYLOM_ERR_UNSUPPORTED, "pylom_tsqr: the library implements PYLOM_PREC_FP64 only here");
  const int64_t P = leaves_of(N, M, leaf_rows);
  const size_t need = tsqr_bytes(N, M, P, Q != nullptr);
  if (!aligned256(ws) || ws_bytes < need)
    return fail(PYLOM_ERR_WORKSPACE, "pylom_tsqr: workspace needs %zu bytes, 256-byte aligned", need);
  if (!device_readable(A, "pylom_tsqr", "A", &A)) return PYLOM_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  char* base = (char*)ws;
  TsqrState ts;
  ts.hdr = (WsHeader*)base;
  tsqr_state_carve(ts, base + sizeof(WsHeader), N, M, P, Q ? M : 0);
  cudaError_t e = cudaMemsetAsync(ts.hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_tsqr: header clear");
  e = cudaMemsetAsync(ts.arrive, 0, sizeof(unsigned) * (size_t)P, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_tsqr: counter clear");
  e = launch_tsqr_fp64(ts, A, lda, xtype, nullptr, 0, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_tsqr: leaf QR / tree");
  e = launch_copy_root_r(ts, R, ldr, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_tsqr: R copy");
  if (Q) {
    e = launch_modes_fp64(ts, nullptr, 0, M, nullptr, 0, Q, ldq, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "pylom_tsqr: explicit Q");
  }
  return PYLOM_OK;
}

// ---------------------------------------------------------------------------
// small SVD (Eq. svdqr2)
// ---------------------------------------------------------------------------

extern "C" size_t pylom_svd_small_workspace_size(int64_t M) {
  if (M < 1 || M > kMaxM) return 0;
  return sizeof(WsHeader) + svd_state_bytes(M);
}

extern "C" pylom_status pylom_svd_small(const double* R, int64_t M, int64_t ldr, double* U,
                                        int64_t ldu, double* S, double* VT, int64_t ldvt,
                                        int max_sweeps, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!R || !U || !S || !VT || !ws) return fail(PYLOM_ERR_ARG, "pylom_svd_small: null pointer argument");
  if (M < 1 || M > kMaxM) return fail(PYLOM_ERR_SHAPE, "pylom_svd_small: need 1 <= M <= %lld", (long long)kMaxM);
  if (ldr < M || ldu < M || ldvt < M) return fail(PYLOM_ERR_ARG, "pylom_svd_small: leading dimension too small");
  if (max_sweeps < 1 || max_sweeps > kMaxSweeps)
    return fail(PYLOM_ERR_ARG, "pylom_svd_small: max_sweeps must be in [1, %d]", kMaxSweeps);
  const size_t need = sizeof(WsHeader) + svd_state_bytes(M);
  if (!aligned256(ws) || ws_bytes < need)
    return fail(PYLOM_ERR_WORKSPACE, "pylom_svd_small: workspace needs %zu bytes, 256-byte aligned", need);
  cudaStream_t st = as_stream(stream);
  SvdState ss;
  ss.hdr = (WsHeader*)ws;
  svd_state_carve(ss, (char*)ws + sizeof(WsHeader), M);
  cudaError_t e = cudaMemsetAsync(ss.hdr, 0, sizeof(WsHeader), st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_svd_small: header clear");
  e = launch_svd_fp64(ss, R, ldr, U, ldu, S, VT, ldvt, max_sweeps, 0.0, M, st);
  if (e != cudaSuccess) return cuda_fail(e, "pylom_svd_small");
  return PYLOM_OK;
}

// ---------------------------------------------------------------------------
// local product of Alg. 4
// ---------------------------------------------------------------------------

extern "C" size_t pylom_matmul_workspace_size(int64_t m, int64_t n, int64_t k) {
  if (m < 1 || n < 1 || k < 1) return 0;
  const size_t b = matmul_ws_bytes(m, n, k);
  return b ? b : 256;
}

extern "C" pylom_status pylom_matmul(int transA, const double* A, const double* B, double* C,
                                     int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb,
                                     int64_t ldc, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!A || !B || !C) return fail(PYLOM_ERR_ARG, "pylom_matmul: null pointer argument");
  if (m < 1 || n < 1 || k < 1) return fail(PYLOM_ERR_SHAPE, "pylom_matmul: sizes must be >= 1");
  if ((transA ? lda < k : lda < m) || ldb < k || ldc < m)
    return fail(PYLOM_ERR_ARG, "pylom_matmul: leading dimension too small");
  const size_t need = matmul_ws_bytes(m, n, k);
  if (need && (!ws || !aligned256(ws) || ws_bytes < need))
    return fail(PYLOM_ERR_WORKSPACE, "pylom_matmul: workspace needs %zu bytes, 256-byte aligned", need);
  cudaError_t e = launch_matmul_fp64(transA ? 1 : 0, A, B, C, m, n, k, lda, ldb, ldc, (double*)ws,
                                     as_stream(stream));
  if (e != cudaSuccess) return cuda_fail(e, "pylom_matmul");
  return PYLOM_OK;
}

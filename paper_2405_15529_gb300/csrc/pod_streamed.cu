// pod_streamed.cu -- POD of a snapshot matrix larger than device memory
// (pyLOM, arXiv 2405.15529: the same Alg. 2 / Alg. 1 / Eqs. svdqr1-3 path,
// with X in host memory).  The leaves are processed in chunks of whole
// leaves streamed from host memory:
//   pass 1, per chunk: X rows (and weights) to the device, the leaf QR with
//     its mean / weight prologue, the leaves' reflectors back to a host
//     scratch matrix; leaf R factors, T factors and the tree stay on the
//     device, and the last-arriver tree merges across chunk launches;
//   then, on the device: the cooperative tree (large M), the small SVD,
//     the truncation and the top-down pass for every leaf;
//   pass 2, per chunk: the reflectors back to the device, the leaves'
//     modes product, the chunk of U to host memory.
// Two chunk buffers alternate; uploads and downloads run on two streams of
// their own (the link's two directions), ordered against the kernels by
// events, so chunk c+1 arrives and chunk c-1 leaves while chunk c computes.
// The results are those of the in-core pylom_pod call with the same leaf
// partition (same kernels on the same leaves).
#include "kernels.h"

namespace pylom {

struct StreamedPlan {
  int64_t P, Lc, nchunks, rows_max;
};

// A chunk must fill the device: a leaf launch over fewer leaves than two per
// SM leaves FP64 pipes idle, and the chunks' launches run one after the
// other.  With leaf_rows = 0 a chunk is therefore 304 leaves (two per SM of
// a 152-SM GB300) of about chunk_rows / 304 rows each, at least
// max(M, 1024) rows.
constexpr int64_t kStreamLeavesPerChunk = 304;
constexpr int64_t kStreamMinLeafRows = 1024;

static int64_t streamed_leaf_rows(int64_t M, int64_t leaf_rows, int64_t chunk_rows) {
  if (leaf_rows > 0) return leaf_rows;
  int64_t b = chunk_rows / kStreamLeavesPerChunk;
  if (b < kStreamMinLeafRows) b = kStreamMinLeafRows;
  if (b < M) b = M;
  return b;
}

static StreamedPlan streamed_plan(int64_t N, int64_t M, int64_t leaf_rows, int64_t chunk_rows) {
  StreamedPlan sp;
  const int64_t b = streamed_leaf_rows(M, leaf_rows, chunk_rows);
  sp.P = leaves_of(N, M, b, PYLOM_PREC_FP64);
  if (leaf_rows > 0) {
    const int64_t avg = N / sp.P > 0 ? N / sp.P : 1;
    sp.Lc = chunk_rows / avg;
  } else {
    sp.Lc = kStreamLeavesPerChunk;
  }
  if (sp.Lc < 1) sp.Lc = 1;
  if (sp.Lc > sp.P) sp.Lc = sp.P;
  sp.nchunks = (sp.P + sp.Lc - 1) / sp.Lc;
  sp.rows_max = 0;
  for (int64_t c = 0; c < sp.nchunks; ++c) {
    const int64_t L0 = c * sp.Lc, L1 = (L0 + sp.Lc < sp.P) ? L0 + sp.Lc : sp.P;
    const int64_t rows = leaf_begin(L1, N, sp.P) - leaf_begin(L0, N, sp.P);
    if (rows > sp.rows_max) sp.rows_max = rows;
  }
  return sp;
}

struct ChunkBufs {
  void* X;
  double *Y, *w, *mean, *U;
};

static size_t chunk_bytes(int64_t rows, int64_t M, int64_t r_max, size_t xs) {
  return align256(xs * (size_t)rows * M) + align256(sizeof(double) * (size_t)rows * M) +
         2 * align256(sizeof(double) * (size_t)rows) + align256(sizeof(double) * (size_t)rows * r_max);
}

static size_t streamed_bytes(int64_t N, int64_t M, const StreamedPlan& sp, int64_t r_max, size_t xs) {
  return sizeof(WsHeader) + tsqr_state_bytes(N, M, sp.P, r_max, false) + svd_state_bytes(M) +
         align256(sizeof(double) * (size_t)M * M) + 2 * chunk_bytes(sp.rows_max, M, r_max, xs);
}

static ChunkBufs carve_chunk(char* p, int64_t rows, int64_t M, int64_t r_max, size_t xs) {
  ChunkBufs b;
  b.X = p;               p += align256(xs * (size_t)rows * M);
  b.Y = (double*)p;      p += align256(sizeof(double) * (size_t)rows * M);
  b.w = (double*)p;      p += align256(sizeof(double) * (size_t)rows);
  b.mean = (double*)p;   p += align256(sizeof(double) * (size_t)rows);
  b.U = (double*)p;
  return b;
}

}  // namespace pylom

using namespace pylom;

extern "C" size_t pylom_pod_streamed_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t chunk_rows,
                                                    int64_t r_max, int xtype) {
  if (!tall_shape_ok(N, M, leaf_rows) || chunk_rows < 1 || r_max < 1 || r_max > M) return 0;
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) return 0;
  const StreamedPlan sp = streamed_plan(N, M, leaf_rows, chunk_rows);
  return streamed_bytes(N, M, sp, r_max, xtype == PYLOM_F32 ? 4 : 8);
}

extern "C" int64_t pylom_pod_streamed_leaf_rows(int64_t N, int64_t M, int64_t leaf_rows, int64_t chunk_rows) {
  if (leaf_rows < 0 || chunk_rows < 1 || !tall_shape_ok(N, M, leaf_rows)) return -1;
  return streamed_leaf_rows(M, leaf_rows, chunk_rows);
}

extern "C" pylom_status pylom_pod_streamed(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype,
                                           const double* w, int remove_mean, double energy, int64_t r_max,
                                           int mode_kind, int64_t leaf_rows, int64_t chunk_rows, double* Yh,
                                           double* U, int64_t ldu, double* S, double* VT, int64_t ldvt,
                                           double* mean, int64_t* r_out, void* ws, size_t ws_bytes,
                                           void* stream) {
  set_error_message("");
  if (!X || !Yh || !U || !S || !VT || !r_out || !ws) {
    set_error_message("pylom_pod_streamed: null pointer argument");
    return PYLOM_ERR_ARG;
  }
  if (xtype != PYLOM_F32 && xtype != PYLOM_F64) {
    set_error_message("pylom_pod_streamed: xtype must be PYLOM_F32 or PYLOM_F64");
    return PYLOM_ERR_ARG;
  }
  if (mode_kind != PYLOM_MODES_ORTHONORMAL && mode_kind != PYLOM_MODES_PHYSICAL) {
    set_error_message("pylom_pod_streamed: bad mode_kind %d", mode_kind);
    return PYLOM_ERR_ARG;
  }
  if (leaf_rows < 0 || chunk_rows < 1 || !tall_shape_ok(N, M, leaf_rows) || r_max < 1 || r_max > M) {
    set_error_message("pylom_pod_streamed: bad shape (N=%lld M=%lld b=%lld chunk=%lld r_max=%lld)", (long long)N,
                      (long long)M, (long long)leaf_rows, (long long)chunk_rows, (long long)r_max);
    return PYLOM_ERR_SHAPE;
  }
  if (ldx < N || ldu < N || ldvt < M) {
    set_error_message("pylom_pod_streamed: leading dimension too small");
    return PYLOM_ERR_ARG;
  }
  const size_t xs = xtype == PYLOM_F32 ? 4 : 8;
  const StreamedPlan sp = streamed_plan(N, M, leaf_rows, chunk_rows);
  const size_t need = streamed_bytes(N, M, sp, r_max, xs);
  if (((uintptr_t)ws & 255) != 0 || ws_bytes < need) {
    set_error_message("pylom_pod_streamed: workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    return PYLOM_ERR_WORKSPACE;
  }
  const int64_t P = sp.P;
  char* base = (char*)ws;
  WsHeader* hdr = (WsHeader*)base;
  TsqrState ts;
  ts.hdr = hdr;
  tsqr_state_carve(ts, base + sizeof(WsHeader), N, M, P, r_max, false);
  char* p2 = base + sizeof(WsHeader) + tsqr_state_bytes(N, M, P, r_max, false);
  SvdState ss;
  ss.hdr = hdr;
  svd_state_carve(ss, p2, M);
  double* UR = (double*)(p2 + svd_state_bytes(M));
  char* pc = (char*)UR + align256(sizeof(double) * (size_t)M * M);
  ChunkBufs cb[2];
  cb[0] = carve_chunk(pc, sp.rows_max, M, r_max, xs);
  cb[1] = carve_chunk(pc + chunk_bytes(sp.rows_max, M, r_max, xs), sp.rows_max, M, r_max, xs);

  cudaStream_t cs = (cudaStream_t)stream;   // kernels
  cudaStream_t up = nullptr, dn = nullptr;  // host-to-device and device-to-host copies
  cudaEvent_t loaded[2] = {nullptr, nullptr}, kdone[2] = {nullptr, nullptr}, cdone[2] = {nullptr, nullptr};
  cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&dn, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&loaded[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&kdone[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cdone[i], cudaEventDisableTiming);
  }
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) {
      if (loaded[i]) cudaEventDestroy(loaded[i]);
      if (kdone[i]) cudaEventDestroy(kdone[i]);
      if (cdone[i]) cudaEventDestroy(cdone[i]);
    }
    if (up) cudaStreamDestroy(up);   // pending work completes first
    if (dn) cudaStreamDestroy(dn);
  };
  auto fail_cuda = [&](const char* what) {
    set_error_message("pylom_pod_streamed: %s: %s", what, cudaGetErrorString(e));
    cleanup();
    return PYLOM_ERR_CUDA;
  };
  if (e != cudaSuccess) return fail_cuda("stream/event setup");
  if ((e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), cs)) != cudaSuccess) return fail_cuda("header clear");
  if ((e = cudaMemsetAsync(ts.arrive, 0, sizeof(unsigned) * (size_t)P, cs)) != cudaSuccess)
    return fail_cuda("counter clear");
  // the copy streams start after the work queued before this call
  if ((e = cudaEventRecord(kdone[0], cs)) != cudaSuccess) return fail_cuda("event");
  if ((e = cudaStreamWaitEvent(up, kdone[0], 0)) != cudaSuccess) return fail_cuda("event");
  if ((e = cudaStreamWaitEvent(dn, kdone[0], 0)) != cudaSuccess) return fail_cuda("event");

  // ---- pass 1: leaves and tree ----
  for (int64_t c = 0; c < sp.nchunks; ++c) {
    const int bi = (int)(c & 1);
    const ChunkBufs& b = cb[bi];
    const int64_t L0 = c * sp.Lc, L1 = (L0 + sp.Lc < P) ? L0 + sp.Lc : P;
    const int64_t r0 = leaf_begin(L0, N, P), rows = leaf_begin(L1, N, P) - r0;
    // the upload overwrites X and w of chunk c-2: its kernels must be done
    if (c >= 2 && (e = cudaStreamWaitEvent(up, kdone[bi], 0)) != cudaSuccess) return fail_cuda("event");
    e = cudaMemcpy2DAsync(b.X, xs * rows, (const char*)X + xs * r0, xs * ldx, xs * rows, M, cudaMemcpyHostToDevice,
                          up);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync(b.w, w + r0, sizeof(double) * rows, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(loaded[bi], up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, loaded[bi], 0);
    if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(cs, cdone[bi], 0);
    if (e != cudaSuccess) return fail_cuda("chunk upload");
    TsqrState tc = ts;
    tc.Y = b.Y;
    tc.leaf0 = L0;
    tc.Pl = L1 - L0;
    tc.row0 = r0;
    tc.ldy = rows;
    e = launch_tsqr_fp64(tc, b.X, rows, xtype, w ? b.w : nullptr, remove_mean, b.mean, cs);
    if (e == cudaSuccess) e = cudaEventRecord(kdone[bi], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dn, kdone[bi], 0);
    if (e != cudaSuccess) return fail_cuda("leaf QR");
    e = cudaMemcpy2DAsync(Yh + r0, sizeof(double) * N, b.Y, sizeof(double) * rows, sizeof(double) * rows, M,
                          cudaMemcpyDeviceToHost, dn);
    if (e == cudaSuccess && mean)
      e = cudaMemcpyAsync(mean + r0, b.mean, sizeof(double) * rows, cudaMemcpyDeviceToHost, dn);
    if (e == cudaSuccess) e = cudaEventRecord(cdone[bi], dn);
    if (e != cudaSuccess) return fail_cuda("reflector download");
  }
  // (a single chunk covers every leaf and its launch already ran the cooperative tree)
  if (!ts.climb && sp.nchunks > 1 && (e = launch_tree(ts, cs)) != cudaSuccess) return fail_cuda("tree");
  if ((e = launch_svd_fp64(ss, ts.Rs, M, UR, M, S, VT, ldvt, 60, energy, r_max, cs)) != cudaSuccess)
    return fail_cuda("small SVD");
  if ((e = launch_down_pass_fp64(ts, UR, M, -1, cs)) != cudaSuccess) return fail_cuda("top-down pass");
  // the truncation rank sizes the downloads of U
  WsHeader h;
  if ((e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, cs)) != cudaSuccess) return fail_cuda("rank");
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return fail_cuda("rank");
  if ((e = cudaStreamSynchronize(up)) != cudaSuccess) return fail_cuda("pass 1");
  if ((e = cudaStreamSynchronize(dn)) != cudaSuccess) return fail_cuda("pass 1");
  if (h.status != PYLOM_OK) {
    cleanup();
    set_error_message("pylom_pod_streamed: device reported status %d", h.status);
    return (pylom_status)h.status;
  }
  const int64_t r = h.r;
  *r_out = r;

  // ---- pass 2: modes ----
  const int physical = mode_kind == PYLOM_MODES_PHYSICAL;
  for (int64_t c = 0; c < sp.nchunks; ++c) {
    const int bi = (int)(c & 1);
    const ChunkBufs& b = cb[bi];
    const int64_t L0 = c * sp.Lc, L1 = (L0 + sp.Lc < P) ? L0 + sp.Lc : P;
    const int64_t r0 = leaf_begin(L0, N, P), rows = leaf_begin(L1, N, P) - r0;
    if (c >= 2 && (e = cudaStreamWaitEvent(up, kdone[bi], 0)) != cudaSuccess) return fail_cuda("event");
    e = cudaMemcpy2DAsync(b.Y, sizeof(double) * rows, Yh + r0, sizeof(double) * N, sizeof(double) * rows, M,
                          cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess && physical && w)
      e = cudaMemcpyAsync(b.w, w + r0, sizeof(double) * rows, cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(loaded[bi], up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, loaded[bi], 0);
    if (e == cudaSuccess && c >= 2) e = cudaStreamWaitEvent(cs, cdone[bi], 0);
    if (e != cudaSuccess) return fail_cuda("reflector upload");
    TsqrState tc = ts;
    tc.Y = b.Y;
    tc.leaf0 = L0;
    tc.Pl = L1 - L0;
    tc.row0 = r0;
    tc.ldy = rows;
    e = launch_leaf_modes_fp64(tc, r, (physical && w) ? b.w : nullptr, physical, b.U, rows, nullptr, cs);
    if (e == cudaSuccess) e = cudaEventRecord(kdone[bi], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dn, kdone[bi], 0);
    if (e != cudaSuccess) return fail_cuda("modes");
    if (r > 0)
      e = cudaMemcpy2DAsync(U + r0, sizeof(double) * ldu, b.U, sizeof(double) * rows, sizeof(double) * rows, r,
                            cudaMemcpyDeviceToHost, dn);
    if (e == cudaSuccess) e = cudaEventRecord(cdone[bi], dn);
    if (e != cudaSuccess) return fail_cuda("modes download");
  }
  // the caller's stream completes after the last copy
  const int last = (int)((sp.nchunks - 1) & 1);
  if ((e = cudaStreamWaitEvent(cs, cdone[last], 0)) != cudaSuccess) return fail_cuda("event");
  cleanup();
  return PYLOM_OK;
}

// kernels.h -- internal launchers behind the C ABI (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pylom {

// Householder panel width of the FP64 leaf QR (two 8-row DMMA tiles).
constexpr int kNB = 16;
// Below kCoopTreeMinP leaves and kCoopTreeMinM columns the tree merges run
// inside the leaf kernel (last-arriver climb); from kCoopTreeMinP leaves on
// at fewer columns, in the column-block pipeline of tree_pipe_kernel; from
// kCoopTreeMinM columns on, in tree_coop_kernel.
constexpr int64_t kCoopTreeMinM = 384;
constexpr int64_t kCoopTreeMinP = 64;
bool use_climb_tree(int64_t M, int64_t P);
bool use_pipe_tree(int64_t M, int64_t P);


// Device pointers of one TSQR (+ modes) problem, carved from a workspace.
struct TsqrState {
  WsHeader* hdr;
  int64_t N, M, P;          // rows, columns, leaves
  int64_t npan;             // panels per leaf = ceil(M / kNB)
  double* Y;                // N x M working matrix -> reflectors (ld N)
  double* tau;              // P x M leaf reflector scalars
  double* T;                // P x npan x kNB x kNB block-reflector factors
  double* Rs;               // P x M x M: leaf R, then merged R (left) or node reflectors (right)
  double* tau_tree;         // P x M tree-node reflector scalars (indexed by right child)
  unsigned* arrive;         // P arrival counters of the tree merges
  double* B;                // P x M x rmax down-pass blocks (nullable if no modes)
  int64_t rmax;
  double* Tt;               // 2 x ceil(P/2) x kNB x kNB: panel T factors in flight in the cooperative tree
  double* Tn;               // P x npan x kNB x kNB: panel T factors of the pipelined tree (by right child)
  int climb;                // 1: leaves run the last-arriver tree; 0: a tree kernel follows them
  int pipe;                 // with climb == 0: 1 tree_pipe_kernel, 0 tree_coop_kernel
  // leaf kernels of a streamed problem run on a slice of the leaves whose
  // rows sit in a device chunk: leaves leaf0 .. leaf0 + Pl - 1, buffer row 0
  // = global row row0, Y (and X, w, mean, U) chunks with leading dimension
  // ldy.  In-core: leaf0 = 0, Pl = P, row0 = 0, ldy = N.
  int64_t leaf0, Pl, row0, ldy;
};

struct SvdState {
  WsHeader* hdr;
  int64_t M, Mp;            // size, padded to even
  double* A;                // M x Mp working columns
  double* V;                // Mp x Mp accumulated rotations
  // binary32 preconditioning (M >= kJac32MinM only, else null)
  int64_t Mb;               // columns padded to a multiple of two blocks
  float* A32;               // M x Mb
  float* V32;               // Mb x Mb
  double* G;                // Mp x Mp Newton-Schulz scratch
  double* Tm;               // Mp x Mp Newton-Schulz scratch
  unsigned* rot32;          // rotations per binary32 sweep
  double* mmws;             // split-K scratch of the binary64 products
};

// From this size on, binary32 block-Jacobi sweeps precondition the binary64
// one-sided Jacobi of the small SVD (svd_jacobi32.cu).  At M = 256 they
// take the SVD from 20.3 to 16.9 ms (11 binary64 sweeps before).
constexpr int64_t kJac32MinM = 256;
size_t jacobi32_extra_bytes(int64_t M);
void jacobi32_carve(SvdState& s, char* p);
cudaError_t launch_jacobi32_precondition(const SvdState& s, const double* R, int64_t ldr, cudaStream_t st);

// with_y: include the N x M FP64 working copy (the FP64 path; the mixed
// path keeps an FP32 copy in its own extra region instead)
size_t tsqr_state_bytes(int64_t N, int64_t M, int64_t P, int64_t rmax, bool with_y = true);
void tsqr_state_carve(TsqrState& s, char* base, int64_t N, int64_t M, int64_t P, int64_t rmax,
                      bool with_y = true);
// precond: room for (and use of) the binary32 preconditioning when M >=
// kJac32MinM; without it the binary64 sweeps start from R^T
size_t svd_state_bytes(int64_t M, bool precond = true);
void svd_state_carve(SvdState& s, char* base, int64_t M, bool precond = true);

// Leaf QR of every row block (with fused mean/weight prologue) and the
// last-arriver tree reduction; the root R ends in Rs[0].
// `mid` (nullable) is recorded between the leaf kernel and the cooperative tree.
cudaError_t launch_tsqr_fp64(const TsqrState& s, const void* X, int64_t ldx, int xtype,
                             const double* w, int remove_mean, double* mean, cudaStream_t st,
                             cudaEvent_t mid = nullptr);

// The tree reduction as one cooperative launch over all blocks (for large
// M); runs after the leaf kernel when s.climb == 0.
cudaError_t launch_tree_coop(const TsqrState& s, cudaStream_t st);
// The tree reduction as a column-block pipeline, one block per merge.
cudaError_t launch_tree_pipe(const TsqrState& s, cudaStream_t st);
// launch_tree_pipe or launch_tree_coop as s.pipe says (s.climb == 0)
cudaError_t launch_tree(const TsqrState& s, cudaStream_t st);

// Copy the root R (upper triangle) into an M x M matrix with zeros below.
cudaError_t launch_copy_root_r(const TsqrState& s, double* R, int64_t ldr, cudaStream_t st);

// Parallel one-sided Jacobi + sort/sign/truncate.  Input R (M x M, ldr).
// Writes U (M x M, ldu), S, VT (ldvt) and, if energy/r_max given, hdr->r.
cudaError_t launch_svd_fp64(const SvdState& s, const double* R, int64_t ldr, double* U, int64_t ldu,
                            double* S, double* VT, int64_t ldvt, int max_sweeps, double energy,
                            int64_t r_max, cudaStream_t st);

// Down pass through the tree (B_root = first r columns of Ur, or identity when
// Ur == nullptr) and the per-leaf modes product U = Q [B_leaf; 0].  The number
// of columns is r_fixed if >= 0, else read from hdr->r on the device.
// `mid` (nullable) is recorded between the down pass and the leaf modes kernel.
cudaError_t launch_modes_fp64(const TsqrState& s, const double* Ur, int64_t ldur, int64_t r_fixed,
                              const double* w, int physical, double* U, int64_t ldu,
                              int64_t* r_out, cudaStream_t st, cudaEvent_t mid = nullptr);

// Adjoint of the POD path (pod_backward.cu).  fs: the forward's TSQR state
// (reflectors, T, tree); UR/S/VT: the forward's small-SVD factors.
size_t pod_backward_bytes(int64_t N, int64_t M, int64_t P, int64_t r);
cudaError_t launch_pod_backward(const TsqrState& fs, const double* UR, const double* S, const double* VT,
                                int64_t ldvt, const double* dU, int64_t lddu, const double* dS,
                                const double* dVT, int64_t lddvt, const double* w, int remove_mean,
                                int physical, int64_t r, void* dX, int64_t lddx, int dxtype,
                                char* bw_base, char* mixed_extra, cudaStream_t st);
// Mixed-precision adjoint support (tsqr_mixed.cu): per leaf C := Q_leaf^T C
// (FP32, ld N) on tcgen05, top M rows into the binary64 slots Z.
cudaError_t launch_leaf_qt_mixed(const TsqrState& s, char* extra, float* C, int64_t r, double* Z, cudaStream_t st);

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  Function attributes belong to a device, so the setting
// is remembered per (device, kernel); thread-safe.
cudaError_t ensure_dyn_smem(const void* func, size_t bytes);

// Records a message for pylom_last_error() on the calling host thread.
void set_error_message(const char* fmt, ...);

// An input the kernels read: memory of the current device, managed memory,
// or page-locked host memory mapped into the device's address space (the
// kernels then read it across the host link, with no separate copy).
// *dev receives the address the kernels use.  Anything else -- pageable host
// memory, another device's memory -- returns false with the error message
// set, before any launch.
bool device_readable(const void* p, const char* who, const char* what, const void** dev);

// Leaf count of a problem (the rule of pylom_leaf_count; the mixed path caps
// the automatic choice at one leaf per SM) and the shape check of the
// tall-skinny entry points (api.cu).
int64_t leaves_of(int64_t N, int64_t M, int64_t leaf_rows, int prec = PYLOM_PREC_FP64);
bool tall_shape_ok(int64_t N, int64_t M, int64_t leaf_rows);

// The leaves' modes product alone (after the top-down pass), for the leaf
// slice of s (streamed problems).
cudaError_t launch_leaf_modes_fp64(const TsqrState& s, int64_t r_fixed, const double* w, int physical, double* U,
                                   int64_t ldu, int64_t* r_out, cudaStream_t st);

// Top-down pass only (B_root from Ur or the identity, then every tree level).
cudaError_t launch_down_pass_fp64(const TsqrState& s, const double* Ur, int64_t ldur, int64_t r_fixed,
                                  cudaStream_t st);

// Mixed-precision leaves (tsqr_mixed.cu): FP32 working copy + 32-column
// panel factors in an extra region; 3xTF32 block reflectors on tcgen05.
size_t mixed_extra_bytes(int64_t N, int64_t M, int64_t P);
cudaError_t launch_tsqr_mixed(const TsqrState& s, char* extra, const void* X, int64_t ldx, int xtype,
                              const double* w, int remove_mean, double* mean, cudaStream_t st,
                              cudaEvent_t mid = nullptr);
cudaError_t launch_modes_mixed(const TsqrState& s, char* extra, const double* Ur, int64_t ldur, int64_t r_fixed,
                               const double* w, int physical, float* U, int64_t ldu, int64_t* r_out,
                               cudaStream_t st, cudaEvent_t mid);

// C = op(A) B in binary64 on the FP64 tensor pipe.
size_t matmul_ws_bytes(int64_t m, int64_t n, int64_t k);
cudaError_t launch_matmul_fp64(int transA, const double* A, const double* B, double* C, int64_t m,
                               int64_t n, int64_t k, int64_t lda, int64_t ldb, int64_t ldc,
                               double* ws, cudaStream_t st);

}  // namespace pylom

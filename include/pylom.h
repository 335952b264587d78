/*
 * pylom.h -- C ABI of the GB300 (sm_103a) POD / TSQR-SVD library.
 *
 * The library computes the proper orthogonal decomposition of a tall-skinny
 * snapshot matrix X (N gridpoints x M snapshots) the way pyLOM does
 * (Eiximeno et al., arXiv 2405.15529, Sec. 3.1 and Algs. 1, 2 and 4):
 *   temporal mean removal (Alg. 2) and optional sqrt(cell-volume) weights,
 *   a TSQR -- blocked Householder QR of row blocks ("leaves") followed by a
 *   binary-tree reduction of the stacked R factors (Alg. 1; on one GPU the
 *   tree runs across thread blocks),
 *   an SVD of the small M x M R (Eq. svdqr2),
 *   and the modes U = Q U_r (Eq. svdqr3).
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *   - Every array argument is DEVICE memory owned by the caller, unless the
 *     comment says "host".  The snapshot inputs (X of pylom_pod, pylom_tsqr,
 *     pylom_dmd and pylom_pod_shard_factor, D of pylom_spod_blocks, and w)
 *     may also be managed memory or page-locked host memory mapped into the
 *     device's address space, read by the kernels across the host link;
 *     pageable host memory or another device's memory there returns
 *     PYLOM_ERR_ARG before any launch.  The library never allocates: each call that needs
 *     scratch takes a caller-provided device workspace whose size comes from
 *     the matching *_workspace_size query.  Workspaces must be 256-byte
 *     aligned and must not be shared by calls that may overlap on the GPU.
 *   - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).
 *   - Arguments are validated on the host before anything is launched; an
 *     invalid call returns an error status and writes no output.
 *   - Conditions only the device can see (non-finite input, Jacobi not
 *     converged, a bounded wait that ran out) are recorded in the workspace
 *     header and read back with pylom_workspace_status().
 *   - A failed CUDA launch returns PYLOM_ERR_CUDA; pylom_last_error() gives
 *     the message (thread-local, valid until the next call on the thread).
 */
#ifndef PYLOM_H
#define PYLOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PYLOM_OK = 0,
  PYLOM_ERR_ARG = 1,         /* null pointer, bad enum, bad leading dimension */
  PYLOM_ERR_SHAPE = 2,       /* N < M, M < 1, leaf height < M, r_max out of range */
  PYLOM_ERR_WORKSPACE = 3,   /* workspace too small or misaligned */
  PYLOM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  PYLOM_ERR_NONFINITE = 5,   /* device: the input holds NaN or Inf */
  PYLOM_ERR_NOCONV = 6,      /* device: Jacobi SVD hit max_sweeps */
  PYLOM_ERR_TIMEOUT = 7,     /* device: a bounded inter-block wait ran out */
  PYLOM_ERR_UNSUPPORTED = 8, /* valid request the library does not implement */
  PYLOM_ERR_SINGULAR = 9     /* device: a matrix that must be positive definite is not (DMD amplitudes) */
} pylom_status;

typedef enum { PYLOM_F32 = 0, PYLOM_F64 = 1, PYLOM_C64 = 2, PYLOM_C128 = 3 } pylom_dtype;

/* Arithmetic of the hot path.
 * FP64: every step in binary64 (trailing updates and the modes product on
 *   the FP64 tensor pipe, mma.sync.m8n8k4).
 * MIXED_3XTF32: FP32 leaf working copy; panel sums compensated in FP32 and
 *   reduced in FP64; the leaves' block-reflector products (trailing updates
 *   and U = Q [B; 0]) on the tcgen05 tensor cores in 3xTF32 (each FP32
 *   operand split into a TF32 high part and an FP32 remainder, three MMAs,
 *   FP32 accumulation in tensor memory); the tree merges, the small SVD of R,
 *   the mean and the top-down pass stay in binary64. */
typedef enum { PYLOM_PREC_FP64 = 0, PYLOM_PREC_MIXED_3XTF32 = 1 } pylom_prec;

/* Which left vectors pylom_pod returns (only differs when w != NULL).
 * ORTHONORMAL: U_w, the left singular vectors of Y_w = diag(sqrt w) Y,
 *              Euclidean-orthonormal.
 * PHYSICAL:    Phi = diag(w)^(-1/2) U_w, orthonormal in the volume-weighted
 *              inner product sum_n w_n Phi_i(n) Phi_j(n) (the discrete form of
 *              the integral orthonormality of Sec. 2.1). */
typedef enum { PYLOM_MODES_ORTHONORMAL = 0, PYLOM_MODES_PHYSICAL = 1 } pylom_mode_kind;

/* Library version string (static storage). */
const char* pylom_version(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* pylom_last_error(void);

/* Number of TSQR leaves for an N-row problem with leaf height hint
 * leaf_rows = b: P = max(1, floor(N / b)); leaf_rows = 0 picks
 * P = max(1, min(304, floor(N / max(M, 1024)))) (the FP64 path; the mixed
 * path of pylom_pod caps the automatic choice at 152, one leaf per SM).  Leaf i owns rows
 * [floor(i N / P), floor((i+1) N / P)), so every leaf has >= M rows.
 * Returns -1 on invalid arguments. */
int64_t pylom_leaf_count(int64_t N, int64_t M, int64_t leaf_rows);

/* Tree reduction of the leaf R factors (Sec. 3.1, the reduce loop of
 * Alg. 1), used by pylom_pod and pylom_tsqr.  Below 384 columns and 64
 * leaves the leaf kernels merge pairs as they finish (the second block to
 * reach a merge performs it); from 64 leaves at fewer than 384 columns, one
 * cooperative launch after the leaves gives every merge one thread block
 * that runs one 16-column block behind its two children (a pipeline over
 * the levels); from 384 columns on, one cooperative launch spreads every
 * merge of a level over all thread blocks, one panel of 16 columns per
 * grid-wide step.  All three leave the same pairing, merged R and node
 * reflectors.  The environment variable PYLOM_TREE = "climb",
 * "pipe" or "coop", read at each call, forces one form (testing and
 * tuning). */

/* Device status recorded in a workspace by the last call that used it.
 * Synchronises `stream`, then returns the recorded pylom_status
 * (PYLOM_OK if none) and, when the pointers are non-NULL, writes to HOST
 * memory the truncation rank chosen by pylom_pod (*r) and the Jacobi sweeps
 * used (*sweeps). */
pylom_status pylom_workspace_status(const void* ws, void* stream, int64_t* r, int* sweeps);

/* ------------------------------------------------------------------------
 * pylom_pod -- POD of Alg. 2: Y = X - xbar 1^T (if remove_mean), weighted
 * Y_w = diag(sqrt w) Y (if w != NULL), then Y_w = U S V^T by TSQR + small
 * SVD + U = Q U_r (Eqs. svdqr1-svdqr3, Alg. 1), truncated by cumulative
 * energy (Sec. 3.1).
 *
 *  X      in   N x M, ldx >= N, element type xtype (PYLOM_F32 or PYLOM_F64).
 *              Not modified.  Device memory of the current device, managed
 *              memory, or page-locked host memory mapped into the device's
 *              address space (cudaHostAlloc / cudaHostRegister): the leaf
 *              kernel's prologue then reads X across the host link, so no
 *              separate upload is needed.  Pageable host memory or another
 *              device's memory returns PYLOM_ERR_ARG before any launch (the
 *              same holds for w, and for the inputs of pylom_tsqr,
 *              pylom_dmd, pylom_pod_shard_factor and pylom_spod_blocks).
 *  w      in   N cell volumes (> 0), or NULL for uniform weights.
 *  remove_mean  1: subtract the per-gridpoint temporal mean (Alg. 2).
 *  energy       keep r = min{k : sum_{i<=k} S_i^2 / sum_i S_i^2 >= energy},
 *               capped at r_max; energy <= 0 keeps r = r_max.
 *  r_max        1 <= r_max <= M: the columns U has room for.
 *  mode_kind    pylom_mode_kind (see above).
 *  leaf_rows    TSQR leaf height hint b (0 = automatic; else b >= M).
 *  U      out  N x r_max, ldu >= N: the first r columns receive the
 *              modes, the rest are left untouched.  Element type: binary64
 *              for PYLOM_PREC_FP64, binary32 for PYLOM_PREC_MIXED_3XTF32.
 *  S      out  M singular values, descending.
 *  VT     out  M x M, ldvt >= M: row i is v_i^T, the temporal coefficients
 *              of mode i (Sec. 3.1).  Each pair (u_i, v_i) is signed so that
 *              the largest-magnitude entry of v_i is positive (lowest index
 *              on a tie).
 *  mean   out  N temporal means (zeros if !remove_mean), or NULL.
 *  r_out  out  device int64: the chosen r, or NULL (also readable through
 *              pylom_workspace_status).
 *  prec         pylom_prec (both implemented).
 *  ws, ws_bytes device workspace of at least pylom_pod_workspace_size().
 * ------------------------------------------------------------------------ */
size_t pylom_pod_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max,
                                int xtype, int prec);
pylom_status pylom_pod(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype,
                       const double* w, int remove_mean, double energy, int64_t r_max,
                       int mode_kind, int64_t leaf_rows,
                       void* U, int64_t ldu, double* S, double* VT, int64_t ldvt,
                       double* mean, int64_t* r_out, int prec,
                       void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_dmd -- exact dynamic mode decomposition with optimal amplitudes
 * (Sec. 3.2, Alg. 3; amplitudes Alg. 5; the product U^T Y2 of Alg. 4).
 *   Y = X - mean (each point's mean over all M snapshots, if remove_mean),
 *   Y1 = Y[:, :M-1], Y2 = Y[:, 1:], Y1 = U S V^T truncated to r,
 *   A = U^T Y2 V S^-1 (r x r), A w = w diag(mu),
 *   phi = Y2 V S^-1 w diag(mu)^-1 (exact DMD modes),
 *   b minimising || S V^T - w diag(b) V_and ||_F, V_and[i, t] = mu_i^t,
 *   modes ordered by |b| descending (a conjugate pair shares the larger |b|
 *   of its members, stays adjacent, positive imaginary part first).
 * One TSQR of Y serves both Y1 and Y2 (Y1's QR is the leading part of Y's),
 * so X is read once and the small steps run on matrices of <= M rows.
 *  X      device N x M (ldx >= N), F32 or F64; 2 <= M <= 4096, N >= M.
 *  energy, r_max  truncation of the SVD of Y1 as in pylom_pod (1 <= r_max
 *         <= M-1); r is further cut to the numerical rank of Y1 (singular
 *         values above max(N, M-1) 2^-52 s_1), so S^-1 exists.
 *  mu, b  device out, 2 r_max doubles each: (re, im) of the sorted
 *         eigenvalues and amplitudes.
 *  Phi    device out N x r_max doubles (ldphi >= N), the sorted modes in
 *         the packed real layout: a real eigenvalue's mode is one column;
 *         a conjugate pair (mu_p, mu_p+1 = conj mu_p) stores Re phi_p in
 *         column p and Im phi_p in column p+1 (phi_p+1 = conj phi_p).
 *         Eigenvectors w are normalised to unit norm with their first
 *         entry of largest modulus real and positive.
 *  S      device out, the M-1 singular values of Y1.
 *  mean   device out N doubles or NULL.  r_out: device int64, the rank r.
 *  leaf_rows as in pylom_pod.  Device statuses (read with
 *  pylom_workspace_status): PYLOM_ERR_NONFINITE, PYLOM_ERR_NOCONV (the
 *  SVD, or the eigenvalue QR after 60 r + 100 double-shift steps),
 *  PYLOM_ERR_SINGULAR (P of the amplitudes not positive definite, e.g.
 *  repeated eigenvalues).  Asynchronous on `stream`; workspace:
 *  pylom_dmd_workspace_size(N, M, leaf_rows, r_max, xtype) bytes,
 *  256-byte aligned.
 * ------------------------------------------------------------------------ */
size_t pylom_dmd_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max, int xtype);
pylom_status pylom_dmd(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype, int remove_mean, double energy,
                       int64_t r_max, int64_t leaf_rows, double* mu, double* b, double* Phi, int64_t ldphi,
                       double* S, double* mean, int64_t* r_out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_pod_streamed -- pylom_pod (binary64 path) for a snapshot matrix in
 * HOST memory that need not fit in device memory (the paper's largest
 * datasets exceed any single device).  The leaves (the partition of
 * pylom_leaf_count) are processed in chunks of whole leaves of at most
 * about chunk_rows rows: pass 1 uploads each chunk of X (and w), runs the
 * leaf QR with its mean / weight prologue and downloads the reflectors to
 * the host scratch Yh; the tree, the small SVD, the truncation and the
 * top-down pass run on the device; pass 2 uploads the reflectors again and
 * downloads each chunk of U.  Two chunk buffers alternate and copies run on
 * a second stream, so transfers overlap the kernels.  Results equal those
 * of pylom_pod with the same leaf partition.
 *  X      host N x M (ldx >= N), F32 or F64; w: host N doubles or NULL;
 *  Yh     host scratch N x M doubles (ld N), overwritten;
 *  U      host out N x r (ldu >= N, at least r_max columns);
 *  S, VT  DEVICE out as in pylom_pod; mean: host N doubles or NULL;
 *  r_out  host out, the truncation rank.
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister)
 * for the copies to overlap.  Synchronises `stream` once (to read r); on
 * return the remaining work is queued on `stream`.  Device workspace:
 * pylom_pod_streamed_workspace_size(N, M, leaf_rows, chunk_rows, r_max,
 * xtype) bytes, 256-byte aligned.  Device statuses (non-finite input, ...)
 * are returned directly.
 *  leaf_rows = 0 sizes the leaves for the chunks: a chunk is 304 leaves
 *  (two per SM, so every chunk launch fills the device) of
 *  b = max(M, 1024, chunk_rows / 304) rows, and the results equal those of
 *  pylom_pod with leaf_rows = b; pylom_pod_streamed_leaf_rows returns the b
 *  a call uses (leaf_rows itself when > 0; -1 for a bad shape).  With
 *  leaf_rows > 0 a chunk holds max(1, chunk_rows / (N / P)) leaves.
 * ------------------------------------------------------------------------ */
int64_t pylom_pod_streamed_leaf_rows(int64_t N, int64_t M, int64_t leaf_rows, int64_t chunk_rows);
size_t pylom_pod_streamed_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t chunk_rows,
                                         int64_t r_max, int xtype);
pylom_status pylom_pod_streamed(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype, const double* w,
                                int remove_mean, double energy, int64_t r_max, int mode_kind, int64_t leaf_rows,
                                int64_t chunk_rows, double* Yh, double* U, int64_t ldu, double* S, double* VT,
                                int64_t ldvt, double* mean, int64_t* r_out, void* ws, size_t ws_bytes,
                                void* stream);

/* ------------------------------------------------------------------------
 * Row-sharded POD -- the paper's parallel form (Sec. 3.1, Alg. 1: every
 * process owns a block of rows, a binary tree reduces their R factors, the
 * result is broadcast back down the tree), with the row blocks as shards
 * that may live on different devices.  The only data exchanged between
 * shards is the G factors R_g (G * M * M doubles), which the caller
 * gathers (an all-gather across devices; Alg. 4's all_reduce is the same
 * collective pattern).  Per shard g holding rows X_g (N_g x M), in order:
 *   pylom_pod_shard_factor  a1-a3 on X_g: mean removal and sqrt(w) weights
 *       (the mean is per row, so local), leaf QR and the tree of the shard's
 *       own leaves; writes R_g (M x M upper triangular, zeros below, ldr >=
 *       M).  The reflectors stay in the shard's workspace ws, which must be
 *       kept unchanged until pylom_pod_shard_modes.
 *   (caller) gather R_0 .. R_{G-1} into one stack, shard g at Rstack +
 *       g M M (each M x M, ld M), on every shard.
 *   pylom_pod_rstack  replicated on every shard: the top of the tree over
 *       the G stacked factors with Alg. 1's XOR pairing (shard ids in place
 *       of process ids; an unpaired shard passes its R up), the SVD of the
 *       root R (Eq. svdqr2), the truncation (energy, r_max as in
 *       pylom_pod), and the top-down pass: B receives G blocks of
 *       M x r_max (ld M), block g at B + g M r_max, the rows of
 *       Q_top [U_r; 0] that belong to shard g.  S (M), VT (M x M, ldvt >= M)
 *       as pylom_pod.  r_out: device int64, the rank r.
 *   pylom_pod_shard_modes  a6-a7 on the shard: the top-down pass through
 *       its own tree from B_g (block g of B) and U_g = Q_g [B_g; 0] for the
 *       shard's rows; r is the device int64 from pylom_pod_rstack.  U: N_g x
 *       r_max (ldu >= N_g), binary64 for PYLOM_PREC_FP64, binary32 for
 *       PYLOM_PREC_MIXED_3XTF32; mode_kind and w as pylom_pod.
 * N_g, M, leaf_rows, r_max, xtype and prec must be the same in a shard's
 * factor and modes calls.  Each shard's rows must satisfy N_g >= M.  The
 * stacked result equals pylom_pod of the stacked X up to rounding (the tree
 * pairs differ).  Device statuses go to the respective workspaces
 * (pylom_workspace_status).  Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
size_t pylom_pod_shard_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r_max, int xtype, int prec);
pylom_status pylom_pod_shard_factor(const void* X, int64_t N, int64_t M, int64_t ldx, int xtype, const double* w,
                                    int remove_mean, int64_t leaf_rows, int64_t r_max, double* mean, double* R,
                                    int64_t ldr, int prec, void* ws, size_t ws_bytes, void* stream);
size_t pylom_pod_rstack_workspace_size(int64_t G, int64_t M, int64_t r_max);
pylom_status pylom_pod_rstack(const double* Rstack, int64_t G, int64_t M, double energy, int64_t r_max, double* S,
                              double* VT, int64_t ldvt, double* B, int64_t* r_out, void* ws, size_t ws_bytes,
                              void* stream);
pylom_status pylom_pod_shard_modes(const double* Bg, const int64_t* r, int64_t N, int64_t M, int64_t leaf_rows,
                                   int64_t r_max, const double* w, int mode_kind, void* U, int64_t ldu, int prec,
                                   void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_pod_backward -- hand-written adjoint of pylom_pod (no counterpart in
 * the paper; it differentiates the composition of Alg. 2, Alg. 1 and Eqs.
 * svdqr1-svdqr3).  Given cotangents dU (of the r returned modes), dS and
 * dVT, writes dX, the cotangent of X.  Q is recomputed from the leaf and
 * tree reflectors that the forward call left in its workspace (Q^T dU by
 * the leaf reflectors and a bottom-up tree pass; Q [B; 0] by the top-down
 * pass); the square SVD adjoint of R runs in binary64 on M x M matrices.
 *  fwd_ws, fwd_ws_bytes  the workspace of the pylom_pod call being
 *                        differentiated, unchanged since (same N, M,
 *                        leaf_rows, r_max, w, remove_mean, mode_kind, prec).
 *  prec    that call's precision: PYLOM_PREC_FP64 (Q applied in binary64 on
 *          the FP64 tensor pipe) or PYLOM_PREC_MIXED_3XTF32 (Q^T dU and
 *          Q [B; 0] by the forward's FP32 reflectors in 3xTF32 on tcgen05,
 *          dU C in FP32; the tree passes and the square SVD adjoint stay
 *          binary64).
 *  r       number of modes whose cotangent dU holds (0 <= r <= r_max).
 *  S, VT   that call's singular values and right vectors (ldvt >= M).
 *  dU      N x r (lddu >= N) or NULL; dS: M or NULL; dVT: M x M or NULL.
 *  dX      out, N x M (lddx >= N), element type dxtype (F32 or F64).
 * Degenerate singular values (s_i == s_j) contribute no coupling term; the
 * singular values of the r modes that carry a cotangent must be nonzero
 * (R itself may be singular, as it is once the mean is removed).
 * ------------------------------------------------------------------------ */
size_t pylom_pod_backward_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int64_t r, int prec);
pylom_status pylom_pod_backward(const void* fwd_ws, size_t fwd_ws_bytes, int64_t N, int64_t M,
                                int64_t leaf_rows, int64_t r_max, int64_t r, const double* w,
                                int remove_mean, int mode_kind, int prec, const double* S, const double* VT,
                                int64_t ldvt, const double* dU, int64_t lddu, const double* dS,
                                const double* dVT, int64_t lddvt, void* dX, int64_t lddx, int dxtype,
                                void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_tsqr -- tall-skinny QR of Alg. 1: A = Q [R; 0] (Eq. svdqr1).
 *  A      in   N x M, lda >= N, xtype F32 or F64 (not modified).
 *  R      out  M x M upper triangular (zeros below the diagonal), ldr >= M.
 *              Row signs follow the Householder convention
 *              beta = -sign(alpha) |x| at every leaf and tree node, so R is
 *              fixed up to row signs by A (compare R^T R or |R_ii|).
 *  Q      out  N x M explicit orthonormal factor, ldq >= N, or NULL to skip
 *              (the top-down broadcast pass of Alg. 1, then Q_i = Q_1i Q_w
 *              on every leaf).
 * ------------------------------------------------------------------------ */
size_t pylom_tsqr_workspace_size(int64_t N, int64_t M, int64_t leaf_rows, int want_q,
                                 int xtype, int prec);
pylom_status pylom_tsqr(const void* A, int64_t N, int64_t M, int64_t lda, int xtype,
                        int64_t leaf_rows, double* R, int64_t ldr, double* Q, int64_t ldq,
                        int prec, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_svd_small -- SVD of the small M x M factor, R = U S V^T
 * (Eq. svdqr2), by parallel one-sided Jacobi in binary64 across thread
 * blocks (round-robin pair ordering; a pair rotates while
 * |a_i.a_j| > M 2^-53 |a_i| |a_j|).  Sorted descending, same sign rule as
 * pylom_pod.  R is any M x M matrix (triangular or not), not modified.
 *  U out M x M (ldu >= M), S out M, VT out M x M (ldvt >= M).
 *  max_sweeps   1..64; not converging records PYLOM_ERR_NOCONV.
 * ------------------------------------------------------------------------ */
size_t pylom_svd_small_workspace_size(int64_t M);
pylom_status pylom_svd_small(const double* R, int64_t M, int64_t ldr, double* U, int64_t ldu,
                             double* S, double* VT, int64_t ldvt, int max_sweeps,
                             void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * SPOD front end (Sec. 2.3, Alg. 6): the matrices Q_f of every frequency.
 * The snapshots D (N points x T instants) are cut into nBlks blocks of npwin
 * instants overlapping by nolap (nBlks = floor((T - nolap)/(npwin - nolap)),
 * block b starting at instant b (npwin - nolap)); optionally each point's
 * temporal mean is removed; every point's block is multiplied by the
 * Hamming window w_j = 0.54 - 0.46 cos(2 pi j/(npwin - 1)), j = 0..npwin-1,
 * transformed (X_k = sum_j x_j w_j exp(-2 pi i k j / npwin)), divided by
 * mean(w) npwin, and the one-sided spectrum k = 0 .. floor(npwin/2) keeps
 * all entries but its first and last doubled (as Alg. 6 writes it).  Q_f
 * gathers frequency f of every block, scaled by 1/sqrt(nBlks), so
 * Q_f = U_f S_f V_f^H is the SVD that pylom_svd_batched_* computes and
 * L_f = S_f^2 the SPOD energies; frequency f is f / (dt npwin).
 *   pylom_spod_shape      nBlks and nfreq = floor(npwin/2) + 1 for T, npwin,
 *                         nolap (2 <= npwin <= 512, 0 <= nolap < npwin,
 *                         T >= npwin).
 *   pylom_spod_blocks     D: device N x T (ldd >= N), dtype F32 or F64, not
 *                         modified.  Q: device complex64, nfreq matrices of
 *                         N x nBlks (column-major, ld ldq >= N), matrix f at
 *                         Q + f * nBlks * ldq elements.  mean: device N
 *                         doubles or NULL (written when remove_mean).
 *                         Workspace: pylom_spod_blocks_workspace_size(N,
 *                         npwin) bytes, 256-byte aligned.  FP32 arithmetic,
 *                         the mean and the tables in binary64.  Capturable.
 *   pylom_spod_order      order[i] = the frequency with the i-th largest
 *                         leading energy S[f * stride]^2 (ties by index),
 *                         S on the device (the packed S of the batched SVD,
 *                         stride nBlks), order: device nfreq int64.
 * ------------------------------------------------------------------------ */
pylom_status pylom_spod_shape(int64_t T, int64_t npwin, int64_t nolap, int64_t* nblks, int64_t* nfreq);
size_t pylom_spod_blocks_workspace_size(int64_t N, int64_t npwin);
pylom_status pylom_spod_blocks(const void* D, int64_t N, int64_t T, int64_t ldd, int dtype, int64_t npwin,
                               int64_t nolap, int remove_mean, void* Q, int64_t ldq, double* mean, void* ws,
                               size_t ws_bytes, void* stream);
pylom_status pylom_spod_order(const double* S, int64_t nfreq, int64_t stride, int64_t* order, void* stream);

/* ------------------------------------------------------------------------
 * Batched complex SVDs -- the per-frequency SVDs of SPOD (Sec. 2.3, Alg. 6:
 * (1/sqrt(nBlks)) Q_f = U_f S_f V_f^H for every frequency bin f), all bins
 * in one cooperative persistent launch.  Each bin: TSQR with complex
 * Householder leaves and a last-arriver tree (Alg. 1), one-sided Jacobi SVD
 * of its R (Eq. svdqr2), modes U_f = Q_f U_r (Eq. svdqr3).
 * Three steps, so the launch can be captured in a CUDA graph:
 *   plan  (host only): bin sizes N[f] x Nb[f] (1 <= Nb <= 128, N >= Nb),
 *         optional per-bin leaf heights (NULL or <= 0: built-in choice, an
 *         autotuner may supply them; leaves never exceed 1024 rows for
 *         complex64 or 512 for complex128 -- a bin is split into more
 *         leaves where needed), kmodes (0..32 modes returned per bin,
 *         capped at Nb), prec: PYLOM_PREC_FP64 (complex128 leaves) or
 *         PYLOM_PREC_MIXED_3XTF32 (complex64 leaves with compensated FP32
 *         sums; tree, Jacobi and R always binary64).  Returns an opaque plan
 *         and the workspace size.
 *   bind  Q[f]: device pointer (host array of them) to bin f's complex64
 *         N x Nb matrix (column-major, ldq[f] >= N), not modified; U[f]:
 *         device complex64 N x min(kmodes, Nb) output (ldu[f] >= N); writes
 *         the plan's tables into the workspace and synchronises `stream`.
 *         Not capturable; call once per set of buffers.
 *   run   S: device doubles, sum_f Nb[f], bin f at offset
 *         pylom_svd_batched_plan_info(plan, f, 2), descending per bin;
 *         U[f] columns carry the phase rule (the largest |entry| of each
 *         right vector real and positive).  Capturable (memsets + one
 *         cooperative kernel, no host synchronisation).
 * Device-side conditions (non-finite input, Jacobi not converged, a bounded
 * wait that expired) go to the workspace header (pylom_workspace_status).
 * ------------------------------------------------------------------------ */
typedef struct pylom_batched_plan pylom_batched_plan;
pylom_status pylom_svd_batched_plan(int nbins, const int64_t* N, const int64_t* Nb,
                                    const int64_t* leaf_rows, int64_t kmodes, int prec,
                                    pylom_batched_plan** plan, size_t* ws_bytes);
pylom_status pylom_svd_batched_bind(pylom_batched_plan* plan, const void* const* Q, const int64_t* ldq,
                                    void* const* U, const int64_t* ldu, void* ws, size_t ws_bytes,
                                    void* stream);
pylom_status pylom_svd_batched_run(const pylom_batched_plan* plan, void* ws, double* S, int max_sweeps,
                                   void* stream);
/* Bind with per-item inputs (instead of pylom_svd_batched_bind): each item
 * f of the plan (N[f] x Nb[f]) is either a complex64 matrix (a SPOD bin,
 * exactly as pylom_svd_batched_bind takes it) or a real snapshot window
 * whose POD (Alg. 2 per window) runs in the same persistent launch: the
 * window's temporal mean removal (each point's mean over its Nb snapshots)
 * and sqrt(w) weights happen in the leaf load, the window then goes through
 * the same leaves, tree, Jacobi SVD and modes as the bins (complex
 * arithmetic on a zero imaginary part), and the real parts of its modes and
 * right vectors are returned.  Windows of different N and Nb (<= 128) and
 * SPOD bins may be mixed in one plan.  Not capturable (synchronises
 * `stream`); call once per set of buffers, then pylom_svd_batched_run. */
typedef struct {
  int xtype;          /* PYLOM_C64: a complex64 bin; PYLOM_F32 / PYLOM_F64: a real window */
  int remove_mean;    /* real windows: 1 = subtract each point's temporal mean */
  int mode_kind;      /* real windows: pylom_mode_kind (as pylom_pod) */
  int reserved;       /* 0 */
  const void* X;      /* device N x Nb input, column-major, ld ldx >= N; not modified */
  int64_t ldx;
  const double* w;    /* real windows: device N cell volumes (> 0), or NULL */
  double* mean;       /* real windows: device N means out, or NULL */
  void* U;            /* device N x min(kmodes, Nb) modes out, ld ldu >= N: complex64 for a bin; for a
                         real window binary32 with complex64 leaves (PYLOM_PREC_MIXED_3XTF32) or
                         binary64 with complex128 leaves (PYLOM_PREC_FP64) */
  int64_t ldu;
  double* VT;         /* real windows: device Nb x Nb right vectors out (row i = v_i^T, the sign rule
                         of pylom_pod; rows of an exactly zero singular value are zero), or NULL */
  int64_t ldvt;
} pylom_batched_item;
pylom_status pylom_svd_batched_bind_items(pylom_batched_plan* plan, const pylom_batched_item* items, void* ws,
                                          size_t ws_bytes, void* stream);
/* what: 0 leaf height, 1 leaf count, 2 offset of the bin's S, 3 grid size,
 * 4 number of leaf items; -1 on a bad argument. */
int64_t pylom_svd_batched_plan_info(const pylom_batched_plan* plan, int bin, int what);
void pylom_svd_batched_plan_destroy(pylom_batched_plan* plan);
/* Longest leaf a bin gets at precision prec (1024 rows for complex64
 * leaves, 512 for complex128): a leaf height hint above it is split into
 * more leaves.  -1 for a bad prec.  Host only. */
int64_t pylom_svd_batched_max_leaf_rows(int prec);

/* ------------------------------------------------------------------------
 * pylom_matmul -- local product of Alg. 4 (matmul_paral) on one device:
 * C = op(A) B, op(A) = A (m x k, lda >= m) or A^T (A stored k x m,
 * lda >= k); B k x n (ldb >= k); C m x n (ldc >= m).  binary64 on the FP64
 * tensor pipe, split along k with a fixed-order reduction (deterministic).
 * The all_reduce of Alg. 4 is the caller's (one device here).
 * ------------------------------------------------------------------------ */
size_t pylom_matmul_workspace_size(int64_t m, int64_t n, int64_t k);
pylom_status pylom_matmul(int transA, const double* A, const double* B, double* C,
                          int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb, int64_t ldc,
                          void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * pylom_svd_small_noalloc -- the SVD of pylom_svd_small for callers that
 * cannot give the library device memory (no counterpart in the paper).
 * A host code that owns all device buffers through its own allocator, or a
 * loop that may not allocate once running, passes only R and the outputs;
 * the scratch is a fixed array inside the library (about 1 MiB per device
 * that loads it, held until the process exits).  The binary64 sweeps start
 * from R^T: this entry point skips the binary32 preconditioning that
 * pylom_svd_small runs from M = 256 on (same SVD, more sweeps).
 *  R, U, S, VT, ldr, ldu, ldvt, max_sweeps   as pylom_svd_small.
 *  M      1 <= M <= 256; larger M returns PYLOM_ERR_SHAPE (use
 *         pylom_svd_small with a workspace).
 *  info   device int[2] or NULL: receives the device status (pylom_status)
 *         and the Jacobi sweeps used, stream-ordered after the SVD.
 * The first call on a device looks up the array's device address (once per
 * device); make it before any stream capture.  The address is kept for the
 * life of the process, so after cudaDeviceReset on a device this entry point
 * must not be called there again without reloading the library.  Devices
 * with an index of 64 or more return PYLOM_ERR_UNSUPPORTED.  All calls share
 * the array: calls that may overlap on the GPU race and must be ordered on
 * one stream.
 * ------------------------------------------------------------------------ */
pylom_status pylom_svd_small_noalloc(const double* R, int64_t M, int64_t ldr, double* U,
                                     int64_t ldu, double* S, double* VT, int64_t ldvt,
                                     int max_sweeps, int* info, void* stream);

/* ------------------------------------------------------------------------
 * pylom_wait_selftest -- runs one of the library's bounded device waits into
 * its time limit on purpose (failure detection; no counterpart in the
 * paper), so that the time-out path can be tested without hanging the GPU.
 * Every cooperative kernel of the library waits on other thread blocks only
 * through these two forms, each polling the GPU's global timer:
 *   kind 0  the grid barrier: `blocks` thread blocks (1..1024) arrive at a
 *           barrier that expects blocks + 1 arrivals, so nothing releases it;
 *           each block then enters a second barrier, which must return at
 *           once because the first one timed out;
 *   kind 1  the mbarrier wait of the tcgen05 commits: one block waits on an
 *           mbarrier that nothing arrives on (`blocks` is ignored).
 * Each wait gives up after limit_ms milliseconds (0 < limit_ms <= 2000; the
 * library's own kernels use 2000), records PYLOM_ERR_TIMEOUT in the
 * workspace header and returns, so the kernel ends and the context stays
 * usable.  gave_up: device unsigned or NULL, receives the number of blocks
 * whose waits gave up.  ws: >= pylom_wait_selftest_workspace_size() bytes,
 * 256-byte aligned; read the outcome with pylom_workspace_status
 * (PYLOM_ERR_TIMEOUT).  Asynchronous on `stream`.
 * ------------------------------------------------------------------------ */
size_t pylom_wait_selftest_workspace_size(void);
pylom_status pylom_wait_selftest(int kind, int blocks, double limit_ms, unsigned* gave_up, void* ws,
                                 size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Phase profiler (measurement support; no counterpart in the paper).
 * Between begin and end, each of the next max_calls pylom_pod calls records
 * CUDA events on its own stream at the boundaries of its phases:
 *   0 leaf Householder QR (the leaf kernel; it includes the tree merges
 *     when the leaves merge as they finish),
 *   1 cooperative tree reduction (zero when the leaves merged),
 *   2 small SVD (Jacobi + sort/sign/truncate),
 *   3 top-down pass of the tree,
 *   4 leaf modes product U = Q [B; 0].
 * pylom_profile_end synchronises on the recorded events and writes to HOST
 * memory the summed milliseconds per phase (phase_ms[PYLOM_PROFILE_PHASES])
 * and the number of calls recorded.  Host-global state: not thread-safe.
 * ------------------------------------------------------------------------ */
#define PYLOM_PROFILE_PHASES 5
pylom_status pylom_profile_begin(int max_calls);
pylom_status pylom_profile_end(double* phase_ms, int* calls);

#ifdef __cplusplus
}
#endif
#endif /* PYLOM_H */

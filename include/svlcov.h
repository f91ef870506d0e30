/*
 * svlcov.h -- C ABI of the GB300 library for updating a rank-k truncated SVD
 * of a sparse matrix with the SV-LCOV method ("Fast Updating Truncated SVD
 * for Representation Learning with Sparse Matrices", arXiv 2401.09703).
 *
 * Object maintained (Section 3.2, extended decomposition):
 *     A_k = U' U'' Sigma V''^T V'^T,   U = U' U'' and V = V' V'' orthonormal,
 * with U' (m x k) and V' (n x k) held in caller-owned device buffers in a
 * storage precision (FP64, FP32 or BF16), and U'', V'' (k x k) and Sigma kept
 * by the library in its workspace.  Each update returns the rank-k truncated
 * SVD of the modified A_k (Section 3.3, "maintaining an approximate rank-k
 * truncated SVD"; Theorem 1) in time proportional to the batch's nonzeros,
 * plus an O(m k^2) reset when a small factor becomes ill-conditioned.
 *
 * Conventions.
 *   - Every pointer argument named as "device" must point to GPU memory
 *     reachable from the current device; "host" pointers to host memory.
 *   - Dense factors are row-major: row i of U' is k contiguous elements.
 *   - A batch of s update vectors of length d is a CSR matrix with s rows
 *     and d columns: row j of the CSR is update vector j (for new columns
 *     E_c (m x s) the CSR holds E_c^T; for new rows E_r it holds E_r; for a
 *     weight update D E_m^T it holds D^T and E_m^T).  Column indices within a
 *     row need not be sorted; duplicates are rejected.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - Ownership: the caller owns every buffer it passes and keeps the factor
 *     buffers and the workspace alive until svlcov_destroy.  The library
 *     holds non-owning pointers and allocates no device memory.
 *
 * Errors.  Functions return SVLCOV_OK or a host-detected error synchronously
 * (argument, capacity or CUDA launch errors; nothing is enqueued then).
 * Errors found on the device (malformed CSR, non-finite values, ...) are
 * OR-ed into a status word in the workspace; every kernel of a step checks it
 * first, so a failed step and all later steps leave the factors unchanged
 * until svlcov_status() has reported and cleared the error.
 */
#ifndef SVLCOV_H
#define SVLCOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return and status codes ------------------------------------------- */
#define SVLCOV_OK 0
#define SVLCOV_ERR_INVALID_ARG 1 /* host: null pointer, bad shape, unsupported k or s */
#define SVLCOV_ERR_CAPACITY 2    /* host: would exceed max_m/max_n/max_s/max_nnz or the workspace */
#define SVLCOV_ERR_CUDA 3        /* host: a CUDA runtime call failed */
#define SVLCOV_ERR_STATE 4       /* host: the handle is not in the state the call needs */
/* device status bits (OR-ed), reported by svlcov_status */
#define SVLCOV_DEV_BAD_CSR 0x10   /* indptr not monotone/out of range, index out of range, duplicate */
#define SVLCOV_DEV_NONFINITE 0x20 /* NaN/Inf in batch values or in a small-step result */
#define SVLCOV_DEV_NOT_PD 0x40    /* residual Gram matrix E^T E - C^T C not finite */
#define SVLCOV_DEV_GAP_WARN 0x80  /* backward: a singular-value pair fell under the gap guard */
#define SVLCOV_DEV_TIMEOUT 0x100  /* a bounded device wait ran out */

/* storage precision of U' and V' (and of the factors read back) */
#define SVLCOV_FP64 0
#define SVLCOV_FP32 1
#define SVLCOV_BF16 2

/* precision of the small dense steps (Gram, CholeskyQR2, Rayleigh-Ritz SVD, folds) */
#define SVLCOV_SMALL_FP64 0  /* all small steps in native FP64 */
#define SVLCOV_SMALL_FP32 1  /* all small steps in FP32 (the plain FP32 path) */
#define SVLCOV_SMALL_MIXED 2 /* FP32 sweeps and factorizations with FP64 Gram/refinement */

#define SVLCOV_MAX_K 128
#define SVLCOV_MAX_S 1024

typedef struct svlcov_handle svlcov_handle;

/* A batch of update vectors in CSR form (all arrays on the device). */
typedef struct {
  int32_t rows;           /* s, number of update vectors (0 <= s <= max_s)      */
  int32_t cols;           /* d, length of each vector                           */
  int64_t nnz;            /* number of stored entries (= indptr[rows])          */
  const int32_t* indptr;  /* device, rows + 1 entries, indptr[0] = 0            */
  const int32_t* indices; /* device, nnz entries in [0, cols)                   */
  const void* values;     /* device, nnz entries of values_dtype                */
  int32_t values_dtype;   /* SVLCOV_FP64 or SVLCOV_FP32                         */
} svlcov_csr;

/* Everything svlcov_init needs. */
typedef struct {
  int64_t m, n;           /* current shape of A                                  */
  int32_t k;              /* rank, 1 <= k <= SVLCOV_MAX_K                        */
  int64_t max_m, max_n;   /* row capacity of ubuf / vbuf                         */
  int32_t max_s;          /* largest batch width, <= SVLCOV_MAX_S                */
  int64_t max_nnz;        /* largest nnz of one batch (per side)                 */
  int32_t storage;        /* SVLCOV_FP64 / FP32 / BF16 for U', V'                */
  int32_t small;          /* SVLCOV_SMALL_*                                      */
  const void* U0;         /* device, m x k row-major, init_dtype: starting U     */
  const double* sigma0;   /* device, k: starting singular values (descending)   */
  const void* V0;         /* device, n x k row-major, init_dtype: starting V     */
  int32_t init_dtype;     /* SVLCOV_FP64 or SVLCOV_FP32                          */
  void* ubuf;             /* device, max_m x k of storage dtype (U')            */
  void* vbuf;             /* device, max_n x k of storage dtype (V')            */
  void* workspace;        /* device, >= svlcov_workspace_bytes(desc) bytes,     */
  size_t workspace_bytes; /*   256-byte aligned                                  */
  double tau;             /* deflation threshold (<= 0: default for `small`)     */
  double reset_threshold; /* cond_1 bound on U'', V'' (<= 0: default for storage) */
  int32_t jacobi_block;   /* tile width of the Jacobi SVD: columns per block,   */
                          /*   1..16 (<= 0: 16); a tuning knob, see autotune    */
  int32_t reorth;         /* re-orthonormalise the projected factor X'W before  */
                          /*   every `reorth`-th step and at init (W <- W       */
                          /*   (W^T X'^T X' W)^-1/2); 0: default (every step    */
                          /*   for BF16 storage, else never); < 0: never.       */
                          /*   Needs small mode FP64 or MIXED.                  */
  int32_t gemm_split;     /* FP64 small products that would leave SMs idle     */
                          /*   split their K over thread-block clusters: 0     */
                          /*   default (on); < 0 never (for handles that run   */
                          /*   side by side, e.g. in svlcov_batch_run, where   */
                          /*   the GPU is full anyway).  Results depend on it  */
                          /*   (summation order), not on how a step is run.    */
  int32_t tensor_gemm;    /* SVLCOV_SMALL_MIXED: > 0 runs its FP64 small       */
                          /*   products (folds, C0, CholeskyQR2 Gram, SVD       */
                          /*   refinement) on the tensor cores as exact BF16    */
                          /*   digit products (Ozaki splitting, see            */
                          /*   svlcov_dgemm); 0 (default): in the update steps  */
                          /*   of FP32 / BF16 factors in double-float on the    */
                          /*   FP32 pipe (svlcov_dgemm engine 2, ~2^-44         */
                          /*   relative, far below those factors' rounding),    */
                          /*   else on the FP64 pipe; < 0: always on the FP64   */
                          /*   pipe.  Other modes: unused                       */
  int32_t s1_secular;     /* FP64 and MIXED small modes, steps of one vector   */
                          /*   (s = 1): SVD_k of K = [[Sigma, c], [0, rho]]     */
                          /*   from the secular equation of the rank-one change */
                          /*   K K^T = diag(Sigma^2, 0) + z z^T and Algorithm 2 */
                          /*   as one normalisation: 0 default (on), < 0 the    */
                          /*   general path (CholeskyQR2 and Jacobi)            */
  int32_t literal_steps;  /* SVLCOV_SMALL_MIXED, add-columns / add-rows steps   */
                          /*   of s > 1 vectors.  0 (default): the step forms   */
                          /*   no R.  Since K G = F Theta, the folds of         */
                          /*   Section 3.2 need only Sigma, G and Theta         */
                          /*   (F[:k] - C_Q F[k:] = Sigma G[:k] Theta^-1,       */
                          /*   R^-1 F[k:] = G[k:] Theta^-1), and K^T K =         */
                          /*   [[Sigma^2, Sigma C0], [C0^T Sigma, E^T E]]       */
                          /*   holds exactly (R^T R is the residual Gram), so   */
                          /*   SVD_k runs FP32 sweeps on K with one FP32        */
                          /*   Cholesky factor of the residual Gram in place of */
                          /*   R and refines on K^T K in FP64; the second       */
                          /*   CholeskyQR2 pass, R^-1 and C_Q are not formed.   */
                          /*   > 0: the literal Algorithm 2 / 3 / 11 route      */
                          /*   (R, X = R^-1, C_Q, K and F formed), which        */
                          /*   svlcov_add_cols_backward and the R / K / F       */
                          /*   intermediates need.  Other modes: unused         */
} svlcov_init_desc;

/* One item of a batched run: kind 0 = add columns (a), 1 = add rows (a),
 * 2 = update weights (a = D^T, b = E_m^T). */
typedef struct {
  int32_t kind;
  svlcov_csr a;
  svlcov_csr b;
} svlcov_op;

/* Size in bytes of the device workspace that `d` needs (host only, no CUDA
 * call).  Reads m, n, k, max_s, max_nnz, small; returns 0 on bad arguments. */
size_t svlcov_workspace_bytes(const svlcov_init_desc* d);

/* Create a handle from a starting rank-k SVD (Section 3.2: U' <- U, V' <- V,
 * U'' = V'' = I).  Copies U0 / V0 into ubuf / vbuf (converted to the storage
 * dtype) and sigma0 into the workspace, on `stream`.  *h receives a host
 * object freed by svlcov_destroy.  The first call on a device also selects
 * kernel attributes (no allocation). */
int svlcov_init(svlcov_handle** h, const svlcov_init_desc* d, void* stream);

/* Add columns: A <- [A  E_c] (Algorithm 3; Section 3.2 for the folds).
 * Ec_T: CSR with s rows (the new columns) of length m.  U' receives a sparse
 * addition on the rows the batch touches; s rows are appended to V'
 * (n <- n + s).  Host errors: INVALID_ARG (cols != m, s > max_s), CAPACITY
 * (n + s > max_n, nnz > max_nnz). */
int svlcov_add_cols(svlcov_handle* h, const svlcov_csr* Ec_T, void* stream);

/* Add rows: A <- [A ; E_r] (Algorithm 11).  Er: CSR with s rows of length n.
 * V' receives the sparse addition, s rows are appended to U' (m <- m + s).
 * Algorithm 11 is Algorithm 3 applied to A^T; the library runs the same
 * kernels with the roles of U and V exchanged. */
int svlcov_add_rows(svlcov_handle* h, const svlcov_csr* Er, void* stream);

/* Update weights: A <- A + D E_m^T (Algorithm 4).  D_T: CSR s x m (columns of
 * D), Em_T: CSR s x n (columns of E_m), same s.  U' and V' both receive
 * sparse additions; no rows are appended. */
int svlcov_update_weights(svlcov_handle* h, const svlcov_csr* D_T, const svlcov_csr* Em_T,
                          void* stream);

/* Materialise U = U' U'' (m x k), Sigma (k) and V = V' V'' (n x k) into
 * caller buffers (device; row-major; out_dtype SVLCOV_FP64 or FP32; any of
 * the three pointers may be NULL to skip it).  m and n are the current shape
 * (svlcov_get_shape). */
int svlcov_get_factors(svlcov_handle* h, void* U, double* sigma, void* V, int32_t out_dtype,
                       void* stream);

/* Query rows (Theorem 1, Query: U[i] = U'[i] U'' in O(k^2)).  side 0 = U,
 * 1 = V; idx: device, cnt row indices (must be < current m or n; rows out of
 * range are written as zeros and flag SVLCOV_DEV_BAD_CSR); out: device,
 * cnt x k row-major of out_dtype. */
int svlcov_query_rows(svlcov_handle* h, int32_t side, const int32_t* idx, int32_t cnt, void* out,
                      int32_t out_dtype, void* stream);

/* Current shape as the host sees it (m, n grow with every append). */
int svlcov_get_shape(const svlcov_handle* h, int64_t* m, int64_t* n, int32_t* k);

/* Synchronise `stream`, read and clear the device status word into
 * *device_code (0 = no error).  After an error the host shape is restored
 * from the device's committed counters. */
int svlcov_status(svlcov_handle* h, int32_t* device_code, void* stream);

/* Copy the small state (FP64, host buffers): Wu = U'' (k x k row-major),
 * Wv = V'' and sigma; any pointer may be NULL.  Synchronises `stream`.
 * Also returns the number of resets performed so far in *resets (may be
 * NULL). */
int svlcov_get_small_state(svlcov_handle* h, double* Wu, double* Wv, double* sigma,
                           int64_t* resets, void* stream);

/* Checkpoint support.  get_state copies U' (m x k), V' (n x k) in the storage
 * dtype and U'', V'', Sigma (FP64) to host buffers; set_state loads them back
 * (shape given by m, n; both synchronise `stream`).  Resuming from a state is
 * bit-identical to never having stopped. */
int svlcov_get_state(svlcov_handle* h, void* Up_host, void* Vp_host, double* Wu_host,
                     double* Wv_host, double* sigma_host, void* stream);
int svlcov_set_state(svlcov_handle* h, int64_t m, int64_t n, const void* Up_host,
                     const void* Vp_host, const double* Wu_host, const double* Wv_host,
                     const double* sigma_host, void* stream);

/* Intermediates of the last step, for per-kernel checks (FP64 host copies,
 * synchronises).  which: 0 = P = X'^T E (k x s), 1 = S_E = E^T E (s x s),
 * 2 = C0 (k x s), 3 = R (s x s), 4 = K ((k+s) x (k+s)), 5 = Theta (k),
 * 6 = F ((k+s) x k), 7 = G ((k+s) x k).  side selects D (0) or E (1) for a
 * weight update.  Column-major; *rows, *cols receive the shape.  Only after
 * an exact step (ERR_STATE after an approximate-space step). */
int svlcov_get_intermediate(svlcov_handle* h, int32_t which, int32_t side, double* host_out,
                            size_t capacity_doubles, int32_t* rows, int32_t* cols, void* stream);

/* ---- approximate augmented space (the -GKL and -RPI variants) -----------
 * Appendix "Approximating the Augmented Space" and the appendix algorithms
 * "Add columns / Update weights with approximated augmented space": instead
 * of an orthonormal basis of the whole residual (I - U U^T) E (Algorithm 2,
 * s vectors), an l-vector basis Q of a Golub-Kahan-Lanczos (Algorithm 9) or
 * randomized power-iteration (Algorithm 10) subspace of it is built in
 * SV-LCOV form, with P = Z^T Q; the step then takes SVD_k of
 * [[Sigma, U^T E], [0, P^T]] ((k+l) x (k+s)) and folds it as Algorithm 3
 * does.  Cost O(s^2 l + (k+l)^2 (k+s)) for the dense part instead of
 * O(s^3 + (k+s)^3); an approximation unless l >= rank of the residual.
 * Add rows is the same on A^T; update weights approximates both sides and
 * takes SVD_k of diag(Sigma, 0) + [U^T D; P_D^T][V^T E; P_E^T]^T. */
#define SVLCOV_APPROX_GKL 1
#define SVLCOV_APPROX_RPI 2
typedef struct {
  int32_t method;       /* SVLCOV_APPROX_GKL or SVLCOV_APPROX_RPI                         */
  int32_t l;            /* rank of the approximate space, 1 <= l <= s (the batch width)   */
  int32_t t;            /* RPI: power iterations (>= 1); ignored by GKL                   */
  const double* start;  /* device FP64: GKL's p_1 (s values; NULL = all ones) or RPI's    */
                        /*   starting matrix (s x l column-major, required); the same     */
                        /*   start serves both sides of a weight update                   */
  void* work;           /* device scratch of svlcov_approx_work_bytes(h, l) bytes,        */
                        /*   256-byte aligned                                             */
} svlcov_approx;
/* Scratch bytes for steps with rank l (0 on bad arguments; host only). */
size_t svlcov_approx_work_bytes(const svlcov_handle* h, int32_t l);
/* As svlcov_add_cols / svlcov_add_rows / svlcov_update_weights, with the
 * approximate space `a` (INVALID_ARG for a bad method, l or missing start or
 * work).  svlcov_add_cols_backward does not apply to these steps. */
int svlcov_add_cols_approx(svlcov_handle* h, const svlcov_csr* Ec_T, const svlcov_approx* a, void* stream);
int svlcov_add_rows_approx(svlcov_handle* h, const svlcov_csr* Er, const svlcov_approx* a, void* stream);
int svlcov_update_weights_approx(svlcov_handle* h, const svlcov_csr* D_T, const svlcov_csr* Em_T,
                                 const svlcov_approx* a, void* stream);

/* Backward of the last add-columns step (Algorithm 3; the fold of Section
 * 3.2): the gradient of a loss L(U_new[S], Theta) with respect to the stored
 * values of that step's batch E_c, from the intermediates the step left in
 * the workspace.  Valid only right after svlcov_add_cols on this handle (no
 * other call in between, ERR_STATE otherwise), with small mode FP64 or MIXED
 * (ERR_INVALID_ARG otherwise), for a batch with no empty or dependent update
 * vector (a deflated direction has no gradient).  The gradient is that of
 * the exact update, which does not depend on how the step stored its
 * factors.  All pointers device, FP64, row-major:
 *   E          the batch as passed to svlcov_add_cols
 *   rows_S     nS rows of U, strictly ascending (0 <= nS <= m)
 *   U_pre_S    nS x k, rows rows_S of the left factor BEFORE the step
 *   U_pre_nnz  nnz x k, the left-factor row (before the step) of each
 *              nonzero of E, in CSR order
 *   dL_dU_S    nS x k, dL/dU_new at rows rows_S
 *   dL_dtheta  k, dL/dTheta (may be NULL for zero)
 *   dL_dvalues nnz output, dL/de for each nonzero, in CSR order
 * gap: singular-value pairs (one of them kept) closer than gap * theta_1
 * are left out of the SVD adjoint, whose pair coefficient is
 * 1 / (theta_j^2 - theta_i^2), and raise SVLCOV_DEV_GAP_WARN in the status
 * word (<= 0 picks 1e-6; the leading singular values of sparse power-law
 * matrices lie ~1e-4 * theta_1 apart, and their pair terms are part of the
 * gradient).  work: device scratch of svlcov_add_cols_backward_work_bytes(h)
 * bytes.  Asynchronous on `stream`; the full SVD of K it needs runs in the
 * handle's small precision (FP64 sweeps, or FP32 sweeps + FP64 refinement).
 * Device-side problems set status bits as for a step; svlcov_set_state
 * invalidates the step's intermediates. */
size_t svlcov_add_cols_backward_work_bytes(const svlcov_handle* h);
int svlcov_add_cols_backward(svlcov_handle* h, const svlcov_csr* E, const int32_t* rows_S, int32_t nS,
                             const double* U_pre_S, const double* U_pre_nnz, const double* dL_dU_S,
                             const double* dL_dtheta, double* dL_dvalues, double gap, void* work,
                             void* stream);

/* Batched updates of many independent handles (configuration "many
 * matrices, uneven k, s and nnz").  Items are enqueued in order on
 * `concurrency` internal streams (1..64) forked from `stream` and joined back
 * into it; all items of one handle go to the same internal stream, so they
 * stay ordered, while different handles run concurrently.  Every handle
 * needs its own workspace.  The call only enqueues work; it can be captured
 * in a CUDA graph by capturing `stream`.  Each item is checked as by the
 * single-item calls; on the first host error nothing more is enqueued, the
 * streams are joined and the error is returned. */
int svlcov_batch_run(svlcov_handle** handles, const svlcov_op* ops, int32_t n_ops, int32_t concurrency,
                     void* stream);

/* Phase timing (the only tracing the library does).  When enabled, every
 * step records CUDA events on its stream around six phases: 0 validation and
 * grouping of the batch, 1 gather + Gram (turning into SV-LCOV form, Lemmas
 * 1-2), 2 CholeskyQR2 of the residual Gram (Algorithm 2), 3 the SVD_k of
 * the Rayleigh-Ritz matrix, 4 the small folds (Section 3.2), 5 the sparse
 * addition / append / reset / commit; a seventh entry, 6, times the Jacobi
 * sweep kernel alone (nested inside phase 3).  svlcov_profile_read
 * synchronises on the recorded events and returns accumulated milliseconds
 * and counts per phase (nphases <= 7); *svd_sweeps (may be NULL; synchronises the device)
 * receives the number of Jacobi sweeps summed over all SVD launches since the
 * last reset; reset != 0 clears the totals. */
int svlcov_profile_enable(svlcov_handle* h, int32_t enable);
int svlcov_profile_read(svlcov_handle* h, double* ms, int64_t* calls, int32_t nphases, int32_t reset,
                        int64_t* svd_sweeps);

/* Scores of index pairs for the downstream tasks (Section 4, task setup of
 * link prediction and collaborative filtering): out[p] = U[rows[p]]^T Sigma
 * V[cols[p]], entry (rows[p], cols[p]) of the maintained U Sigma V^T, and
 * with `symmetric` nonzero (undirected graph) the larger of that and
 * U[cols[p]]^T Sigma V[rows[p]].  Computed from the extended decomposition
 * as U'[i] M V'[j]^T with M = U'' diag(Sigma) V''^T, without materialising
 * U or V; arithmetic in FP32 for FP32 / BF16 storage, FP64 for FP64 storage.
 * rows, cols: device int32, npairs each; out: device FP64, npairs.  A pair
 * with an index out of range (rows[p] >= m or cols[p] >= n, both directions
 * for `symmetric`) scores NaN and sets SVLCOV_DEV_BAD_CSR in the status word.
 * Asynchronous on `stream`; uses the handle's step scratch, so it must not
 * overlap a step of the same handle. */
int svlcov_score_pairs(svlcov_handle* h, const int32_t* rows, const int32_t* cols, int64_t npairs, int32_t symmetric,
                       double* out, void* stream);

/* Projection of update vectors onto the current singular space without
 * updating it (Lemma 1, the gather that turns a batch into SV-LCOV form):
 * P = X'^T E^T and, if C0 is not NULL, C0 = X''^T P = X^T E^T, where side 0
 * takes X = U (E: s x m, each row an update vector over the m rows of A, as
 * for add_cols) and side 1 takes X = V (E: s x n, as for add_rows).  One
 * launch serves any number of vectors, e.g. the look-ahead projection of
 * many pending batches (X' changes between steps only at the rows a step
 * scatters to) or folding new users / items into the current
 * representation.  P, C0: device FP64, k x s column-major.  k must be a
 * multiple of 4 (SVLCOV_ERR_INVALID_ARG otherwise).  An index out of range
 * sets SVLCOV_DEV_BAD_CSR and is skipped.  Asynchronous on `stream`; C0 uses
 * the handle's step scratch for FP32 handles, so it must not overlap a step
 * of the same handle. */
int svlcov_project(svlcov_handle* h, int32_t side, const svlcov_csr* E, double* P, double* C0, void* stream);

/* Process-wide number of kernels this library has launched so far. */
uint64_t svlcov_kernel_launches(void);

/* Release the host object (device buffers stay with the caller). */
void svlcov_destroy(svlcov_handle* h);

/* Human-readable name of a return or status code. */
const char* svlcov_strerror(int32_t code);

/* ---- standalone dense kernels (same code as inside a step) -------------- */

/* C (M x N) = alpha op(A) op(B) + beta C in FP64, column-major (op = the
 * matrix or its transpose, ta / tb nonzero for the transpose; lda, ldb, ldc
 * leading dimensions), all pointers device memory; the small dense products
 * of a step (Section 3.2 folds, C0 = W^T P, CholeskyQR2, Rayleigh-Ritz
 * refinement).  engine 0: the FP64 pipe (tiled SIMT, split K over a
 * cluster for small products); engine 1: the tensor cores -- every row of
 * op(A) and column of op(B) is written on the grid of its largest exponent
 * and cut into eight 7-bit digits (Ozaki splitting, exact), the products of
 * the digit pairs with s + t < 8 are accumulated exactly by BF16
 * tcgen05.mma in FP32 tensor memory, and the groups are summed in FP64;
 * accurate to ~2^-52 of max_k |a_ik| max_k |b_kj| per term (FP64 GEMM
 * accuracy), subnormal inputs read as zero, a non-finite input gives NaN in
 * its row / column.  engine 2: double-float on the FP32 pipe -- each operand
 * split into FP32 hi + lo parts, the hi parts' products exact (product plus
 * FMA error), the cross terms to FP32 rounding, TwoSum accumulation; accurate
 * to a few 2^-44 of sum_k |a_ik b_kj| (the refinement products of steps whose
 * factors are stored in FP32 / BF16); operands must lie in FP32 range.
 * M, N, K <= 4096.  Asynchronous on `stream`; returns
 * SVLCOV_ERR_INVALID_ARG for bad sizes or pointers, SVLCOV_ERR_CUDA for a
 * launch error. */
int svlcov_dgemm(int32_t ta, int32_t tb, int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                 int32_t lda, const double* B, int32_t ldb, double beta, double* C, int32_t ldc, int32_t engine,
                 void* stream);

/* Rank-k SVD of a small dense matrix (the Rayleigh-Ritz step of Section 2.1,
 * SVD_k of K): one-sided Jacobi.  K: device, n x n column-major FP64 (not
 * modified).  F (n x k), theta (k), G (n x k): device FP64 outputs,
 * column-major, theta descending.  precision: SVLCOV_SMALL_FP64 (FP64
 * sweeps), SVLCOV_SMALL_FP32 (FP32 sweeps on K rounded to FP32) or
 * SVLCOV_SMALL_MIXED (FP32 sweeps, then one FP64 first-order refinement of
 * the leading k triplets built from GEMMs).  work: device scratch of
 * svlcov_small_svd_work_bytes(n) bytes.  Returns the number of
 * sweeps in *sweeps (host, may be NULL; synchronises when non-NULL). */
size_t svlcov_small_svd_work_bytes(int32_t n);
int svlcov_small_svd(const double* K, int32_t n, int32_t k, double* F, double* theta, double* G,
                     int32_t precision, void* work, int32_t* sweeps, void* stream);

/* SVD_k of the Rayleigh-Ritz matrix of a one-vector step (s = 1; Algorithms
 * 3 and 11): K = [[diag(sigma), c], [0, rho]], (k+1) x (k+1), k <=
 * SVLCOV_MAX_K, sigma descending and >= 0.  Since K K^T = diag(sigma^2, 0) +
 * z z^T with z = [c; rho], the values are the roots of the secular equation
 * of this rank-one change (one warp per root, FP64) and the vectors follow
 * from them in closed form with the z that the computed roots make exact
 * (Loewner), which keeps them orthogonal; deflation handles negligible z_i
 * and coinciding poles.  sigma, c (k), rho (1): device FP64.  F, G:
 * (k+1) x k column-major, theta (k) descending: device FP64 outputs.  work:
 * device scratch of svlcov_small_svd_arrow_work_bytes() bytes, 256-byte
 * aligned.  This is the kernel one-vector steps of the FP64 and mixed small
 * modes use (init option s1_secular).  Asynchronous on `stream`. */
size_t svlcov_small_svd_arrow_work_bytes(void);
int svlcov_small_svd_arrow(const double* sigma, const double* c, const double* rho, int32_t k, double* F,
                           double* theta, double* G, void* work, void* stream);

/* The same rank-k small SVD for callers that cannot allocate device memory
 * (for example code running under another component's caching allocator,
 * which owns the free device memory, or latency-sensitive code that must not
 * let cudaMalloc / cudaFree synchronise the device).  The paper has no
 * counterpart: this is a deployment variant of svlcov_small_svd, with the
 * same three precisions and the same results (SVLCOV_SMALL_MIXED included:
 * FP32 sweeps, then the FP64 refinement).  Its scratch is a fixed array of
 * 8 MiB compiled into the library (every GPU that loads the library holds
 * one until the process exits), so there is no `work` argument; the caller
 * still provides K, F, theta and G as for svlcov_small_svd.  n above
 * SVLCOV_SMALL_SVD_STATIC_MAX_N returns SVLCOV_ERR_CAPACITY before any CUDA
 * call; every n <= SVLCOV_SMALL_SVD_STATIC_MAX_N with any k <= n and any
 * precision fits.  The first call on each device looks up the array's
 * device address (a CUDA runtime query, no allocation); make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents: calls that overlap on the GPU race, so
 * serialise them.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Launch errors are reported as by svlcov_small_svd. */
#define SVLCOV_SMALL_SVD_STATIC_MAX_N 256
int svlcov_small_svd_static(const double* K, int32_t n, int32_t k, double* F, double* theta, double* G,
                            int32_t precision, int32_t* sweeps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SVLCOV_H */

// Kernel launchers of the SV-LCOV GB300 library (host-side declarations).
#pragma once
#include "common.cuh"

namespace svl {

constexpr int kChunk = 32;  // nonzeros per gather/Gram work item (one warp)

// Per-side scratch for one batch: CSR validation output, the hash-grouped
// column view (entries grouped by their index into U'/V'), and the chunked
// partial sums of the fused gather + Gram kernel.
struct SideScratch {
  int* rowid;      // [max_nnz]  batch row of each nonzero
  int* slot;       // [max_nnz]  hash slot of each nonzero
  int* rank_tmp;   // [max_nnz]
  int* tmp_j;      // [max_nnz]
  int* tmp_e;      // [max_nnz]
  int* seg_j;      // [max_nnz]  grouped view: batch row, sorted within a group
  double* seg_v;   // [max_nnz]  grouped view: value
  int* hkey;       // [Hmax]
  int* hcnt;       // [Hmax]
  int* hstart;     // [Hmax]
  int* occ;        // [Hmax]     occupied slots (distinct touched rows), count in counts[0]
  int* counts;     // [4]        0: occupied slots, 1: total chunks
  int* chunk_off;  // [max_s+1]
  int* chunk_row;  // [max_chunks]
  void* Ppart;     // [max_chunks * k] accumulator type
  double* SEpart;  // [max_chunks * max_s]
};

int64_t max_chunks(int64_t max_s, int64_t max_nnz);

// Process-wide count of kernels launched by the library (a diagnostic for
// benchmarks: how many of this library's kernels ran in a timed region).
void note_launches(int n);
uint64_t launches_total();

// ---- sparse side (templated on storage TS and small-step type TC) ----------
void launch_validate(const svlcov_csr& b, int64_t d, int* rowid, int* status, cudaStream_t st);
void launch_group(const svlcov_csr& b, int logH, const SideScratch& w, int* status, cudaStream_t st);
template <typename TS, typename TC>
void launch_gather_gram(const svlcov_csr& b, const TS* Xp, int k, const TC* W, const SideScratch& w,
                        TC* P, TC* SE, TC* C0, TC* e2, int* status, cudaStream_t st);
template <typename TS, typename TC>
void launch_scatter(TS* Xp, int k, const TC* Mt, int64_t nnz, const SideScratch& w, const int* status,
                    cudaStream_t st);
template <typename TS, typename TC>
void launch_append(TS* Xp, int64_t row0, int k, int s, const TC* Nt, const int* status, cudaStream_t st);
template <typename TS, typename TC>
void launch_reset(TS* Xp, int64_t rows, int k, const TC* Wn, const int* do_reset, const int* status,
                  cudaStream_t st);
template <typename TS, typename TC>
void launch_materialize(const TS* Xp, int64_t rows, int64_t src_rows, int k, const TC* W, void* out,
                        int out_dtype, const int32_t* idx, cudaStream_t st, int* status);
template <typename TS>
void launch_convert_in(const void* src, int src_dtype, TS* dst, int64_t count, cudaStream_t st);

// ---- dense small steps (templated on TC) -----------------------------------
// tri (optional): 1 op(A) upper, 2 op(A) lower, 4 op(B) upper, 8 op(B) lower triangular
template <typename T>
void gemm(bool ta, bool tb, int M, int N, int Kd, T alpha, const T* A, int lda, const T* B, int ldb,
          T beta, T* C, int ldc, const int* status, cudaStream_t st, int tri = 0);
enum { TRI_A_UP = 1, TRI_A_LO = 2, TRI_B_UP = 4, TRI_B_LO = 8 };
// The FP64 product in double-float arithmetic on the FP32 pipe (operands
// split into FP32 hi + lo, exact hi products, TwoSum accumulation): a few
// 2^-44 of sum_k |a_ik b_kj|, for the refinement of FP32 / BF16 factors.
void gemm_df(bool ta, bool tb, int M, int N, int Kd, double alpha, const double* A, int lda, const double* B, int ldb,
             double beta, double* C, int ldc, const int* status, cudaStream_t st, int tri = 0);
// Route this host thread's FP64 gemm calls to gemm_df (update steps of
// mixed-mode handles with FP32 / BF16 factors): 0 never, 1 products of 2^21
// multiply-adds and more, 2 all.
void set_gemm_df(int mode);
// The same FP64 product on the tensor cores: operands split into 7-bit BF16
// digits (Ozaki), exact digit-pair products accumulated in FP32 tensor
// memory by tcgen05.mma, summed in FP64 (csrc/tcgemm.cu).
void ozaki_gemm(bool ta, bool tb, int M, int N, int Kd, double alpha, const double* A, int lda, const double* B,
                int ldb, double beta, double* C, int ldc, const int* status, cudaStream_t st, int tri = 0);
// Whether this host thread's FP64 gemm() calls run as ozaki_gemm (set for the
// steps of mixed-mode handles whose tensor_gemm option is on).
void set_gemm_tc(bool on);
bool gemm_tc();
struct GemmTcScope {
  bool prev;
  explicit GemmTcScope(bool on) : prev(gemm_tc()) { set_gemm_tc(on); }
  ~GemmTcScope() { set_gemm_tc(prev); }
};
size_t cholinv_smem_bytes(int s, size_t elem);
// Cholesky with deflation S = L L^T and Y = L^-1 (dropped rows and columns
// zeroed), factor arithmetic in T on SrcT data: one CTA in shared memory when
// the packed triangle fits, else blocked with GEMM panels and trailing
// updates, using the scratch Awork and Twork (s x s each).  DELTA: S = I + A
// with small A (the second CholeskyQR pass), factored in the delta form.
// factor_only: L alone (Y not formed; where one CTA holds the triangle, only
// the lower triangle of L is written).
template <typename T, typename SrcT, bool DELTA>
void launch_cholinv(const SrcT* S, int s, const SrcT* ref, T tau, SrcT* L, SrcT* Y, unsigned char* defl,
                    SrcT* Awork, SrcT* Twork, int* status, cudaStream_t st, bool factor_only = false);
template <typename T>
void launch_build_K_add(const T* sigma, const T* C0, const T* R, int k, int s, T* K, const int* status,
                        cudaStream_t st);
template <typename T>
void launch_build_L(const T* C0, const T* R, int k, int s, T* L, const int* status, cudaStream_t st);
template <typename T>
void launch_add_diag(T* K, int n, const T* sigma, int k, const int* status, cudaStream_t st);
size_t jacobi_work_bytes(int n);
// FP32 sweeps by the Gram-form cluster kernel where it fits (default on).
void set_jacobi_gram(bool on);
int* jacobi_sweeps_ptr(void* work, int n, int elem);
size_t refine_work_bytes(int n, int k);
// Mixed SVD_k from FP32 sweeps on Kc and FP64 steps on M = K^T K (theta, G only).
int launch_mixed_svd_gram(const double* Kc, const double* M, int n, int k, double* theta, double* G, void* jwork,
                          void* rwork, int* status, cudaStream_t st, int64_t* sweep_total, int bcap,
                          const int* n_active, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join,
                          int iters, double stop_tol);
void launch_build_K_chol(const double* sigma, const double* C0, const double* L, int k, int s, const int* perm,
                         double* Kp, const int* status, cudaStream_t st);
void launch_build_M(const double* sigma, const double* C0, const double* SE, int k, int s, const int* perm,
                    double* Mp, const int* status, cudaStream_t st);
void launch_rfree_fold_inputs(const double* sigma, const double* G, const double* theta, int k, int s, double* T,
                              double* Y, const int* status, cudaStream_t st);
// n_active (optional, device): columns >= *n_active of K are zero; the
// cluster form of the Jacobi then plays its tournament over the blocks
// holding the active columns only.
int launch_mixed_svd(const double* K, int n, int k, double* F, double* theta, double* G, void* jwork, void* rwork,
                     int* status, cudaStream_t st, int64_t* sweep_total, int bcap = 0,
                     const int* n_active = nullptr, cudaStream_t side = nullptr, cudaEvent_t ev_fork = nullptr,
                     cudaEvent_t ev_join = nullptr);
// Whether this host thread's FP64 products may split K over clusters (off
// while svlcov_batch_run enqueues concurrent handles).
void set_gemm_split(bool on);
// Events the next Jacobi launches of this host thread record around their
// sweep kernel (phase timing; nullptr: none).
void set_jacobi_events(cudaEvent_t before, cudaEvent_t after);
template <typename T>
int launch_jacobi(const T* K, int n, int k, T* F, T* theta, T* G, void* work, int* status, cudaStream_t st,
                  int64_t* sweep_total = nullptr, int bcap = 0, const int* n_active = nullptr,
                  double stop_tol = 0.0);
// Empty update vectors to the end: perm (s) lists the non-empty batch
// vectors first; *n_active = k + their number (device).
void launch_active_columns(const int32_t* indptr, int s, int k, int* perm, int* n_active, const int* status,
                           cudaStream_t st);
template <typename T>
void launch_permute_cols(const T* K, int n, int k, const int* perm, T* Kp, const int* status, cudaStream_t st);
template <typename T>
void launch_unpermute_rows(const T* Gp, int n, int k, int cols, const int* perm, T* G, const int* status,
                           cudaStream_t st);
// Guarded k x k inverse (Winv = I and *do_reset = 1 when W is singular or
// cond_1(W) > thr).  tmp (2 k^2, may be NULL): scratch of the FP32 +
// Newton form used for FP64 W when thr <= 1e3.
template <typename T>
void launch_inverse(const T* W, int k, T* Winv, double thr, int* do_reset, int* status, cudaStream_t st,
                    T* tmp = nullptr, int newton = 2);
template <typename T>
void launch_copy(const T* src, T* dst, int64_t count, const int* status, cudaStream_t st);
void launch_triu(double* A, int n, const int* status, cudaStream_t st);
template <typename T>
void launch_commit(T* Wu, const T* Wu_new, const int* reset_u, T* Wv, const T* Wv_new, const int* reset_v,
                   T* sigma, const T* theta, int k, int64_t* counters, int64_t dm, int64_t dn,
                   int64_t* resets, int* status, cudaStream_t st);
template <typename T>
void launch_check_finite(const T* x, int64_t count, int* status, cudaStream_t st);
template <typename A, typename B>
void launch_cast(const A* src, B* dst, int64_t count, cudaStream_t st);
template <typename T>
void launch_copy2d(const T* src, int lds, T* dst, int ldd, int rows, int cols, const int* status, cudaStream_t st);
template <typename T>
void launch_set_identity(T* W, int k, cudaStream_t st);
template <typename T> struct FiniteSet {
  const T* ptr[6];
  int64_t count[6];
  int n;
};
template <typename T>
void launch_check_finite_multi(const FiniteSet<T>& set, int* status, cudaStream_t st);

// ---- re-orthonormalisation of a low-precision factor X'W ---------------------
size_t reorth_work_bytes(int k, int64_t max_rows);
template <typename TS>
void launch_reorth(const TS* Xp, int64_t rows, int k, double* W, void* work, int* status, cudaStream_t st);

// ---- approximate augmented space (-GKL / -RPI variants) ----------------------
// GKL: l Lanczos steps on the residual Gram S (s x s) from p1 (NULL: all
// ones); outputs W (s x l) coefficients of Q, P (s x l) = Z^T Q.  Scratch: Pm
// (s x (l+1)), wr, u (s), ab (2l + 2).
template <typename T>
void launch_gkl(const T* S, int s, int l, const T* p1, T* Pm, T* W, T* wr, T* u, T* ab, T* P, const int* status,
                cudaStream_t st);
template <typename T>
void launch_mgs_cols(T* P, int s, int l, const int* status, cudaStream_t st);
template <typename T>
void launch_diag_quad(const T* W, const T* TM, int s, int l, T* e2, const int* status, cudaStream_t st);
template <typename T>
void launch_build_K_rect(const T* sigma, const T* C0, const T* P, int k, int s, int l, T* K, const int* status,
                         cudaStream_t st);
template <typename T>
void launch_build_L_rect(const T* C0, const T* P, int k, int s, int l, T* L, const int* status, cudaStream_t st);
template <typename T>
void launch_scale_cols(T* G, int rows, int ld, int k, const T* theta, const int* status, cudaStream_t st);

// ---- backward of one add-columns step (FP64 small state) -------------------
// Intermediates the forward step left in the workspace (column-major, FP64).
struct BackwardInputs {
  const double *C0, *R, *X, *CQ, *Y;        // k x s, s x s, s x s, k x s, s x k
  const double *K, *F, *G, *theta;          // (k+s)^2, (k+s) x k, (k+s) x k, k
  const int *rowid, *slot, *hstart, *hcnt;  // CSR row of each nonzero; grouped view
  const int* seg_j;
  const double* seg_v;
  void* jwork;                              // Jacobi scratch for k + s
  bool mixed;                               // full SVD of K: FP32 sweeps + FP64 refinement, else FP64 sweeps
};
size_t backward_work_bytes(int n, int k, int s, int64_t nnz);
int launch_add_cols_backward(const svlcov_csr& E, int k, const BackwardInputs& in, const int32_t* S, int nS,
                             const double* Upre_S, const double* Upre_nnz, const double* Ubar, const double* thbar,
                             double* dvalues, double gap, void* work, int* status, cudaStream_t st);

// SVD_k of K = [[diag(sigma), c], [0, rho]] (a one-vector step) through the
// secular equation of K K^T = diag(sigma^2, 0) + z z^T (csrc/arrow.cu).
size_t arrow_work_bytes();
void launch_arrow_svd(const double* sigma, const double* c, const double* rho, int k, double* F, double* theta,
                      double* G, void* work, const int* status, cudaStream_t st);
// Algorithm 2 for one vector: R = sqrt(S) unless S <= tau e2 (deflated: R = X
// = 0), X = 1 / R, C_Q = C0 X.
void launch_s1_orth(const double* S, const double* e2, const double* C0, int k, double tau, double* R, double* X,
                    double* CQ, unsigned char* defl1, unsigned char* defl2, int* status, cudaStream_t st);

// Scores U'[i] M V'[j]^T (M = W_U diag(sigma) W_V^T) of index pairs, the
// larger of both directions when `symmetric` (csrc/score.cu).
template <typename TS, typename TC>
void launch_score_pairs(const TS* Up, const TS* Vp, int64_t m, int64_t n, int k, const TC* Wu, const TC* Wv,
                        const TC* sigma, const int32_t* rows, const int32_t* cols, int64_t npairs, int symmetric,
                        double* out, double* Mwork, int* status, cudaStream_t st);

// P (k x s, column-major) = X'^T E^T for a batch E (s x rows), one warp per
// update vector (csrc/project.cu); k a multiple of 4.
template <typename TS, typename TP>
void launch_project(const svlcov_csr& b, const TS* Xp, int64_t rows, int k, TP* P, int* status, cudaStream_t st);

// out = X' W on the tensor cores (BF16 pieces, FP32 accumulation) for BF16 /
// FP32 storage with k a multiple of 16 up to 128 (csrc/tcrowmul.cu); out may
// be X' (the reset of the extended decomposition).
bool rowmul_tc_ok(int storage_bytes, int k);
template <typename TS, typename TC, typename TO>
void launch_rowmul_tc(const TS* X, int64_t rows, int k, const TC* W, TO* out, const int* do_reset, const int* status,
                      cudaStream_t st);

// Return code of an entry point after its launches: SVLCOV_ERR_CUDA if a
// launch error is pending on this host thread (cudaGetLastError, which also
// clears it), else SVLCOV_OK.
inline int last_launch() { return cudaGetLastError() == cudaSuccess ? SVLCOV_OK : SVLCOV_ERR_CUDA; }

}  // namespace svl

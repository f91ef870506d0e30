// Backward of one add-columns step (Algorithm 3): gradient of a loss of the
// updated left vectors U_new (rows S) and singular values Theta with respect
// to the stored values of the batch E_c, from the intermediates the forward
// step left in the workspace.
//
// Forward (Algorithm 3 in the CholeskyQR2 form of this library):
//   C0 = U^T E,  S = E^T E - C0^T C0 = R^T R,  X = R^-1,  C_Q = C0 X,
//   K = [[Sigma, C0], [0, R]] = F Theta G^T (square SVD, first k kept),
//   U_new = U X_u + E Y  with  X_u = F[:k] - C_Q F[k:],  Y = X F[k:].
// Reverse, given U_bar (rows S of dL/dU_new) and Theta_bar:
//   X_u_bar = U[S]^T U_bar,  Y_bar = E[S,:]^T U_bar,
//   F_bar[:k] = X_u_bar,  F_bar[k:] = -C_Q^T X_u_bar + X^T Y_bar,
//   C_Q_bar = -X_u_bar F[k:]^T,  R_bar = -X^T Y_bar Y^T - C_Q^T C_Q_bar X^T,
//   C0_bar = C_Q_bar X^T,
//   square-SVD adjoint: K_bar = F (Theta_bar + (Fm o (F^T F_bar - F_bar^T F)) Theta) G^T,
//     Fm_ij = 1 / (theta_j^2 - theta_i^2), zeroed for pairs with |theta_i - theta_j|
//     below gap * theta_1 that involve a kept index (flags SVLCOV_DEV_GAP_WARN),
//   C0_bar += K_bar[:k, k:],  R_bar += triu(K_bar[k:, k:]),
//   Cholesky adjoint (S = L L^T, L = R^T): S_bar = sym(X Phi(R triu(R_bar)^T) X^T),
//     Phi = lower triangle with halved diagonal,
//   C0_bar -= 2 C0 S_bar,
//   dL/de_ij = 2 (E S_bar)_ij + (U C0_bar)_ij + (U_bar Y^T)_ij   (i in S for the last).
#include <algorithm>

#include "kernels.cuh"

namespace svl {

__global__ void k_bw_pos(const int32_t* __restrict__ indices, int64_t nnz, const int32_t* __restrict__ S, int nS,
                         int* __restrict__ pos, const int* status) {
  if (failed(status)) return;
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  int i = indices[e];
  int lo = 0, hi = nS - 1, p = -1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = S[mid];
    if (v == i) { p = mid; break; }
    if (v < i) lo = mid + 1;
    else hi = mid - 1;
  }
  pos[e] = p;
}

// Y_bar[j, :] = sum over the nonzeros (i, j) with i in S of e_ij U_bar[pos(i), :]
__global__ void k_bw_ybar(const int32_t* __restrict__ indptr, const void* __restrict__ values, int vdtype, int s,
                          int k, const int* __restrict__ pos, const double* __restrict__ Ubar,
                          double* __restrict__ Ybar, const int* status) {
  if (failed(status)) return;
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= s) return;
  for (int c = lane; c < k; c += 32) {
    double acc = 0.0;
    for (int64_t e = indptr[j]; e < indptr[j + 1]; ++e) {
      int p = pos[e];
      if (p >= 0) acc += load_val<double>(values, vdtype, e) * Ubar[(int64_t)p * k + c];
    }
    Ybar[j + (int64_t)c * s] = acc;
  }
}

// Inner = diag(Theta_bar) + (Fm o M) Theta with M = A1-part antisymmetrised:
// M_ij = [j<k] A1[i,j] - [i<k] A1[j,i]  (A1 = F^T F_bar, n x k).
__global__ void k_bw_svd_inner(const double* __restrict__ A1, const double* __restrict__ th, const double* thbar,
                               int n, int k, double gap, double* __restrict__ Inner, int* warn, const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t % n), j = (int)(t / n);
  double v = 0.0;
  if (i == j) {
    v = (i < k && thbar) ? thbar[i] : 0.0;
  } else if (i < k || j < k) {
    double m = (j < k ? A1[i + (int64_t)j * n] : 0.0) - (i < k ? A1[j + (int64_t)i * n] : 0.0);
    double ti = th[i], tj = th[j];
    if (fabs(ti - tj) < gap * th[0]) {
      if (m != 0.0) atomicOr(warn, SVLCOV_DEV_GAP_WARN);
    } else {
      v = m * tj / (tj * tj - ti * ti);
    }
  }
  Inner[t] = v;
}

// C0_bar += K_bar[:k, k:],  R_bar = triu(R_bar + K_bar[k:, k:])
__global__ void k_bw_blocks(const double* __restrict__ Kbar, int n, int k, int s, double* __restrict__ C0bar,
                            double* __restrict__ Rbar, const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)k * s) {
    int a = (int)(t % k), j = (int)(t / k);
    C0bar[t] += Kbar[a + (int64_t)(k + j) * n];
  }
  if (t < (int64_t)s * s) {
    int i = (int)(t % s), j = (int)(t / s);
    Rbar[t] = i <= j ? Rbar[t] + Kbar[(k + i) + (int64_t)(k + j) * n] : 0.0;
  }
}

// The gap warning is kept apart while the backward runs (a set status word
// stops every later kernel) and reported at the end.
__global__ void k_bw_finish(const int* warn, int* status) {
  if (*warn) flag(status, *warn);
}

// P = Phi(T): lower triangle, diagonal halved
__global__ void k_bw_phi(const double* __restrict__ T, int s, double* __restrict__ P, const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)s * s) return;
  int i = (int)(t % s), j = (int)(t / s);
  P[t] = i > j ? T[t] : (i == j ? 0.5 * T[t] : 0.0);
}

__global__ void k_bw_sym(const double* __restrict__ A, int s, double* __restrict__ B, const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)s * s) return;
  int i = (int)(t % s), j = (int)(t / s);
  B[t] = 0.5 * (A[t] + A[j + (int64_t)i * s]);
}

// dL/de for every nonzero (one warp each)
__global__ void k_bw_ebar(const int32_t* __restrict__ rowid, int64_t nnz, int s, int k, const int* __restrict__ slot,
                          const int* __restrict__ hstart, const int* __restrict__ hcnt, const int* __restrict__ seg_j,
                          const double* __restrict__ seg_v, const double* __restrict__ Sbar,
                          const double* __restrict__ Upre_nnz, const double* __restrict__ C0bar,
                          const int* __restrict__ pos, const double* __restrict__ Ubar, const double* __restrict__ Y,
                          double* __restrict__ out, const int* status) {
  if (failed(status)) return;
  int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (e >= nnz) return;
  int j = rowid[e];
  int h = slot[e];
  double acc = 0.0;
  for (int q = hstart[h] + lane; q < hstart[h] + hcnt[h]; q += 32) acc += 2.0 * seg_v[q] * Sbar[seg_j[q] + (int64_t)j * s];
  for (int c = lane; c < k; c += 32) acc += Upre_nnz[e * k + c] * C0bar[c + (int64_t)j * k];
  int p = pos[e];
  if (p >= 0)
    for (int c = lane; c < k; c += 32) acc += Ubar[(int64_t)p * k + c] * Y[j + (int64_t)c * s];
  acc = warp_sum(acc);
  if (lane == 0) out[e] = acc;
}

struct BwBufs {
  double *Ff, *Gf, *thf, *Kbar, *T5, *Inner, *A1, *Fbar, *Xbar, *Ybar, *CQbar, *C0bar, *Rbar, *T1, *T2, *T3, *P,
      *T4, *Sbar;
  int *pos, *warn;
  void* rwork;
};

static BwBufs bw_layout(void* base, int n, int k, int s, int64_t nnz, size_t* total) {
  BwBufs b{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base ? (char*)base + off : nullptr;
    off += bytes;
    return p;
  };
  size_t n2 = (size_t)n * n, ss = (size_t)s * s;
  b.Ff = (double*)take(8 * n2);
  b.Gf = (double*)take(8 * n2);
  b.thf = (double*)take(8 * (size_t)n);
  b.Kbar = (double*)take(8 * n2);
  b.T5 = (double*)take(8 * n2);
  b.Inner = (double*)take(8 * n2);
  b.A1 = (double*)take(8 * (size_t)n * k);
  b.Fbar = (double*)take(8 * (size_t)n * k);
  b.Xbar = (double*)take(8 * (size_t)k * k);
  b.Ybar = (double*)take(8 * (size_t)s * k);
  b.CQbar = (double*)take(8 * (size_t)k * s);
  b.C0bar = (double*)take(8 * (size_t)k * s);
  b.Rbar = (double*)take(8 * ss);
  b.T1 = (double*)take(8 * (size_t)s * k);
  b.T2 = (double*)take(8 * ss);
  b.T3 = (double*)take(8 * ss);
  b.P = (double*)take(8 * ss);
  b.T4 = (double*)take(8 * ss);
  b.Sbar = (double*)take(8 * ss);
  b.pos = (int*)take(4 * (size_t)std::max<int64_t>(nnz, 1));
  b.warn = (int*)take(4);
  b.rwork = take(refine_work_bytes(n, n));
  *total = (off + 255) & ~(size_t)255;
  return b;
}

size_t backward_work_bytes(int n, int k, int s, int64_t nnz) {
  size_t total = 0;
  bw_layout(nullptr, n, k, s, nnz, &total);
  return total;
}

int launch_add_cols_backward(const svlcov_csr& E, int k, const BackwardInputs& in, const int32_t* S, int nS,
                             const double* Upre_S, const double* Upre_nnz, const double* Ubar, const double* thbar,
                             double* dvalues, double gap, void* work, int* status, cudaStream_t st) {
  const int s = E.rows, n = k + s;
  const int64_t nnz = E.nnz;
  size_t total = 0;
  BwBufs b = bw_layout(work, n, k, s, nnz, &total);
  const int TB = 256;
  if (cudaMemsetAsync(b.warn, 0, sizeof(int), st) != cudaSuccess) return SVLCOV_ERR_CUDA;
  // positions of the nonzeros' rows in S, and Y_bar
  if (nnz > 0) {
    note_launches(1);
    k_bw_pos<<<(int)cdiv(nnz, TB), TB, 0, st>>>(E.indices, nnz, S, nS, b.pos, status);
  }
  note_launches(1);
  k_bw_ybar<<<(int)cdiv(s, 8), 256, 0, st>>>(E.indptr, E.values, E.values_dtype, s, k, b.pos, Ubar, b.Ybar, status);
  // X_u_bar = U[S]^T U_bar  (row-major nS x k buffers are column-major k x nS)
  gemm<double>(false, true, k, k, nS, 1.0, Upre_S, k, Ubar, k, 0.0, b.Xbar, k, status, st);
  // F_bar
  launch_copy2d<double>(b.Xbar, k, b.Fbar, n, k, k, status, st);
  gemm<double>(true, false, s, k, k, -1.0, in.CQ, k, b.Xbar, k, 0.0, b.Fbar + k, n, status, st);
  gemm<double>(true, false, s, k, s, 1.0, in.X, s, b.Ybar, s, 1.0, b.Fbar + k, n, status, st);
  // C_Q_bar, R_bar, C0_bar from the folds
  gemm<double>(false, true, k, s, k, -1.0, b.Xbar, k, in.F + k, n, 0.0, b.CQbar, k, status, st);
  gemm<double>(true, false, s, k, s, 1.0, in.X, s, b.Ybar, s, 0.0, b.T1, s, status, st);           // X^T Y_bar
  gemm<double>(false, true, s, s, k, -1.0, b.T1, s, in.Y, s, 0.0, b.Rbar, s, status, st);          // -X^T Y_bar Y^T
  gemm<double>(true, false, s, s, k, 1.0, in.CQ, k, b.CQbar, k, 0.0, b.T2, s, status, st);         // C_Q^T C_Q_bar
  gemm<double>(false, true, s, s, s, -1.0, b.T2, s, in.X, s, 1.0, b.Rbar, s, status, st);          // - ... X^T
  gemm<double>(false, true, k, s, s, 1.0, b.CQbar, k, in.X, s, 0.0, b.C0bar, k, status, st);       // C_Q_bar X^T
  // full SVD of K (all n triplets), with the forward's own leading k triplets
  int e = in.mixed ? launch_mixed_svd(in.K, n, n, b.Ff, b.thf, b.Gf, in.jwork, b.rwork, status, st, nullptr)
                   : launch_jacobi<double>(in.K, n, n, b.Ff, b.thf, b.Gf, in.jwork, status, st);
  if (e) return SVLCOV_ERR_CUDA;
  launch_copy2d<double>(in.F, n, b.Ff, n, n, k, status, st);
  launch_copy2d<double>(in.G, n, b.Gf, n, n, k, status, st);
  launch_copy<double>(in.theta, b.thf, k, status, st);
  // square-SVD adjoint
  gemm<double>(true, false, n, k, n, 1.0, b.Ff, n, b.Fbar, n, 0.0, b.A1, n, status, st);           // F^T F_bar
  note_launches(1);
  k_bw_svd_inner<<<(int)cdiv((int64_t)n * n, TB), TB, 0, st>>>(b.A1, b.thf, thbar, n, k, gap, b.Inner, b.warn, status);
  gemm<double>(false, false, n, n, n, 1.0, b.Ff, n, b.Inner, n, 0.0, b.T5, n, status, st);
  gemm<double>(false, true, n, n, n, 1.0, b.T5, n, b.Gf, n, 0.0, b.Kbar, n, status, st);
  note_launches(1);
  k_bw_blocks<<<(int)cdiv((int64_t)std::max(k, s) * s, TB), TB, 0, st>>>(b.Kbar, n, k, s, b.C0bar, b.Rbar, status);
  // Cholesky adjoint: S_bar = sym(X Phi(R triu(R_bar)^T) X^T)
  gemm<double>(false, true, s, s, s, 1.0, in.R, s, b.Rbar, s, 0.0, b.T3, s, status, st, TRI_A_UP | TRI_B_LO);
  note_launches(1);
  k_bw_phi<<<(int)cdiv((int64_t)s * s, TB), TB, 0, st>>>(b.T3, s, b.P, status);
  gemm<double>(false, false, s, s, s, 1.0, in.X, s, b.P, s, 0.0, b.T4, s, status, st, TRI_A_UP | TRI_B_LO);
  gemm<double>(false, true, s, s, s, 1.0, b.T4, s, in.X, s, 0.0, b.T2, s, status, st, TRI_B_LO);
  note_launches(1);
  k_bw_sym<<<(int)cdiv((int64_t)s * s, TB), TB, 0, st>>>(b.T2, s, b.Sbar, status);
  gemm<double>(false, false, k, s, s, -2.0, in.C0, k, b.Sbar, s, 1.0, b.C0bar, k, status, st);    // -2 C0 S_bar
  if (nnz > 0) {
    note_launches(1);
    k_bw_ebar<<<(int)cdiv(nnz * 32, TB), TB, 0, st>>>(in.rowid, nnz, s, k, in.slot, in.hstart, in.hcnt, in.seg_j,
                                                      in.seg_v, b.Sbar, Upre_nnz, b.C0bar, b.pos, Ubar, in.Y,
                                                      dvalues, status);
  }
  note_launches(1);
  k_bw_finish<<<1, 1, 0, st>>>(b.warn, status);
  return cudaGetLastError() == cudaSuccess ? 0 : SVLCOV_ERR_CUDA;
}

}  // namespace svl

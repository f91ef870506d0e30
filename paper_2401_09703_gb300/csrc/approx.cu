// Approximate augmented space (the -GKL and -RPI variants, Appendix
// "Approximating the Augmented Space"): an l-vector basis Q = E W - U (C0 W)
// of a Krylov (Golub-Kahan-Lanczos, Algorithm 9) or power-iteration (RPI,
// Algorithm 10) subspace of the residual Z = (I - U U^T) E, with
// P = Z^T Q (s x l).  In SV-LCOV form every operation of both algorithms
// acts on s-vectors through the residual Gram S = E^T E - C0^T C0 (Lemma 2):
//   GKL:  b'_i = E w_i, c'_i = C0 w_i,  alpha_i^2 = w_i^T S w_i,
//         p_{i+1} = S w_i - alpha_i p_i  (w_i normalised),
//   RPI:  the SV-LCOV QR of (E W, C0 W) is the Cholesky factor of W^T S W,
//         and P = B0^T B' - C0^T C' = S W.
// So the basis costs O(s^2 l) on the s x s Gram the step has already formed,
// instead of the O(s^3) CholeskyQR2 of the full residual.
#include <algorithm>

#include "kernels.cuh"

namespace svl {

// y = S x for a symmetric s x s S (column i = row i, coalesced), warp per row.
template <typename T>
__global__ void k_symv(const T* __restrict__ S, int s, const T* __restrict__ x, T* __restrict__ y, const int* status) {
  if (failed(status)) return;
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= s) return;
  const T* row = S + (size_t)i * s;
  T acc = 0;
  for (int j = lane; j < s; j += 32) acc = fma(row[j], x[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) y[i] = acc;
}

// Sum over the CTA (blockDim a multiple of 32, <= 1024); every thread gets it.
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = lane < nw ? red[lane] : (T)0;
  return warp_sum(t);
}

// GKL state: Pm (s x (l+1)) right Lanczos vectors, W (s x l) coefficients of
// the left ones, wr (s) the unnormalised next coefficient vector, u (s) = S wr,
// ab[0..l) alpha, ab[l..2l) beta, ab[2l] running scale, ab[2l+1] stop flag.
template <typename T>
__global__ void k_gkl_start(const T* __restrict__ p1, int s, int l, T* __restrict__ Pm, T* __restrict__ W,
                            T* __restrict__ wr, T* __restrict__ ab, const int* status) {
  if (failed(status)) return;
  __shared__ T red[32];
  const int i = threadIdx.x;
  T v = i < s ? (p1 ? p1[i] : (T)1) : (T)0;
  T nrm2 = block_sum(v * v, red);
  T inv = nrm2 > (T)0 ? (T)1 / sqrt(nrm2) : (T)0;
  if (i < s) {
    Pm[i] = v * inv;
    wr[i] = v * inv;
    for (int c = 0; c < l; ++c) W[(size_t)c * s + i] = (T)0;
    for (int c = 1; c <= l; ++c) Pm[(size_t)c * s + i] = (T)0;
  }
  for (int t = i; t < 2 * l + 2; t += blockDim.x) ab[t] = (T)0;
}

// One Lanczos step (one CTA, one thread per entry, s <= blockDim):
//   alpha = sqrt(wr^T u); w_i = wr / alpha; v = u / alpha - alpha p_i;
//   v orthogonalised against p_1..p_i (modified Gram-Schmidt); beta = |v|;
//   p_{i+1} = v / beta; next wr = p_{i+1} - beta w_i.
// A breakdown (alpha or beta below 1e-13 of the largest seen) stops the
// recurrence: later vectors stay zero.
template <typename T>
__global__ void __launch_bounds__(1024) k_gkl_step(int it, int s, int l, T* __restrict__ Pm, T* __restrict__ W,
                                                   T* __restrict__ wr, const T* __restrict__ u, T* __restrict__ ab,
                                                   const int* status) {
  if (failed(status)) return;
  __shared__ T red[32];
  const int i = threadIdx.x;
  const bool on = i < s;
  if (ab[2 * l + 1] != (T)0) return;   // stopped (uniform)
  T w = on ? wr[i] : (T)0, ui = on ? u[i] : (T)0;
  T a2 = block_sum(w * ui, red);
  T a = sqrt(fmax(a2, (T)0));
  T scale = fmax(ab[2 * l], a);
  if (!(a > (T)1e-13 * scale)) {
    if (i == 0) ab[2 * l + 1] = (T)1;
    return;
  }
  w /= a;
  if (on) W[(size_t)it * s + i] = w;
  T v = on ? ui / a - a * Pm[(size_t)it * s + i] : (T)0;
  for (int j = 0; j <= it; ++j) {
    T pj = on ? Pm[(size_t)j * s + i] : (T)0;
    T d = block_sum(pj * v, red);
    v -= d * pj;
  }
  T b = sqrt(block_sum(v * v, red));
  scale = fmax(scale, b);
  const bool brk = !(b > (T)1e-13 * scale);
  if (i == 0) {
    ab[it] = a;
    ab[l + it] = brk ? (T)0 : b;
    ab[2 * l] = scale;
    if (brk) ab[2 * l + 1] = (T)1;
  }
  if (on) {
    T p = brk ? (T)0 : v / b;
    Pm[(size_t)(it + 1) * s + i] = p;
    wr[i] = p - (brk ? (T)0 : b) * w;
  }
}

// P = P_{l+1} H^T: column i = alpha_i p_i + beta_i p_{i+1}
template <typename T>
__global__ void k_gkl_finish(const T* __restrict__ Pm, const T* __restrict__ ab, int s, int l, T* __restrict__ P,
                             const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)s * l) return;
  int i = (int)(t % s), c = (int)(t / s);
  P[t] = ab[c] * Pm[(size_t)c * s + i] + ab[l + c] * Pm[(size_t)(c + 1) * s + i];
}

// Orthonormal columns of P (s x l, one CTA, modified Gram-Schmidt; a column
// that vanishes stays zero).
template <typename T>
__global__ void __launch_bounds__(1024) k_mgs_cols(T* __restrict__ P, int s, int l, const int* status) {
  if (failed(status)) return;
  __shared__ T red[32];
  const int i = threadIdx.x;
  const bool on = i < s;
  for (int c = 0; c < l; ++c) {
    T v = on ? P[(size_t)c * s + i] : (T)0;
    for (int j = 0; j < c; ++j) {
      T pj = on ? P[(size_t)j * s + i] : (T)0;
      T d = block_sum(pj * v, red);
      v -= d * pj;
    }
    T n2 = block_sum(v * v, red);
    T inv = n2 > (T)0 ? (T)1 / sqrt(n2) : (T)0;
    if (on) P[(size_t)c * s + i] = v * inv;
    __syncthreads();
  }
}

// e2_j = w_j^T M w_j for the columns of W (s x l), given T = M W: one warp per column.
template <typename T>
__global__ void k_diag_quad(const T* __restrict__ W, const T* __restrict__ TM, int s, int l, T* __restrict__ e2,
                            const int* status) {
  if (failed(status)) return;
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= l) return;
  T acc = 0;
  for (int i = lane; i < s; i += 32) acc = fma(W[(size_t)c * s + i], TM[(size_t)c * s + i], acc);
  acc = warp_sum(acc);
  if (lane == 0) e2[c] = acc;
}

// K = [[diag(sigma), C0], [0, P^T]]  ((k+l) x (k+s), column-major, ld k+l)
template <typename T>
__global__ void k_build_K_rect(const T* __restrict__ sigma, const T* __restrict__ C0, const T* __restrict__ P, int k,
                               int s, int l, T* __restrict__ K, const int* status) {
  if (failed(status)) return;
  const int rows = k + l, cols = k + s;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * cols) return;
  int i = (int)(t % rows), j = (int)(t / rows);
  T v = (T)0;
  if (i < k && j < k) v = i == j ? sigma[i] : (T)0;
  else if (i < k) v = C0[(size_t)(j - k) * k + i];
  else if (j >= k) v = P[(size_t)(i - k) * s + (j - k)];
  K[t] = v;
}

// L = [C0; P^T]  ((k+l) x s)
template <typename T>
__global__ void k_build_L_rect(const T* __restrict__ C0, const T* __restrict__ P, int k, int s, int l,
                               T* __restrict__ L, const int* status) {
  if (failed(status)) return;
  const int rows = k + l;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * s) return;
  int i = (int)(t % rows), j = (int)(t / rows);
  L[t] = i < k ? C0[(size_t)j * k + i] : P[(size_t)(i - k) * s + j];
}

// G[:, j] /= theta_j (0 for a zero singular value)
template <typename T>
__global__ void k_scale_cols(T* __restrict__ G, int rows, int ld, int k, const T* __restrict__ theta,
                             const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)rows * k) return;
  int i = (int)(t % rows), j = (int)(t / rows);
  T th = theta[j];
  G[(size_t)j * ld + i] = th > (T)0 ? G[(size_t)j * ld + i] / th : (T)0;
}

template <typename T>
void launch_gkl(const T* S, int s, int l, const T* p1, T* Pm, T* W, T* wr, T* u, T* ab, T* P, const int* status,
                cudaStream_t st) {
  const int threads = std::max(32, (int)cdiv(s, 32) * 32);
  note_launches(1);
  k_gkl_start<T><<<1, threads, 0, st>>>(p1, s, l, Pm, W, wr, ab, status);
  for (int it = 0; it < l; ++it) {
    note_launches(2);
    k_symv<T><<<(int)cdiv(s, 8), 256, 0, st>>>(S, s, wr, u, status);
    k_gkl_step<T><<<1, threads, 0, st>>>(it, s, l, Pm, W, wr, u, ab, status);
  }
  note_launches(1);
  k_gkl_finish<T><<<(int)cdiv((int64_t)s * l, 256), 256, 0, st>>>(Pm, ab, s, l, P, status);
}

template <typename T>
void launch_mgs_cols(T* P, int s, int l, const int* status, cudaStream_t st) {
  note_launches(1);
  k_mgs_cols<T><<<1, std::max(32, (int)cdiv(s, 32) * 32), 0, st>>>(P, s, l, status);
}

template <typename T>
void launch_diag_quad(const T* W, const T* TM, int s, int l, T* e2, const int* status, cudaStream_t st) {
  note_launches(1);
  k_diag_quad<T><<<(int)cdiv(l, 8), 256, 0, st>>>(W, TM, s, l, e2, status);
}

template <typename T>
void launch_build_K_rect(const T* sigma, const T* C0, const T* P, int k, int s, int l, T* K, const int* status,
                         cudaStream_t st) {
  note_launches(1);
  k_build_K_rect<T><<<(int)cdiv((int64_t)(k + l) * (k + s), 256), 256, 0, st>>>(sigma, C0, P, k, s, l, K, status);
}

template <typename T>
void launch_build_L_rect(const T* C0, const T* P, int k, int s, int l, T* L, const int* status, cudaStream_t st) {
  note_launches(1);
  k_build_L_rect<T><<<(int)cdiv((int64_t)(k + l) * s, 256), 256, 0, st>>>(C0, P, k, s, l, L, status);
}

template <typename T>
void launch_scale_cols(T* G, int rows, int ld, int k, const T* theta, const int* status, cudaStream_t st) {
  note_launches(1);
  k_scale_cols<T><<<(int)cdiv((int64_t)rows * k, 256), 256, 0, st>>>(G, rows, ld, k, theta, status);
}

#define SVL_APPROX_INST(T)                                                                                      \
  template void launch_gkl<T>(const T*, int, int, const T*, T*, T*, T*, T*, T*, T*, const int*, cudaStream_t); \
  template void launch_mgs_cols<T>(T*, int, int, const int*, cudaStream_t);                                   \
  template void launch_diag_quad<T>(const T*, const T*, int, int, T*, const int*, cudaStream_t);              \
  template void launch_build_K_rect<T>(const T*, const T*, const T*, int, int, int, T*, const int*,           \
                                       cudaStream_t);                                                         \
  template void launch_build_L_rect<T>(const T*, const T*, int, int, int, T*, const int*, cudaStream_t);      \
  template void launch_scale_cols<T>(T*, int, int, int, const T*, const int*, cudaStream_t);
SVL_APPROX_INST(float)
SVL_APPROX_INST(double)

}  // namespace svl

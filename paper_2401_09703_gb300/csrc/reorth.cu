// Re-orthonormalisation of a low-precision factor X = X' W (used for BF16
// storage).  Rounding X' to BF16 (8-bit mantissa) on every append, scatter
// and reset moves X'W away from orthonormal; the update formulas of Section
// 3.2 assume U^T U = I (the residual Gram E^T E - C0^T C0, Lemma 2), so the
// drift feeds straight into Sigma.  The correction replaces W by
// W (W^T X'^T X' W)^{-1/2}: the closest orthonormal basis to X'W (its polar
// factor), which keeps every column on its singular vector to first order and
// removes the first-order error of the column norms.  The paper has no such
// step (it assumes exact arithmetic); it is a storage-precision safeguard,
// like the reset of the small factors.
#include <algorithm>

#include "kernels.cuh"

namespace svl {

constexpr int kGramRows = 32;  // rows of X' staged in shared memory per pass

// Partial Grams of X' (rows x k, storage TS) over row chunks: CTA c sums the
// outer products of its rows in registers (8 x 8 tile per thread) and writes
// the k x k partial in FP64.  Accumulation type: FP32 for BF16 storage (the
// products are exact in FP32, the sum's rounding is far below BF16's), FP64
// otherwise (a correction must be more accurate than the storage it fixes).
template <typename TS> struct GramAcc { using type = double; };
template <> struct GramAcc<__nv_bfloat16> { using type = float; };

template <typename TS>
__global__ void __launch_bounds__(256) k_gram_rows(const TS* __restrict__ Xp, int64_t rows, int k, int64_t chunk,
                                                   double* __restrict__ part, const int* status) {
  using A = typename GramAcc<TS>::type;
  if (failed(status)) return;
  extern __shared__ __align__(16) unsigned char gsm[];
  A* xs = (A*)gsm;   // kGramRows x k
  const int nt = (k + 7) / 8;
  const int t = threadIdx.x;
  const bool own = t < nt * nt;
  const int i0 = own ? (t / nt) * 8 : 0, j0 = own ? (t % nt) * 8 : 0;
  A acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = (A)0;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  for (int64_t rb = r0; rb < r1; rb += kGramRows) {
    const int nr = (int)min((int64_t)kGramRows, r1 - rb);
    __syncthreads();
    for (int e = t; e < nr * k; e += blockDim.x) xs[e] = (A)to_f64(Xp[(rb + e / k) * k + e % k]);
    __syncthreads();
    if (own) {
      for (int r = 0; r < nr; ++r) {
        const A* x = xs + r * k;
        A xa[8], xb[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          xa[a] = i0 + a < k ? x[i0 + a] : (A)0;
          xb[a] = j0 + a < k ? x[j0 + a] : (A)0;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fma(xa[a], xb[b], acc[a][b]);
      }
    }
  }
  if (own) {
    double* P = part + (size_t)blockIdx.x * k * k;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (i0 + a < k && j0 + b < k) P[(size_t)(j0 + b) * k + (i0 + a)] = (double)acc[a][b];
  }
}

// G = sum of the partials, in chunk order (deterministic)
__global__ void k_sum_partials(const double* __restrict__ part, int nchunks, int kk, double* __restrict__ G,
                               const int* status) {
  if (failed(status)) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kk) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * kk + e];
  G[e] = s;
}

// T = 1.5 I - 0.5 A (the Newton-Schulz factor)
__global__ void k_ns_factor(const double* __restrict__ A, int k, double* __restrict__ T, const int* status) {
  if (failed(status)) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int i = e % k, j = e / k;
  T[e] = (i == j ? 1.5 : 0.0) - 0.5 * A[e];
}

__global__ void k_set_identity_d(double* __restrict__ A, int k, const int* status) {
  if (failed(status)) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < k * k) A[e] = (e % k == e / k) ? 1.0 : 0.0;
}

int reorth_chunks(int64_t rows) { return (int)std::max<int64_t>(1, std::min<int64_t>(128, cdiv(rows, 512))); }

size_t reorth_work_bytes(int k, int64_t max_rows) {
  return sizeof(double) * ((size_t)reorth_chunks(max_rows) * k * k + 6 * (size_t)k * k) + 8 * 256;
}

// W <- W (W^T X'^T X' W)^{-1/2} by the coupled Newton-Schulz iteration
// (Y_0 = M, Z_0 = I, T = (3I - Z Y)/2, Y <- Y T, Z <- T Z; Z -> M^{-1/2}),
// which converges quadratically while |I - M| < 1 (the drift here is ~1e-3).
template <typename TS>
void launch_reorth(const TS* Xp, int64_t rows, int k, double* W, void* work, int* status, cudaStream_t st) {
  if (rows <= 0) return;
  const int nch = reorth_chunks(rows);
  const int64_t chunk = cdiv(rows, nch);
  char* w = (char*)work;
  auto take = [&](size_t bytes) { char* p = w; w += (bytes + 255) & ~(size_t)255; return (double*)p; };
  const size_t kk = (size_t)k * k;
  double* part = take(sizeof(double) * nch * kk);
  double *G = take(8 * kk), *M = take(8 * kk), *Y = take(8 * kk), *Z = take(8 * kk), *T = take(8 * kk),
         *A = take(8 * kk);
  note_launches(2);
  k_gram_rows<TS><<<nch, 256, sizeof(typename GramAcc<TS>::type) * kGramRows * k, st>>>(Xp, rows, k, chunk, part,
                                                                                      status);
  k_sum_partials<<<(int)cdiv(kk, 256), 256, 0, st>>>(part, nch, (int)kk, G, status);
  gemm<double>(false, false, k, k, k, 1.0, G, k, W, k, 0.0, A, k, status, st);      // G W
  gemm<double>(true, false, k, k, k, 1.0, W, k, A, k, 0.0, M, k, status, st);       // M = W^T G W
  launch_copy<double>(M, Y, (int64_t)kk, status, st);
  note_launches(1);
  k_set_identity_d<<<(int)cdiv(kk, 256), 256, 0, st>>>(Z, k, status);
  for (int it = 0; it < 4; ++it) {
    gemm<double>(false, false, k, k, k, 1.0, Z, k, Y, k, 0.0, A, k, status, st);    // Z Y
    note_launches(1);
    k_ns_factor<<<(int)cdiv(kk, 256), 256, 0, st>>>(A, k, T, status);
    gemm<double>(false, false, k, k, k, 1.0, Y, k, T, k, 0.0, A, k, status, st);    // Y T
    launch_copy<double>(A, Y, (int64_t)kk, status, st);
    gemm<double>(false, false, k, k, k, 1.0, T, k, Z, k, 0.0, A, k, status, st);    // T Z
    launch_copy<double>(A, Z, (int64_t)kk, status, st);
  }
  gemm<double>(false, false, k, k, k, 1.0, W, k, Z, k, 0.0, A, k, status, st);      // W M^{-1/2}
  launch_copy<double>(A, W, (int64_t)kk, status, st);
}

template void launch_reorth<double>(const double*, int64_t, int, double*, void*, int*, cudaStream_t);
template void launch_reorth<float>(const float*, int64_t, int, double*, void*, int*, cudaStream_t);
template void launch_reorth<__nv_bfloat16>(const __nv_bfloat16*, int64_t, int, double*, void*, int*, cudaStream_t);

}  // namespace svl

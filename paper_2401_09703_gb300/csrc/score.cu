// Scores of node (user, item) pairs from the maintained truncated SVD: the
// inference step of the paper's downstream tasks (Section 4, task setup of
// link prediction and collaborative filtering), the inner product
// U[i]^T Sigma V[j] of the two representations, i.e. entry (i, j) of
// U Sigma V^T; for an undirected graph the larger of the two directions.
//
// With the extended decomposition U = U' W_U, V = V' W_V (Section 3.2):
//   score(i, j) = U'[i] M V'[j]^T,   M = W_U diag(Sigma) W_V^T  (k x k),
// so a pair costs two row gathers of U' and V' (2 k storage elements) and a
// k x k bilinear form; the factors are never materialised.  M is formed once
// per call (k CTAs, one row each), then one warp per pair with M staged in
// shared memory (FP32 for FP32 / BF16 storage, FP64 for FP64 storage, as the
// other row kernels compute).
#include <cmath>

#include "kernels.cuh"

namespace svl {

namespace {

// M(a, b) = sum_l W_U(a, l) sigma_l W_V(b, l); W column-major k x k; M row-major.
template <typename TC>
__global__ void k_score_M(const TC* __restrict__ Wu, const TC* __restrict__ Wv, const TC* __restrict__ sigma, int k,
                          double* __restrict__ M, const int* status) {
  if (failed(status)) return;
  const int a = blockIdx.x;
  for (int b = threadIdx.x; b < k; b += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < k; ++l)
      acc = fma((double)Wu[(int64_t)l * k + a] * (double)sigma[l], (double)Wv[(int64_t)l * k + b], acc);
    M[(int64_t)a * k + b] = acc;
  }
}

// u M v^T by one warp: lane t holds u_a and v_a for a = t + 32 q.
template <typename A, int NQ>
__device__ __forceinline__ A bilinear(const A* __restrict__ Ms, int k, const A* ur, const A* vr, int lane) {
  A w[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) w[q] = (A)0;
#pragma unroll
  for (int qa = 0; qa < NQ; ++qa) {
    for (int t = 0; t < 32; ++t) {
      const int a = 32 * qa + t;
      if (a >= k) break;
      const A ua = __shfl_sync(0xffffffffu, ur[qa], t);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int b = lane + 32 * q;
        if (b < k) w[q] = fma(ua, Ms[(int64_t)a * k + b], w[q]);
      }
    }
  }
  A s = (A)0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) s = fma(w[q], vr[q], s);
  return warp_sum(s);
}

template <typename TS, typename A, int NQ>
__device__ __forceinline__ void load_row(const TS* __restrict__ X, int64_t r, int k, int lane, A* reg) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int a = lane + 32 * q;
    reg[q] = a < k ? (A)to_f64(X[r * k + a]) : (A)0;
  }
}

template <typename TS, typename A, int NQ>
__global__ void __launch_bounds__(256) k_score_pairs(const TS* __restrict__ Up, const TS* __restrict__ Vp, int64_t m,
                                                     int64_t n, int k, const double* __restrict__ M,
                                                     const int32_t* __restrict__ rows,
                                                     const int32_t* __restrict__ cols, int64_t npairs, int symmetric,
                                                     double* __restrict__ out, int* status) {
  extern __shared__ __align__(16) unsigned char sc_smem[];
  A* Ms = (A*)sc_smem;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Ms[t] = (A)M[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t p = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5); p < npairs; p += (int64_t)gridDim.x * nw) {
    const int64_t i = rows[p], j = cols[p];
    const bool ok = i >= 0 && i < m && j >= 0 && j < n && (!symmetric || (j < m && i < n));
    if (!ok) {
      if (lane == 0) {
        out[p] = __longlong_as_double(0x7FF8000000000000ll);   // NaN
        flag(status, SVLCOV_DEV_BAD_CSR);
      }
      continue;
    }
    A ur[NQ], vr[NQ];
    load_row<TS, A, NQ>(Up, i, k, lane, ur);
    load_row<TS, A, NQ>(Vp, j, k, lane, vr);
    double sc = (double)bilinear<A, NQ>(Ms, k, ur, vr, lane);
    if (symmetric) {   // undirected graph: the larger direction
      load_row<TS, A, NQ>(Up, j, k, lane, ur);
      load_row<TS, A, NQ>(Vp, i, k, lane, vr);
      sc = fmax(sc, (double)bilinear<A, NQ>(Ms, k, ur, vr, lane));
    }
    if (lane == 0) out[p] = sc;
  }
}

int g_score_sms = 0;

}  // namespace

size_t score_work_bytes(int k) { return sizeof(double) * (size_t)k * k; }

template <typename TS, typename TC>
void launch_score_pairs(const TS* Up, const TS* Vp, int64_t m, int64_t n, int k, const TC* Wu, const TC* Wv,
                        const TC* sigma, const int32_t* rows, const int32_t* cols, int64_t npairs, int symmetric,
                        double* out, double* Mwork, int* status, cudaStream_t st) {
  if (npairs <= 0) return;
  using A = typename Acc<TS>::type;
  if (!g_score_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_score_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_score_sms <= 0) g_score_sms = 152;
  }
  note_launches(2);
  k_score_M<TC><<<k, 128, 0, st>>>(Wu, Wv, sigma, k, Mwork, status);
  const size_t smem = sizeof(A) * (size_t)k * k;
  const int64_t want = cdiv(npairs, 8);
  const int grid = (int)std::min<int64_t>(want, (int64_t)g_score_sms * 4);
  auto launch = [&](auto fn) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fn<<<grid, 256, smem, st>>>(Up, Vp, m, n, k, Mwork, rows, cols, npairs, symmetric, out, status);
  };
  if (k <= 32) launch(k_score_pairs<TS, A, 1>);
  else if (k <= 64) launch(k_score_pairs<TS, A, 2>);
  else if (k <= 96) launch(k_score_pairs<TS, A, 3>);
  else launch(k_score_pairs<TS, A, 4>);
}

#define INST_SCORE(TS, TC)                                                                                    \
  template void launch_score_pairs<TS, TC>(const TS*, const TS*, int64_t, int64_t, int, const TC*, const TC*, \
                                           const TC*, const int32_t*, const int32_t*, int64_t, int, double*,  \
                                           double*, int*, cudaStream_t);
INST_SCORE(double, double)
INST_SCORE(double, float)
INST_SCORE(float, double)
INST_SCORE(float, float)
INST_SCORE(__nv_bfloat16, double)
INST_SCORE(__nv_bfloat16, float)

}  // namespace svl

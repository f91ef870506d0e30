// Projection of many update vectors onto the current singular space in one
// launch: P = X'^T E^T (k x s) and C0 = W^T P = X^T E^T, the first step of
// turning a batch into SV-LCOV form (Lemma 1: the projection gathers rows of
// U' at the vectors' nonzeros and multiplies by the small factor once).
//
// Uses: the look-ahead projection of many pending batches at once (the rows
// of X' change between steps only where a step scatters, so a projection
// taken ahead stays exact on every other row), and folding new vectors into
// the current representation without updating it.  It is the gather of the
// update step without the Gram matrix, so it shows what that gather costs
// when X' does not fit in L2: one warp per update vector streams the rows of
// X' it touches (k storage elements per nonzero, as 8- or 16-byte vectors,
// four rows in flight per warp) and writes its column of P.
#include "kernels.cuh"

namespace svl {

namespace {

// Four consecutive elements of a row per lane (k <= 128 = 32 lanes x 4), as
// one 8-byte (BF16) or 16-byte (FP32) load, or two 16-byte loads (FP64).
template <typename TS> struct RowVec;
template <> struct RowVec<__nv_bfloat16> {
  using V = uint2;
  __device__ static V load(const __nv_bfloat16* p) { return *(const uint2*)p; }
  __device__ static void unpack(const V& v, float* o) {
    o[0] = __uint_as_float(v.x << 16);
    o[1] = __uint_as_float(v.x & 0xFFFF0000u);
    o[2] = __uint_as_float(v.y << 16);
    o[3] = __uint_as_float(v.y & 0xFFFF0000u);
  }
};
template <> struct RowVec<float> {
  using V = float4;
  __device__ static V load(const float* p) { return *(const float4*)p; }
  __device__ static void unpack(const V& v, float* o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <> struct RowVec<double> {
  struct V { double2 a, b; };
  __device__ static V load(const double* p) { return V{((const double2*)p)[0], ((const double2*)p)[1]}; }
  __device__ static void unpack(const V& v, double* o) { o[0] = v.a.x; o[1] = v.a.y; o[2] = v.b.x; o[3] = v.b.y; }
};

// One warp per update vector j: P[:, j] = sum over its nonzeros (i, v) of
// v X'[i, :].  Lane t owns elements [E t, E t + E) of a row (k / E lanes
// active); NB rows are loaded before they are accumulated.
template <typename TS, typename TP>
__global__ void __launch_bounds__(256) k_project(const int32_t* __restrict__ indptr,
                                                 const int32_t* __restrict__ indices, const void* __restrict__ values,
                                                 int vdtype, int s, const TS* __restrict__ Xp, int64_t rows, int k,
                                                 TP* __restrict__ P, int* status) {
  using RV = RowVec<TS>;
  using A = typename Acc<TS>::type;
  constexpr int E = 4, NB = 4;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= s) return;
  const bool act = lane * E < k;    // k is a multiple of 4 (checked by the host), k <= 128
  A acc[E];
#pragma unroll
  for (int t = 0; t < E; ++t) acc[t] = (A)0;
  const int64_t e0 = indptr[j], e1 = indptr[j + 1];
  for (int64_t e = e0; e < e1; e += NB) {
    typename RV::V v[NB];
    A w[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      w[u] = (A)0;
      if (e + u < e1) {
        const int i = indices[e + u];
        if (i < 0 || (int64_t)i >= rows) {
          if (lane == 0) flag(status, SVLCOV_DEV_BAD_CSR);
        } else {
          w[u] = (A)load_val<double>(values, vdtype, e + u);
          if (act) v[u] = RV::load(Xp + (int64_t)i * k + lane * E);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      if (w[u] != (A)0 && act) {
        A x[E];
        RV::unpack(v[u], x);
#pragma unroll
        for (int t = 0; t < E; ++t) acc[t] = fma(w[u], x[t], acc[t]);
      }
    }
  }
  if (act) {
#pragma unroll
    for (int t = 0; t < E; ++t) P[(int64_t)j * k + lane * E + t] = (TP)acc[t];
  }
}

}  // namespace

template <typename TS, typename TP>
void launch_project(const svlcov_csr& b, const TS* Xp, int64_t rows, int k, TP* P, int* status, cudaStream_t st) {
  if (b.rows <= 0) return;
  note_launches(1);
  const int wpb = 8;
  k_project<TS, TP><<<(unsigned)cdiv(b.rows, wpb), wpb * 32, 0, st>>>(b.indptr, b.indices, b.values, b.values_dtype,
                                                                      b.rows, Xp, rows, k, P, status);
}

template void launch_project<double, double>(const svlcov_csr&, const double*, int64_t, int, double*, int*,
                                             cudaStream_t);
template void launch_project<float, double>(const svlcov_csr&, const float*, int64_t, int, double*, int*,
                                            cudaStream_t);
template void launch_project<__nv_bfloat16, double>(const svlcov_csr&, const __nv_bfloat16*, int64_t, int, double*,
                                                    int*, cudaStream_t);

}  // namespace svl

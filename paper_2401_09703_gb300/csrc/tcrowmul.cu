// The dense fold of a small factor into a stored factor on the tensor cores:
// out (rows x k) = X' (rows x k, row-major, BF16 or FP32 storage) W (k x k,
// column-major).  It is the reset of the extended decomposition (X' <- X' W,
// W <- I, when the conditioning guard fires; Section 3.2) and the
// materialisation U = U' U'' of the factors (Theorem 1's query, for every
// row), a contraction of k terms per output that the FP32 pipe finishes at
// ~1/4 of the HBM rate at k = 128; BF16 tcgen05.mma with FP32 accumulation
// in tensor memory keeps it HBM-bound.
//
// Precision: FP32 results from BF16 pieces.  W (FP64 or FP32) is rounded to
// FP32 and split exactly into three BF16 pieces W0 + W1 + W2 (8 significant
// bits each); BF16 storage is one piece, FP32 storage three pieces X0 + X1 +
// X2 the same way.  The products kept are those above 2^-32 relative
// (X_a W_b with a + b <= 3: three MMAs per K-step for BF16 storage -- all of
// them --, eight for FP32), all accumulated in one FP32 accumulator; each
// piece product is exact in FP32, so the result carries the accumulator's
// rounding only.
//
// Persistent CTAs (one per SM): W's pieces are staged once in shared memory
// in the MMA's no-swizzle K-major layout; per 128-row tile the threads read
// the rows (32-byte vectors, coalesced), split them into the A pieces in
// shared memory, one thread issues the MMAs, and after the commit the
// accumulator is read back with tcgen05.ld and stored.  Rows of one tile are
// read completely before any is written, and tiles are disjoint, so the
// fold may run in place (out == X').
#include <algorithm>

#include "kernels.cuh"

namespace svl {

namespace {

constexpr int RT_M = 128;          // rows per tile (MMA M, tensor-memory lanes)
constexpr int RT_THREADS = 256;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// no-swizzle K-major matrix descriptor (version 1): start, leading byte
// offset (next 8-element K chunk), stride byte offset (next 8-row group)
__device__ __forceinline__ uint64_t rdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool rt_wait(uint32_t mbar, uint32_t phase) {
  for (long it = 0; it < (1L << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// FP32 -> BF16 pieces: x = p0 + p1 + p2 exactly for normal FP32 x (each
// piece takes the next 8 significant bits, round to nearest)
__device__ __forceinline__ void split3(float x, uint16_t& p0, uint16_t& p1, uint16_t& p2) {
  const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b1);
  const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
  p0 = __bfloat16_as_ushort(b0);
  p1 = __bfloat16_as_ushort(b1);
  p2 = __bfloat16_as_ushort(b2);
}

template <typename TO> __device__ __forceinline__ TO cvt_out(float v);
template <> __device__ __forceinline__ float cvt_out<float>(float v) { return v; }
template <> __device__ __forceinline__ double cvt_out<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void tmem_ld32x32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Pieces of the A operand: one for BF16 storage, three for FP32.
template <typename TS> struct APieces { static constexpr int n = 1; };
template <> struct APieces<float> { static constexpr int n = 3; };

// Shared layout of one operand piece with R rows and K = k columns: element
// (r, c) at (c / 8) (R 16) + r 16 + (c % 8) 2 -- K chunks of 8 elements,
// each a column of R / 8 core matrices (8 rows x 16 bytes, contiguous): the
// leading byte offset is R 16, the stride byte offset 128.
template <typename TS, typename TC, typename TO>
__global__ void __launch_bounds__(RT_THREADS, 1) k_rowmul_tc(const TS* X, int64_t rows, int k,
                                                             const TC* __restrict__ W, TO* out,
                                                             const int* do_reset, const int* status, uint32_t tcols) {
  constexpr int NA = APieces<TS>::n;
  extern __shared__ unsigned char rt_raw[];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  if (do_reset && *(volatile const int*)do_reset == 0) return;
  if (status && failed(status)) return;
  unsigned char* sm = (unsigned char*)(((uintptr_t)rt_raw + 127) & ~(uintptr_t)127);
  const uint32_t planeA = (uint32_t)RT_M * k * 2, planeW = (uint32_t)k * k * 2;
  unsigned char* Ap = sm;                       // NA pieces of the 128 x k tile
  unsigned char* Wp = sm + (size_t)NA * planeA;  // 3 pieces of W^T (k x k, row n = column n of W)
  const int tid = threadIdx.x, warp = tid >> 5;
  // W^T pieces: element (n, c) = W(c, n) = W[n k + c]
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int n = e / k, c = e - n * k;
    uint16_t p0, p1, p2;
    split3((float)W[(int64_t)n * k + c], p0, p1, p2);
    const uint32_t off = (uint32_t)((c >> 3) * (k * 16) + n * 16 + (c & 7) * 2);
    *(uint16_t*)(Wp + off) = p0;
    *(uint16_t*)(Wp + planeW + off) = p1;
    *(uint16_t*)(Wp + 2 * planeW + off) = p2;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot, mb = su32(&mbar);
  // instruction descriptor: D FP32, A and B BF16, K-major both, N = k, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(k >> 3) << 17) | ((uint32_t)(RT_M >> 4) << 24);
  const int64_t ntiles = cdiv(rows, RT_M);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t r0 = tile * RT_M;
    // ---- A pieces: item (row r, 32-byte segment q of the row)
    constexpr int SEG = 32 / (int)sizeof(TS);       // elements per 32-byte segment: 16 BF16 or 8 FP32
    const int nseg = k / SEG;
    for (int it = tid; it < RT_M * nseg; it += blockDim.x) {
      const int r = it % RT_M, q = it / RT_M;         // consecutive threads: consecutive rows
      const int64_t gr = r0 + r;
      uint4 v0 = make_uint4(0, 0, 0, 0), v1 = make_uint4(0, 0, 0, 0);
      if (gr < rows) {
        const uint4* src = (const uint4*)(X + gr * k + q * SEG);
        v0 = src[0];
        v1 = src[1];
      }
      if constexpr (NA == 1) {   // BF16: two 8-element chunks, copied as they are
        const int c0 = q * 2;
        *(uint4*)(Ap + (size_t)c0 * (RT_M * 16) + r * 16) = v0;
        *(uint4*)(Ap + (size_t)(c0 + 1) * (RT_M * 16) + r * 16) = v1;
      } else {                   // FP32: one 8-element chunk, three pieces
        const float f[8] = {__uint_as_float(v0.x), __uint_as_float(v0.y), __uint_as_float(v0.z),
                            __uint_as_float(v0.w), __uint_as_float(v1.x), __uint_as_float(v1.y),
                            __uint_as_float(v1.z), __uint_as_float(v1.w)};
        uint16_t p[3][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) split3(f[e], p[0][e], p[1][e], p[2][e]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          uint4 w;
          w.x = (uint32_t)p[a][0] | ((uint32_t)p[a][1] << 16);
          w.y = (uint32_t)p[a][2] | ((uint32_t)p[a][3] << 16);
          w.z = (uint32_t)p[a][4] | ((uint32_t)p[a][5] << 16);
          w.w = (uint32_t)p[a][6] | ((uint32_t)p[a][7] << 16);
          *(uint4*)(Ap + (size_t)a * planeA + (size_t)q * (RT_M * 16) + r * 16) = w;
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(Ap), w0 = su32(Wp);
      bool first = true;
      for (int ks = 0; ks < k / 16; ++ks) {
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int b = 0; b < 3 && a + b <= 3; ++b) {
            const uint64_t ad = rdesc(a0 + a * planeA + ks * 2 * (RT_M * 16), RT_M * 16, 128);
            const uint64_t bd = rdesc(w0 + b * planeW + ks * 2 * (k * 16), k * 16, 128);
            const uint32_t acc = first ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
            first = false;
          }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    ok = __syncthreads_and(rt_wait(mb, phase) ? 1 : 0) != 0;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (tid == 0 && status) flag((int*)status, SVLCOV_DEV_TIMEOUT);
      rt_wait(mb, phase ^ 1u);   // the MMAs in flight, bounded again
      break;
    }
    // ---- epilogue: warp w reads lanes 32 (w % 4).. (rows), columns 32 (w / 4) + 64 j ..
    const int quad = warp & 3, half = warp >> 2;
    const int r = 32 * quad + (tid & 31);
    const int64_t gr = r0 + r;
    for (int c0 = 32 * half; c0 < k; c0 += 64) {
      float v[32];
      tmem_ld32x32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0, v);
      if (gr < rows) {   // X and out may be the same rows: every read of them came before the barrier
        TO* dst = out + gr * k + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < k) dst[j] = cvt_out<TO>(v[j]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // the accumulator and the A pieces are free for the next tile
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

int g_rt_sms = 0;

}  // namespace

// Whether the tensor-core fold applies: BF16 or FP32 storage, k a multiple
// of 16 between 16 and 128, whole factor (no row index list).
bool rowmul_tc_ok(int storage_bytes, int k) { return storage_bytes != 8 && k >= 16 && k <= 128 && k % 16 == 0; }

template <typename TS, typename TC, typename TO>
void launch_rowmul_tc(const TS* X, int64_t rows, int k, const TC* W, TO* out, const int* do_reset, const int* status,
                      cudaStream_t st) {
  if (rows <= 0) return;
  if (!g_rt_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_rt_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_rt_sms <= 0) g_rt_sms = 152;
  }
  const size_t smem = (size_t)APieces<TS>::n * RT_M * k * 2 + 3 * (size_t)k * k * 2 + 128;
  const uint32_t tcols = k <= 32 ? 32u : (k <= 64 ? 64u : 128u);
  auto fn = k_rowmul_tc<TS, TC, TO>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = (int)std::min<int64_t>(cdiv(rows, RT_M), g_rt_sms);
  note_launches(1);
  fn<<<grid, RT_THREADS, smem, st>>>(X, rows, k, W, out, do_reset, status, tcols);
}

#define INST_RT(TS, TC, TO)                                                                                   \
  template void launch_rowmul_tc<TS, TC, TO>(const TS*, int64_t, int, const TC*, TO*, const int*, const int*, \
                                             cudaStream_t);
INST_RT(float, double, float)
INST_RT(float, float, float)
INST_RT(float, double, double)
INST_RT(float, float, double)
INST_RT(__nv_bfloat16, double, __nv_bfloat16)
INST_RT(__nv_bfloat16, float, __nv_bfloat16)
INST_RT(__nv_bfloat16, double, float)
INST_RT(__nv_bfloat16, float, float)
INST_RT(__nv_bfloat16, double, double)
INST_RT(__nv_bfloat16, float, double)

}  // namespace svl

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
// in the MMA's 128-byte-swizzled K-major layout; per 128-row tile each warp
// holds whole rows in registers (loaded while the previous tile was being
// multiplied and written), splits them into the A pieces in shared memory,
// one thread issues the MMAs, and after the commit the accumulator is read
// back with tcgen05.ld, staged in shared memory and written out as whole row
// segments (coalesced).  Rows of one tile
// are read completely before any is written, and tiles are disjoint, so the
// fold may run in place (out == X').
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kernels.cuh"

namespace svl {

namespace {

constexpr int RT_M = 128;          // rows per tile (MMA M, tensor-memory lanes)
constexpr int RT_THREADS = 256;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32x16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Pieces of the A operand: one for BF16 storage, three for FP32.
template <typename TS> struct APieces { static constexpr int n = 1; };
template <> struct APieces<float> { static constexpr int n = 3; };

// Shared layout of every operand piece (A tile: 128 rows; W^T: k rows), K
// padded to kp = a multiple of 64: the 128-byte-swizzled K-major layout of
// the MMA -- K atoms of 64 elements, each holding its rows 128 bytes apart,
// 8-row groups 1024 bytes apart, the 16-byte chunk c of row r stored at chunk
// c ^ (r % 8).  A warp writing one row's 128 bytes touches every bank once.
__device__ __forceinline__ uint32_t swz(int rows, int r, int c) {   // byte offset of element (r, c)
  const int atom = c >> 6, w = c & 63;
  return (uint32_t)(atom * rows * 128 + r * 128 + ((((w >> 3) ^ (r & 7)) << 4) | ((w & 7) << 1)));
}

// 128-byte-swizzle K-major descriptor: start, LBO 16 (unused for this
// layout), SBO 1024 (8-row groups), version 1, layout type 2 (SWIZZLE_128B)
__device__ __forceinline__ uint64_t sdesc128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

constexpr int RT_SLD = 36;   // staging row stride (floats): 32 columns + 4 (16-byte rows, 4 wavefronts per warp access)

// four consecutive outputs from an FP32 quadruple
__device__ __forceinline__ void store4(float* p, float4 x) { *(float4*)p = x; }
__device__ __forceinline__ void store4(double* p, float4 x) {
  ((double2*)p)[0] = make_double2(x.x, x.y);
  ((double2*)p)[1] = make_double2(x.z, x.w);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, float4 x) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(x.x, x.y), b = __floats2bfloat162_rn(x.z, x.w);
  *(uint2*)p = make_uint2(*(const uint32_t*)&a, *(const uint32_t*)&b);
}

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
  unsigned char* sm = (unsigned char*)(((uintptr_t)rt_raw + 1023) & ~(uintptr_t)1023);   // swizzle atoms: 1024-B aligned
  const int kp = (k + 63) & ~63;
  const uint32_t planeA = (uint32_t)RT_M * kp * 2, planeW = (uint32_t)k * kp * 2;
  unsigned char* Ap = sm;                        // NA pieces of the 128 x kp tile
  unsigned char* Wp = sm + (size_t)NA * planeA;   // 3 pieces of W^T (k x kp, row n = column n of W)
  float* stg = (float*)(Wp + 3 * (size_t)planeW); // 128 x RT_SLD FP32 staging of the output
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // W^T pieces: element (n, c) = W(c, n) = W[n k + c]; zero for c >= k
  for (int e = tid; e < k * kp; e += blockDim.x) {
    const int n = e / kp, c = e - n * kp;
    uint16_t p0 = 0, p1 = 0, p2 = 0;
    if (c < k) split3((float)W[(int64_t)n * k + c], p0, p1, p2);
    const uint32_t off = swz(k, n, c);
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
  constexpr int RPW = RT_M / (RT_THREADS / 32);   // rows per warp in the fill: 16
  // Rows of a tile: warp w loads rows w, w + 8, ... (lane l holds elements
  // 4l .. 4l + 3, k <= 128).  The next tile's loads are issued right after the
  // current tile's MMAs, so they are in flight during the MMAs and the
  // epilogue (software pipelining across tiles).
  using VL = typename std::conditional<sizeof(TS) == 4, float4, uint2>::type;   // 4 elements
  const bool act = 4 * lane < k;
  VL v[RPW];
  auto load_tile = [&](int64_t tl) {
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const int64_t gr = tl * RT_M + warp + 8 * i;
      if (act && gr < rows) v[i] = *reinterpret_cast<const VL*>(X + gr * k + 4 * lane);
      else memset(&v[i], 0, sizeof(VL));
    }
  };
  if ((int64_t)blockIdx.x < ntiles) load_tile(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t r0 = tile * RT_M;
    // ---- A pieces from the rows already in registers
    // rows warp + 8 i share r % 8, so their swizzled offsets differ by 1024 i
    const uint32_t off0 = swz(RT_M, warp, 4 * lane);
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      if (4 * lane < kp) {
        const uint32_t off = off0 + 1024u * (uint32_t)i;
        if constexpr (NA == 1) {
          *(uint2*)(Ap + off) = *(const uint2*)&v[i];
        } else {
          const float* f = (const float*)&v[i];
          uint16_t p[3][4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split3(f[e], p[0][e], p[1][e], p[2][e]);
#pragma unroll
          for (int a = 0; a < 3; ++a)
            *(uint2*)(Ap + (size_t)a * planeA + off) =
                make_uint2((uint32_t)p[a][0] | ((uint32_t)p[a][1] << 16), (uint32_t)p[a][2] | ((uint32_t)p[a][3] << 16));
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(Ap), w0 = su32(Wp);
      bool first = true;
      for (int ks = 0; ks < kp / 16; ++ks) {
        const uint32_t koff = (uint32_t)((ks & 3) * 32);   // byte offset of the K-step inside its atom
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int b = 0; b < 3 && a + b <= 3; ++b) {
            const uint64_t ad = sdesc128(a0 + a * planeA + (ks >> 2) * (RT_M * 128) + koff);
            const uint64_t bd = sdesc128(w0 + b * planeW + (ks >> 2) * (k * 128) + koff);
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
    // the next tile's rows: in place (out == X) they are other rows than this
    // tile's, so reading them before this tile is written is safe
    if (tile + gridDim.x < ntiles) load_tile(tile + gridDim.x);
    ok = __syncthreads_and(rt_wait(mb, phase) ? 1 : 0) != 0;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (tid == 0 && status) flag((int*)status, SVLCOV_DEV_TIMEOUT);
      rt_wait(mb, phase ^ 1u);   // the MMAs in flight, bounded again
      break;
    }
    // ---- epilogue, 32 columns per pass: warp w reads TMEM lanes 32 (w % 4) .. (rows)
    //      and 16 columns 16 (w / 4) .. of the pass into the staging tile (row-major,
    //      stride RT_SLD floats); then the warps write whole row segments: lane l
    //      takes row 4 i' + l / 8 of its rows and columns 4 (l % 8) .. + 3 (16-byte
    //      shared reads, coalesced global writes of 128 B per row)
    const int quad = warp & 3, half = warp >> 2;
    for (int c0 = 0; c0 < k; c0 += 32) {
      const int cc = c0 + 16 * half;
      if (cc < k) {
        float v[16];
        tmem_ld32x16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)cc, v);
        float* sg = stg + (32 * quad + lane) * RT_SLD + 16 * half;
#pragma unroll
        for (int j = 0; j < 4; ++j) *(float4*)(sg + 4 * j) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
      __syncthreads();
      const int nq = min(32, k - c0) / 4;   // float4 columns in this pass
      const int cq = lane & 7;
#pragma unroll
      for (int i = 0; i < RPW / 4; ++i) {
        const int r = warp * RPW + 4 * i + (lane >> 3);
        const int64_t gr = r0 + r;
        if (gr < rows && cq < nq) {
          const float4 x = *(const float4*)(stg + r * RT_SLD + 4 * cq);
          store4(out + gr * k + c0 + 4 * cq, x);
        }
      }
      __syncthreads();
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
  const int kp = (k + 63) & ~63;
  const size_t smem = (size_t)APieces<TS>::n * RT_M * kp * 2 + 3 * (size_t)k * kp * 2 +
                      (size_t)RT_M * RT_SLD * sizeof(float) + 1024;
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

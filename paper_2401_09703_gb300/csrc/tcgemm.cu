// FP64 products on the tensor cores: the small dense products of the mixed
// small-step mode (the folds of Section 3.2, C0 = W^T P, the CholeskyQR2
// Gram of the second pass, the refinement of SVD_k) at FP64 accuracy from
// BF16 tcgen05.mma with FP32 accumulation in tensor memory.
//
// Splitting (Ozaki, Ogita, Oishi & Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012): every row i of op(A) is
// written on the grid of its largest exponent E_i, a_ik = +-q_ik 2^(E_i-1075)
// with q_ik < 2^53 the significand shifted right by E_i - e(a_ik), and q_ik
// is cut into S = 8 digits of 7 bits, q = sum_s d_s 2^(46 - 7 s) (the last
// digit holds the lowest 4 bits, shifted left by 3: q is represented
// exactly).  Columns of op(B) the same with their own F_j.  Each digit is an integer of magnitude <= 127,
// exact in BF16, each digit product exact in FP32, and a sum of at most 1024
// of them stays below 2^24: so the tensor cores accumulate the partial
// product of every digit pair without rounding, in any order.  Pairs with
// the same s + t = g share the scale 2^(92 - 7 g + E_i + F_j - 2150) and one
// FP32 accumulator in tensor memory (8 groups x 64 columns fill the 512
// columns); pairs with s + t >= 8 are dropped (together below 2^-53 of the
// product of the row and column scales per term).  The epilogue turns the S exact
// integer accumulators into FP64 and sums them, smallest first.
//
// One CTA computes a 128 x 64 tile of C over a share of K (<= 1024).  Small
// products split K over a thread-block cluster, summed in rank order from
// distributed shared memory (deterministic).  Operands are digitised by all
// threads straight into shared memory in the no-swizzle K-major layout of
// the MMA (8-row x 16-byte core matrices); one thread issues the MMAs.
#include <cooperative_groups.h>

#include <algorithm>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace svl {

namespace {

constexpr int OZ_S = 8;        // digits per element; also the number of accumulator groups
constexpr int OZ_TM = 128;     // MMA M: rows of op(A) per CTA (tensor-memory lanes)
constexpr int OZ_TN = 64;      // MMA N: columns of op(B) per CTA
constexpr int OZ_KC = 64;      // K per shared-memory fill (4 MMAs of K = 16)
constexpr int OZ_KMAX = 1024;  // K per CTA keeping every accumulator exact (127^2 * 1024 < 2^24)
constexpr int OZ_THREADS = 256;
constexpr int OZ_TMEM_COLS = 512;  // >= OZ_S * OZ_TN, a power of two
constexpr uint32_t OZ_SBO = (OZ_KC / 8) * 128;          // bytes between 8-row groups
constexpr uint32_t OZ_ASLICE = (OZ_TM / 8) * OZ_SBO;    // one digit plane of the A tile
constexpr uint32_t OZ_BSLICE = (OZ_TN / 8) * OZ_SBO;
constexpr size_t OZ_SMEM = (size_t)OZ_S * (OZ_ASLICE + OZ_BSLICE) + 1024;  // + alignment slack
static_assert((size_t)OZ_TM * OZ_TN * sizeof(double) <= (size_t)OZ_S * (OZ_ASLICE + OZ_BSLICE),
              "the FP64 partial tile reuses the digit planes");
static_assert(OZ_S * OZ_TN <= OZ_TMEM_COLS, "tensor-memory columns");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05 for a no-swizzle K-major
// operand: start address, leading byte offset (between the two 16-byte core
// matrices along K of one MMA), stride byte offset (between 8-row groups),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_TN >> 3) << 17) |
                              ((uint32_t)(OZ_TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(ad), "l"(bd), "r"(OZ_IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
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

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
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

// Element (r, k) of op(X) for X column-major with leading dimension ld
// (trans: op(X) = X^T), zero outside rows x kend and outside the triangle
// that `tri` keeps (1: k >= r, 2: k <= r).
__device__ __forceinline__ uint64_t elem_bits(const double* X, int ld, bool trans, int r, int k, int rows, int kend,
                                              int tri) {
  if (r >= rows || k >= kend) return 0ull;
  if ((tri & 1) && k < r) return 0ull;
  if ((tri & 2) && k > r) return 0ull;
  const double v = trans ? X[(int64_t)r * ld + k] : X[(int64_t)k * ld + r];
  return (uint64_t)__double_as_longlong(v);
}

// The eight 7-bit digits of one element on the grid of exponent emax, as
// signed BF16 bit patterns (an integer d <= 127 has at most 7 significant
// bits, so its FP32 pattern shifted right by 16 is its exact BF16).
__device__ __forceinline__ void digits(uint64_t u, int emax, uint16_t* d) {
  const int e = (int)((u >> 52) & 0x7FF);
  uint64_t q = 0;
  if (e != 0 && e != 0x7FF) {               // zero, subnormal (flushed) and non-finite give no digits
    const int sh = emax - e;
    const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    q = sh < 53 ? (m >> sh) : 0ull;
  }
  const uint16_t sg = (uint16_t)((u >> 63) << 15);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    const uint32_t di = (uint32_t)(s < 7 ? (q >> (46 - 7 * s)) : (q << 3)) & 127u;
    d[s] = (uint16_t)(__float_as_uint((float)di) >> 16) | (di ? sg : (uint16_t)0);
  }
}

struct OzParams {
  int M, N, K;
  double alpha, beta;
  const double* A;
  int lda;
  const double* B;
  int ldb;
  double* C;
  int ldc;
  int ta, tb, tri;
  const int* status;
};

// Largest exponent field of each of the `rows` rows of an operand tile over
// [k0, k1) and whether a non-finite value occurs there.  Item = (row, group of
// 8 consecutive k).
__device__ void scan_rows(const double* X, int ld, bool trans, int row0, int rows_total, int k0, int k1, int tri,
                          int nrows, int* emax, int* bad) {
  const int ngroups = (k1 - k0 + 7) / 8;
  for (int it = threadIdx.x; it < nrows * ngroups; it += blockDim.x) {
    const int r = trans ? it / ngroups : it % nrows;   // the contiguous index varies fastest
    const int g = trans ? it % ngroups : it / nrows;
    int mx = 0, nf = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + 8 * g + j;
      const uint64_t u = elem_bits(X, ld, trans, row0 + r, k, rows_total, k1, tri);
      const int e = (int)((u >> 52) & 0x7FF);
      if (e == 0x7FF) nf = 1;
      else mx = max(mx, e);
    }
    if (mx) atomicMax(&emax[r], mx);
    if (nf) bad[r] = 1;
  }
}

// Digit planes of one K-chunk [kc, kc + OZ_KC) of an operand tile into
// shared memory: plane s at base + s * slice; element (r, k) of a plane at
// (r / 8) * OZ_SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
__device__ void fill_planes(const double* X, int ld, bool trans, int row0, int rows_total, int kc, int kend, int tri,
                            int nrows, const int* emax, unsigned char* base, uint32_t slice) {
  constexpr int NG = OZ_KC / 8;
  for (int it = threadIdx.x; it < nrows * NG; it += blockDim.x) {
    const int r = trans ? it / NG : it % nrows;
    const int g = trans ? it % NG : it / nrows;
    uint16_t d[8][OZ_S];
    const int em = emax[r];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      digits(elem_bits(X, ld, trans, row0 + r, kc + 8 * g + j, rows_total, kend, tri), em, d[j]);
    unsigned char* dst = base + (r >> 3) * OZ_SBO + g * 128 + (r & 7) * 16;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      uint4 v;
      v.x = (uint32_t)d[0][s] | ((uint32_t)d[1][s] << 16);
      v.y = (uint32_t)d[2][s] | ((uint32_t)d[3][s] << 16);
      v.z = (uint32_t)d[4][s] | ((uint32_t)d[5][s] << 16);
      v.w = (uint32_t)d[6][s] | ((uint32_t)d[7][s] << 16);
      *(uint4*)(dst + (size_t)s * slice) = v;
    }
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozaki_gemm(OzParams p) {
  extern __shared__ unsigned char oz_raw[];
  __shared__ int rexp[OZ_TM], rbad[OZ_TM], cexp[OZ_TN], cbad[OZ_TN];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_slot;
  // A failed step skips the product -- but only a CTA without cluster
  // partners may leave early: a kernel on another stream of the same step
  // could flag the status word between two CTAs' reads, and a CTA that left
  // would never reach the cluster barriers below.
  if (gridDim.z == 1 && p.status && failed(p.status)) return;
  unsigned char* sm = (unsigned char*)(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Ap = sm;
  unsigned char* Bp = sm + (size_t)OZ_S * OZ_ASLICE;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * OZ_TM, n0 = blockIdx.y * OZ_TN;
  const int ks = (int)gridDim.z, kz = (int)blockIdx.z;
  // K range where op(A) rows [m0, m0 + TM) and op(B) columns [n0, n0 + TN)
  // can both be nonzero (triangular operands), then this CTA's share of it
  int kbeg = 0, kend = p.K;
  if (p.tri & 1) kbeg = max(kbeg, m0);
  if (p.tri & 2) kend = min(kend, m0 + OZ_TM);
  if (p.tri & 4) kend = min(kend, n0 + OZ_TN);
  if (p.tri & 8) kbeg = max(kbeg, n0);
  kbeg = kbeg / OZ_KC * OZ_KC;
  {
    const int nch = kend > kbeg ? (kend - kbeg + OZ_KC - 1) / OZ_KC : 0;
    const int per = (nch + ks - 1) / ks;
    const int b0 = kbeg + kz * per * OZ_KC;
    kend = min(kend, b0 + per * OZ_KC);
    kbeg = b0;
  }
  const int nchunks = kend > kbeg ? (kend - kbeg + OZ_KC - 1) / OZ_KC : 0;
  const int triA = p.tri & 3;                                       // op(A): 1 k >= m, 2 k <= m
  const int triB = ((p.tri & 4) ? 2 : 0) | ((p.tri & 8) ? 1 : 0);   // op(B)^T row n, column k
  for (int i = tid; i < OZ_TM; i += blockDim.x) { rexp[i] = 0; rbad[i] = 0; }
  for (int i = tid; i < OZ_TN; i += blockDim.x) { cexp[i] = 0; cbad[i] = 0; }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(OZ_TMEM_COLS)
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
  const uint32_t tmem = tmem_slot;
  // op(B) is handled as its transpose (N x K, K-major like op(A)): element
  // (n, k) of op(B)^T is op(B)(k, n) = B[n ld + k] (no transpose) or B[k ld + n]
  const bool bt_trans = !p.tb;
  if (nchunks > 0) {
    scan_rows(p.A, p.lda, p.ta, m0, p.M, kbeg, kend, triA, OZ_TM, rexp, rbad);
    scan_rows(p.B, p.ldb, bt_trans, n0, p.N, kbeg, kend, triB, OZ_TN, cexp, cbad);
  }
  __syncthreads();
  const uint32_t mb = su32(&mbar);
  bool ok = true;
  int issued = 0;   // chunks whose MMAs were committed to the mbarrier
  for (int c = 0; c < nchunks; ++c) {
    const int kc = kbeg + c * OZ_KC;
    if (c > 0) {   // the previous chunk's MMAs have read the planes (uniform outcome)
      ok = __syncthreads_and(mbar_wait(mb, (uint32_t)((c - 1) & 1)) ? 1 : 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    fill_planes(p.A, p.lda, p.ta, m0, p.M, kc, kend, triA, OZ_TM, rexp, Ap, OZ_ASLICE);
    fill_planes(p.B, p.ldb, bt_trans, n0, p.N, kc, kend, triB, OZ_TN, cexp, Bp, OZ_BSLICE);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = su32(Ap), b0 = su32(Bp);
#pragma unroll 1
      for (int kk = 0; kk < OZ_KC / 16; ++kk) {
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
#pragma unroll
          for (int t = 0; t + s < OZ_S; ++t) {
            const int g = s + t;
            const uint64_t ad = sdesc(a0 + s * OZ_ASLICE + kk * 256, 128, OZ_SBO);
            const uint64_t bd = sdesc(b0 + t * OZ_BSLICE + kk * 256, 128, OZ_SBO);
            // the first product into accumulator g starts it: chunk 0, K-step 0, s = 0
            const uint32_t acc = (c > 0 || kk > 0 || s > 0) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(g * OZ_TN), ad, bd, acc);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    issued = c + 1;
  }
  if (ok && issued > 0) {
    ok = __syncthreads_and(mbar_wait(mb, (uint32_t)((issued - 1) & 1)) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok) {
    if (tid == 0 && p.status) flag((int*)p.status, SVLCOV_DEV_TIMEOUT);
    if (issued > 0) mbar_wait(mb, (uint32_t)((issued - 1) & 1));   // the MMAs in flight, bounded again
  }
  // ---- epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows), columns 32 (w / 4) .. + 31
  const int quad = warp & 3, half = warp >> 2;
  const int r = 32 * quad + (tid & 31);
  double out[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) out[j] = 0.0;
  if (issued > 0 && ok) {
    // Horner from the smallest group: out = sum_g acc_g 2^(-7 g)
#pragma unroll 1
    for (int g = OZ_S - 1; g >= 0; --g) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(g * OZ_TN + 32 * half), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) out[j] = fma(out[j], 0.0078125, (double)v[j]);
    }
    const int ei = rexp[r];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int cj = 32 * half + j;
      const int sh = 92 + ei + cexp[cj] - 2150;
      double x = ldexp(out[j], sh) * p.alpha;
      if (rbad[r] || cbad[cj]) x = __longlong_as_double(0x7FF8000000000000ll);   // NaN
      out[j] = x;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();   // every tensor-memory read is done; the digit planes are free
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  double* part = (double*)sm;   // FP64 partial tile [TN][TM] over the digit planes
  if (ks > 1) {
#pragma unroll
    for (int j = 0; j < 32; ++j) part[(size_t)(32 * half + j) * OZ_TM + r] = out[j];
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();   // every partial tile is in its CTA's shared memory
    if (kz == 0) {
#pragma unroll
      for (int j = 0; j < 32; ++j) out[j] = 0.0;
      for (int z = 0; z < ks; ++z) {
        const double* pz = cl.map_shared_rank(part, z);
#pragma unroll
        for (int j = 0; j < 32; ++j) out[j] += pz[(size_t)(32 * half + j) * OZ_TM + r];
      }
    }
    cl.sync();   // the others keep their shared memory until rank 0 has read it
    if (kz != 0) return;
  }
  const int gm = m0 + r;
  if (gm < p.M) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int gn = n0 + 32 * half + j;
      if (gn < p.N) {
        double* cp = p.C + (int64_t)gn * p.ldc + gm;
        *cp = p.beta == 0.0 ? out[j] : out[j] + p.beta * *cp;
      }
    }
  }
}

int g_sms = 0;

}  // namespace

// C (M x N) = alpha op(A) op(B) + beta C, FP64, column-major, on the tensor
// cores (digit splitting above).  tri: as for gemm().  The cluster split of K
// is chosen so that the tiles fill about one wave of the GPU, every CTA
// keeps at least one K-chunk and no CTA more than OZ_KMAX of K.
void ozaki_gemm(bool ta, bool tb, int M, int N, int Kd, double alpha, const double* A, int lda, const double* B,
                int ldb, double beta, double* C, int ldc, const int* status, cudaStream_t st, int tri) {
  if (M <= 0 || N <= 0) return;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 152;
    attr_done = true;
  }
  const int tm = (int)cdiv(M, OZ_TM), tn = (int)cdiv(N, OZ_TN);
  const int nch = (int)cdiv(std::max(Kd, 1), OZ_KC);
  int ks = (int)cdiv(nch * OZ_KC, OZ_KMAX);                  // exactness bound
  while (ks < 8 && ks < nch && (int64_t)tm * tn * ks * 2 <= g_sms) ks *= 2;
  ks = std::min(ks, std::min(8, nch));
  if ((int64_t)cdiv(nch, ks) * OZ_KC > OZ_KMAX) ks = (int)std::min<int64_t>(8, cdiv(nch * OZ_KC, OZ_KMAX));
  OzParams p{M, N, Kd, alpha, beta, A, lda, B, ldb, C, ldc, ta ? 1 : 0, tb ? 1 : 0, tri, status};
  note_launches(1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)tm, (unsigned)tn, (unsigned)ks);
  cfg.blockDim = dim3(OZ_THREADS);
  cfg.dynamicSmemBytes = OZ_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = (unsigned)ks;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_ozaki_gemm, p);
}

}  // namespace svl

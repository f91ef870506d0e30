// Rank-k SVD of a small dense matrix for callers that cannot allocate device
// memory.  Some callers may not call cudaMalloc at all: code that runs under
// another component's caching allocator (which owns every free byte and
// would be bypassed or starved by a raw cudaMalloc), or latency-sensitive
// code where cudaMalloc / cudaFree would synchronise the whole device.  For
// them svlcov_small_svd_static keeps its scratch in a fixed array compiled
// into this library instead of taking a caller-provided workspace.
//
// The scratch is one file-scope __device__ array; every GPU that loads the
// library holds its own copy until the process exits.  All calls on a device
// share it and it keeps the contents of the last call, so calls that overlap
// on the GPU (two streams, two host threads) race on it; calls must be
// serialised by the caller.
#include <mutex>

#include "kernels.cuh"

using namespace svl;

namespace {

// 8 MiB: the largest layout below (SVLCOV_SMALL_MIXED at n = k = 256, about
// 6 MB) fits; the size test at that bound keeps the two in step.
constexpr size_t kStaticScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_small_svd_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current, and cached.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SVLCOV_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SVLCOV_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_small_svd_scratch);
    if (e != cudaSuccess || p == nullptr) return SVLCOV_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SVLCOV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Offsets into the scratch array: status word | Jacobi work | then either the
// FP32 staging (SVLCOV_SMALL_FP32) or the FP64 refinement work
// (SVLCOV_SMALL_MIXED).  end is the bytes the call needs.
struct StaticLayout {
  size_t status = 0, jw = 0, kf = 0, ff = 0, gf = 0, tf = 0, rw = 0, end = 0;
  StaticLayout(int n, int k, int precision) {
    jw = align256(status + 4 * sizeof(int));
    size_t tail = align256(jw + jacobi_work_bytes(n));
    end = tail;
    if (precision == SVLCOV_SMALL_FP32) {
      kf = tail;
      ff = align256(kf + sizeof(float) * (size_t)n * n);
      gf = align256(ff + sizeof(float) * (size_t)n * k);
      tf = align256(gf + sizeof(float) * (size_t)n * k);
      end = tf + sizeof(float) * (size_t)k;
    } else if (precision == SVLCOV_SMALL_MIXED) {
      rw = tail;
      end = rw + refine_work_bytes(n, k);
    }
  }
};

}  // namespace

extern "C" int svlcov_small_svd_static(const double* K, int32_t n, int32_t k, double* F, double* theta, double* G,
                                       int32_t precision, int32_t* sweeps, void* stream) {
  if (!K || !F || !theta || !G || n <= 0 || k <= 0 || k > n) return SVLCOV_ERR_INVALID_ARG;
  if (precision != SVLCOV_SMALL_FP64 && precision != SVLCOV_SMALL_FP32 && precision != SVLCOV_SMALL_MIXED)
    return SVLCOV_ERR_INVALID_ARG;
  if (n > SVLCOV_SMALL_SVD_STATIC_MAX_N) return SVLCOV_ERR_CAPACITY;
  const StaticLayout L(n, k, precision);
  if (L.end > kStaticScratchBytes) return SVLCOV_ERR_CAPACITY;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != SVLCOV_OK) return rc;
  char* w = (char*)base;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)(w + L.status);
  void* jw = w + L.jw;
  // the array keeps the previous call's contents: clear the status word (the
  // Jacobi set-up kernel re-initialises its own counters and working copies,
  // and the refinement writes every buffer it reads)
  if (cudaMemsetAsync(status, 0, 4 * sizeof(int), st) != cudaSuccess) return SVLCOV_ERR_CUDA;
  int e = 0;
  if (precision == SVLCOV_SMALL_FP32) {
    float* Kf = (float*)(w + L.kf);
    float* Ff = (float*)(w + L.ff);
    float* Gf = (float*)(w + L.gf);
    float* tf = (float*)(w + L.tf);
    launch_cast<double, float>(K, Kf, (int64_t)n * n, st);
    e = launch_jacobi<float>(Kf, n, k, Ff, tf, Gf, jw, status, st);
    launch_cast<float, double>(Ff, F, (int64_t)n * k, st);
    launch_cast<float, double>(Gf, G, (int64_t)n * k, st);
    launch_cast<float, double>(tf, theta, k, st);
  } else if (precision == SVLCOV_SMALL_MIXED) {
    e = launch_mixed_svd(K, n, k, F, theta, G, jw, w + L.rw, status, st, nullptr);
  } else {
    e = launch_jacobi<double>(K, n, k, F, theta, G, jw, status, st);
  }
  if (e) return SVLCOV_ERR_CUDA;
  if (sweeps) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return SVLCOV_ERR_CUDA;
    int* sw = jacobi_sweeps_ptr(jw, n, precision == SVLCOV_SMALL_FP64 ? 8 : 4);
    if (cudaMemcpy(sweeps, sw, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SVLCOV_ERR_CUDA;
  }
  return last_launch();
}

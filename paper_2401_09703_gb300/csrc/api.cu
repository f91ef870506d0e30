// C ABI of the SV-LCOV GB300 library: handle, workspace layout and the launch
// sequence of one update step (Algorithms 3, 4 and 11 on the extended
// decomposition of Section 3.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"

using namespace svl;

namespace {

// ---- workspace carving ------------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T> T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct SideBufs {
  SideScratch sc;
  double *P, *SE, *C0, *e2, *S, *L1, *Y1, *T1, *S2, *L2, *Y2, *R, *X, *CQ, *Lm, *Y, *Mt;
  unsigned char *defl1, *defl2;
};

int log2_ceil(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}

}  // namespace

// Phase timing with CUDA events (enabled by svlcov_profile_enable).
// PH_JACOBI is nested inside PH_SVD: the sweep kernel alone (no set-up,
// extract or refinement), for the roofline of that kernel.
enum { PH_PREP = 0, PH_GATHER, PH_CHOLQR, PH_SVD, PH_FOLD, PH_APPLY, PH_JACOBI, PH_COUNT };

struct Prof {
  bool on = false;
  struct Rec {
    int ph;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  double ms[PH_COUNT] = {};
  int64_t calls[PH_COUNT] = {};
  int open = -1;
  void begin(int ph, cudaStream_t st) {
    if (!on) return;
    Rec r{ph, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, st);
    recs.push_back(r);
    open = (int)recs.size() - 1;
  }
  void end(cudaStream_t st) {
    if (!on || open < 0) return;
    cudaEventRecord(recs[open].b, st);
    open = -1;
  }
  void next(int ph, cudaStream_t st) {
    end(st);
    begin(ph, st);
  }
  // a nested record whose two events are recorded elsewhere (the Jacobi
  // launcher records them around the sweep kernel)
  bool nested(int ph, cudaEvent_t& a, cudaEvent_t& b) {
    if (!on) return false;
    Rec r{ph, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    recs.push_back(r);
    a = r.a;
    b = r.b;
    return true;
  }
  void resolve() {
    for (auto& r : recs) {
      float t = 0.f;
      cudaEventSynchronize(r.b);
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.ph] += t;
        calls[r.ph] += 1;
      } else {
        cudaGetLastError();   // a nested pair that was never recorded
      }
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    recs.clear();
  }
};

struct svlcov_handle {
  svlcov_init_desc d;
  Prof prof;
  int64_t m, n;  // host view of the shape
  int k;
  int64_t Hmax;
  // persistent device state
  int* status;
  int64_t* counters;  // [0] m, [1] n committed
  int64_t* resets;
  int64_t* stats;     // [0] Jacobi sweeps summed over launches
  int* flags;         // [0] reset_u, [1] reset_v
  double *Wu, *Wv, *sigma;
  // step scratch
  SideBufs side[2];
  double *K, *F, *G, *theta, *Xu, *Xv, *Wu_new, *Wv_new, *Wu_inv, *Wv_inv, *Nt, *Itmp;
  double* Itmp2;     // the second side's inverse scratch (the two folds run concurrently)
  cudaStream_t side_st = nullptr;   // the second fold's stream (forked from and joined into the step's)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double *K2, *G2;   // K with the empty batch vectors' columns moved last, and its right vectors
  int *perm, *nact;  // that column order (max_s) and k + the number of non-empty vectors
  void* jwork;
  void* rwork;  // FP64 refinement scratch of the mixed SVD
  void* rowork = nullptr;  // re-orthonormalisation scratch (when enabled)
  char* awork = nullptr;   // SVD_k of a one-vector step (secular equation), FP64 small modes
  // bookkeeping of the last step
  int last_op = -1, last_s = 0;
  bool last_rfree = false;   // the last step formed no R, K or F (mixed R-free route)
  int64_t steps = 0;  // steps enqueued (schedules the re-orthonormalisation)
};

// The handle's split-K setting for the FP64 products it enqueues (restored
// on leaving the entry point).
// The same scope sets where the handle's FP64 products run: on the tensor
// cores (ozaki_gemm) for the mixed small-step mode when the handle's
// tensor_gemm option is positive, else on the FP64 pipe.
// In the update steps (`step`) of that mode with the default tensor_gemm = 0
// and factors stored in FP32 / BF16, they run in double-float on the FP32
// pipe (gemm_df): ~2^-44 relative, far below the rounding of those factors --
// the larger products of a lone handle, all of them for handles that run side
// by side (gemm_split < 0), whose FP64 products fill the GPU.
struct SplitScope {
  explicit SplitScope(const svlcov_handle* h, bool step = false) {
    set_gemm_split(!h || h->d.gemm_split >= 0);
    set_gemm_tc(h && h->d.small == SVLCOV_SMALL_MIXED && h->d.tensor_gemm > 0);
    const bool df = step && h && h->d.small == SVLCOV_SMALL_MIXED && h->d.tensor_gemm == 0 &&
                    h->d.storage != SVLCOV_FP64;
    set_gemm_df(!df ? 0 : h->d.gemm_split < 0 ? 2 : 1);
  }
  ~SplitScope() {
    set_gemm_split(true);
    set_gemm_tc(false);
    set_gemm_df(0);
  }
};

// Re-orthonormalisation of the projected factor(s) before a step (see the
// init descriptor): on by default for BF16 storage, needs FP64 small factors.
static bool reorth_on(const svlcov_init_desc& d) {
  return d.small != SVLCOV_SMALL_FP32 && (d.reorth > 0 || (d.reorth == 0 && d.storage == SVLCOV_BF16));
}

static void layout(svlcov_handle* h, void* base, size_t* total) {
  const svlcov_init_desc& d = h->d;
  int64_t k = d.k, s = d.max_s, n2 = k + s, nnz = std::max<int64_t>(d.max_nnz, 1);
  int64_t H = h->Hmax, ch = max_chunks(s, nnz);
  Carver c(base);
  h->status = c.take<int>(4);
  h->counters = c.take<int64_t>(4);
  h->resets = c.take<int64_t>(2);
  h->stats = c.take<int64_t>(4);
  h->flags = c.take<int>(8);
  h->Wu = c.take<double>(k * k);
  h->Wv = c.take<double>(k * k);
  h->sigma = c.take<double>(k);
  for (int sd = 0; sd < 2; ++sd) {
    SideBufs& b = h->side[sd];
    b.sc.rowid = c.take<int>(nnz);
    b.sc.slot = c.take<int>(nnz);
    b.sc.rank_tmp = c.take<int>(nnz);
    b.sc.tmp_j = c.take<int>(nnz);
    b.sc.tmp_e = c.take<int>(nnz);
    b.sc.seg_j = c.take<int>(nnz);
    b.sc.seg_v = c.take<double>(nnz);
    b.sc.hkey = c.take<int>(H);
    b.sc.hcnt = c.take<int>(H);
    b.sc.hstart = c.take<int>(H);
    b.sc.occ = c.take<int>(H);
    b.sc.counts = c.take<int>(4);
    b.sc.chunk_off = c.take<int>(s + 1);
    b.sc.chunk_row = c.take<int>(ch);
    b.sc.Ppart = c.take<double>(ch * k);
    b.sc.SEpart = c.take<double>(ch * s);
    b.P = c.take<double>(k * s);
    b.SE = c.take<double>(s * s);
    b.C0 = c.take<double>(k * s);
    b.e2 = c.take<double>(s);
    b.S = c.take<double>(s * s);
    b.L1 = c.take<double>(s * s);
    b.Y1 = c.take<double>(s * s);
    b.T1 = c.take<double>(s * s);
    b.S2 = c.take<double>(s * s);
    b.L2 = c.take<double>(s * s);
    b.Y2 = c.take<double>(s * s);
    b.R = c.take<double>(s * s);
    b.X = c.take<double>(s * s);
    b.CQ = c.take<double>(k * s);
    b.Lm = c.take<double>(n2 * s);
    b.Y = c.take<double>(s * k);
    b.Mt = c.take<double>(k * s);
    b.defl1 = c.take<unsigned char>(s);
    b.defl2 = c.take<unsigned char>(s);
  }
  h->K = c.take<double>(n2 * n2);
  h->F = c.take<double>(n2 * k);
  h->G = c.take<double>(n2 * k);
  h->theta = c.take<double>(k);
  h->Xu = c.take<double>(k * k);
  h->Xv = c.take<double>(k * k);
  h->Wu_new = c.take<double>(k * k);
  h->Wv_new = c.take<double>(k * k);
  h->Wu_inv = c.take<double>(k * k);
  h->Wv_inv = c.take<double>(k * k);
  h->Nt = c.take<double>(k * s);
  h->Itmp = c.take<double>(2 * k * k);
  h->Itmp2 = c.take<double>(2 * k * k);
  h->K2 = c.take<double>(n2 * n2);
  h->G2 = c.take<double>(n2 * k);
  h->perm = c.take<int>(s);
  h->nact = c.take<int>(4);
  h->jwork = c.take<char>(jacobi_work_bytes((int)n2));
  h->rwork = c.take<char>(d.small == SVLCOV_SMALL_MIXED ? refine_work_bytes((int)n2, (int)k) : 256);
  h->rowork = reorth_on(d) ? c.take<char>(reorth_work_bytes((int)k, std::max(d.max_m, d.max_n))) : nullptr;
  h->awork = d.small != SVLCOV_SMALL_FP32 ? c.take<char>(arrow_work_bytes()) : nullptr;
  *total = (c.off + 255) & ~(size_t)255;
}

static bool desc_ok(const svlcov_init_desc* d) {
  if (!d) return false;
  if (d->k < 1 || d->k > SVLCOV_MAX_K) return false;
  if (d->max_s < 1 || d->max_s > SVLCOV_MAX_S) return false;
  if (d->m < 0 || d->n < 0 || d->max_m < d->m || d->max_n < d->n || d->max_nnz < 0) return false;
  if (d->storage < SVLCOV_FP64 || d->storage > SVLCOV_BF16) return false;
  if (d->jacobi_block > 16) return false;
  if (d->small < SVLCOV_SMALL_FP64 || d->small > SVLCOV_SMALL_MIXED) return false;
  if (d->reorth > 0 && d->small == SVLCOV_SMALL_FP32) return false;
  return true;
}

static bool small_is_f32(const svlcov_handle* h) { return h->d.small == SVLCOV_SMALL_FP32; }

// One-vector steps of the FP64 small modes take the secular-equation SVD_k
// and the scalar CholeskyQR (unless the handle's s1_secular option is < 0).
// FP64 Newton steps after the FP32 inverse of a guarded k x k factor (FP32 /
// BF16 storage, cond_1 <= 1e2 / 1e1 by default): one leaves ~(thr eps32)^2,
// below the rounding of the stored factors; FP64 storage keeps two.
static int inv_newton(const svlcov_handle* h) { return h->d.storage == SVLCOV_FP64 ? 2 : 1; }
// The FP32 sweeps and the first-order FP64 steps of the mixed SVD_k in an
// add step without R.  Each step squares the error of the leading vectors
// left by the sweeps.  FP64 storage: sweeps to 1e-3 off-diagonality and
// three steps, to FP64 rounding.  FP32 / BF16 storage: sweeps to 1e-2 and two
// steps, far below the rounding of the stored factors (the C2 trajectory of
// 196 node batches ends 2.5e-7 from the FP64 oracle with either setting).
static int refine_iters(const svlcov_handle* h) { return h->d.storage == SVLCOV_FP64 ? 3 : 2; }
static double sweep_stop(const svlcov_handle* h) { return h->d.storage == SVLCOV_FP64 ? 1e-3 : 1e-2; }
static bool s1_fast(const svlcov_handle* h) { return h->d.small != SVLCOV_SMALL_FP32 && h->d.s1_secular >= 0; }
// Add-columns / add-rows steps of the mixed mode that form no R (init option
// literal_steps): every s except the one-vector secular path.
static bool rfree(const svlcov_handle* h, int s) {
  return h->d.small == SVLCOV_SMALL_MIXED && h->d.literal_steps <= 0 && !(s == 1 && s1_fast(h));
}

extern "C" size_t svlcov_workspace_bytes(const svlcov_init_desc* d) {
  if (!desc_ok(d)) return 0;
  svlcov_handle tmp;
  tmp.d = *d;
  tmp.k = d->k;
  tmp.Hmax = (int64_t)1 << std::max(4, log2_ceil(2 * std::max<int64_t>(d->max_nnz, 1)));
  size_t total = 0;
  layout(&tmp, nullptr, &total);
  return total;
}

#define CUDA_OK(x)                                    \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return SVLCOV_ERR_CUDA;    \
  } while (0)


static void reorth_side(svlcov_handle* h, int side, cudaStream_t st) {
  const void* X = side == 0 ? h->d.ubuf : h->d.vbuf;
  int64_t rows = side == 0 ? h->m : h->n;
  double* W = side == 0 ? h->Wu : h->Wv;
  switch (h->d.storage) {
    case SVLCOV_FP64: launch_reorth<double>((const double*)X, rows, h->k, W, h->rowork, h->status, st); break;
    case SVLCOV_FP32: launch_reorth<float>((const float*)X, rows, h->k, W, h->rowork, h->status, st); break;
    default: launch_reorth<__nv_bfloat16>((const __nv_bfloat16*)X, rows, h->k, W, h->rowork, h->status, st);
  }
}

// sides: bit 0 U, bit 1 V
static void maybe_reorth(svlcov_handle* h, int sides, cudaStream_t st) {
  if (!h->rowork) return;
  int every = h->d.reorth > 0 ? h->d.reorth : 1;
  if (h->steps % every != 0) return;
  if (sides & 1) reorth_side(h, 0, st);
  if (sides & 2) reorth_side(h, 1, st);
}

template <typename TC>
static void init_small(svlcov_handle* h, cudaStream_t st) {
  launch_set_identity<TC>((TC*)h->Wu, h->k, st);
  launch_set_identity<TC>((TC*)h->Wv, h->k, st);
  if (sizeof(TC) == 8) cudaMemcpyAsync(h->sigma, h->d.sigma0, sizeof(double) * h->k, cudaMemcpyDeviceToDevice, st);
  else launch_cast<double, float>(h->d.sigma0, (float*)h->sigma, h->k, st);
}

template <typename TS>
static void init_factors(svlcov_handle* h, cudaStream_t st) {
  launch_convert_in<TS>(h->d.U0, h->d.init_dtype, (TS*)h->d.ubuf, h->d.m * h->d.k, st);
  launch_convert_in<TS>(h->d.V0, h->d.init_dtype, (TS*)h->d.vbuf, h->d.n * h->d.k, st);
}

extern "C" int svlcov_init(svlcov_handle** out, const svlcov_init_desc* d, void* stream) {
  if (!out || !desc_ok(d)) return SVLCOV_ERR_INVALID_ARG;
  if (!d->ubuf || !d->vbuf || !d->workspace || !d->sigma0) return SVLCOV_ERR_INVALID_ARG;
  if ((d->m > 0 && !d->U0) || (d->n > 0 && !d->V0)) return SVLCOV_ERR_INVALID_ARG;
  if (d->init_dtype != SVLCOV_FP64 && d->init_dtype != SVLCOV_FP32) return SVLCOV_ERR_INVALID_ARG;
  if (((uintptr_t)d->workspace & 255) != 0) return SVLCOV_ERR_INVALID_ARG;
  size_t need = svlcov_workspace_bytes(d);
  if (need == 0 || d->workspace_bytes < need) return SVLCOV_ERR_CAPACITY;
  svlcov_handle* h = new (std::nothrow) svlcov_handle();
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  h->d = *d;
  SplitScope split_scope(h);
  h->k = d->k;
  h->m = d->m;
  h->n = d->n;
  h->Hmax = (int64_t)1 << std::max(4, log2_ceil(2 * std::max<int64_t>(d->max_nnz, 1)));
  if (h->d.tau <= 0) h->d.tau = d->small == SVLCOV_SMALL_FP32 ? 1e-6 : 1e-12;
  if (h->d.reset_threshold <= 0)
    h->d.reset_threshold = d->storage == SVLCOV_FP64 ? 1e8 : (d->storage == SVLCOV_FP32 ? 1e2 : 1e1);
  size_t total = 0;
  layout(h, d->workspace, &total);
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(h->status, 0, sizeof(int) * 4, st);
  cudaMemsetAsync(h->resets, 0, sizeof(int64_t) * 2, st);
  cudaMemsetAsync(h->stats, 0, sizeof(int64_t) * 4, st);
  cudaMemsetAsync(h->flags, 0, sizeof(int) * 8, st);
  int64_t counters[4] = {d->m, d->n, 0, 0};
  cudaMemcpyAsync(h->counters, counters, sizeof(counters), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);  // the host array above must outlive the copy
  if (small_is_f32(h)) init_small<float>(h, st);
  else init_small<double>(h, st);
  if (d->storage == SVLCOV_FP64) init_factors<double>(h, st);
  else if (d->storage == SVLCOV_FP32) init_factors<float>(h, st);
  else init_factors<__nv_bfloat16>(h, st);
  if (h->rowork) {   // the rounding of the start to the storage type
    reorth_side(h, 0, st);
    reorth_side(h, 1, st);
  }
  if (last_launch() != SVLCOV_OK) {
    delete h;
    return SVLCOV_ERR_CUDA;
  }
  // the second fold's stream and its fork/join events; without them the two
  // folds run one after the other on the step's stream
  if (cudaStreamCreateWithFlags(&h->side_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h->side_st) cudaStreamDestroy(h->side_st);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    h->side_st = nullptr;
    h->ev_fork = h->ev_join = nullptr;
  }
  *out = h;
  return SVLCOV_OK;
}

extern "C" void svlcov_destroy(svlcov_handle* h) {
  if (!h) return;
  h->prof.resolve();
  if (h->side_st) cudaStreamDestroy(h->side_st);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
}

extern "C" int svlcov_profile_enable(svlcov_handle* h, int32_t enable) {
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  h->prof.on = enable != 0;
  return SVLCOV_OK;
}

extern "C" int svlcov_profile_read(svlcov_handle* h, double* ms, int64_t* calls, int32_t nphases, int32_t reset,
                                   int64_t* svd_sweeps) {
  if (!h || nphases < 0) return SVLCOV_ERR_INVALID_ARG;
  h->prof.resolve();
  if (svd_sweeps) {
    CUDA_OK(cudaDeviceSynchronize());
    CUDA_OK(cudaMemcpy(svd_sweeps, h->stats, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (reset) CUDA_OK(cudaMemset(h->stats, 0, sizeof(int64_t)));
  }
  for (int i = 0; i < nphases && i < PH_COUNT; ++i) {
    if (ms) ms[i] = h->prof.ms[i];
    if (calls) calls[i] = h->prof.calls[i];
  }
  if (reset)
    for (int i = 0; i < PH_COUNT; ++i) {
      h->prof.ms[i] = 0.0;
      h->prof.calls[i] = 0;
    }
  return SVLCOV_OK;
}

extern "C" uint64_t svlcov_kernel_launches(void) { return launches_total(); }

// ---------------------------------------------------------------------------
// One side of Algorithm 2 in the CholeskyQR2 form: from the batch, the
// projected factor X' and its small factor W, compute C0 = W^T X'^T E, the
// residual Gram S = E^T E - C0^T C0, R = R2 R1 and X = R^-1 (with dropped
// directions zeroed), and C_Q = C0 X (so that B = E X and Q = B - U C_Q).
// Turning the batch into SV-LCOV form (Lemmas 1-2): validation, the grouped
// view, C0 = W^T X'^T E, S_E = E^T E and the residual Gram S = S_E - C0^T C0.
template <typename TS, typename TC>
static void prepare_side(svlcov_handle* h, const svlcov_csr& b, int64_t d_len, const TS* Xp, const TC* W, SideBufs& sb,
                         cudaStream_t st) {
  int k = h->k, s = b.rows;
  int* status = h->status;
  h->prof.begin(PH_PREP, st);
  launch_validate(b, d_len, sb.sc.rowid, status, st);
  int logH = std::max(4, log2_ceil(2 * std::max<int64_t>(b.nnz, 1)));
  launch_group(b, logH, sb.sc, status, st);
  TC *P = (TC*)sb.P, *SE = (TC*)sb.SE, *C0 = (TC*)sb.C0, *e2 = (TC*)sb.e2;
  h->prof.next(PH_GATHER, st);
  launch_gather_gram<TS, TC>(b, Xp, k, W, sb.sc, P, SE, C0, e2, status, st);
  h->prof.next(PH_CHOLQR, st);
  TC* S = (TC*)sb.S;
  launch_copy<TC>(SE, S, (int64_t)s * s, status, st);
  gemm<TC>(true, false, s, s, k, (TC)-1, C0, k, C0, k, (TC)1, S, s, status, st);        // S = S_E - C0^T C0
}

// Independent branches of a step (the two folds, the two sides of the apply
// phase, R and X = R^-1 of CholeskyQR2, the orthogonality product of the
// refinement) share no buffer but the status word, so one of them runs on the
// handle's side stream, forked from the step's stream and joined back into it
// (capturable in a CUDA graph like any fork/join).
// svlcov_batch_run turns the fork off while it enqueues: its handles already
// run side by side, and the extra event calls slowed the host-bound eager
// enqueue of many handles (148k -> 118k update vectors/s at 64 matrices).
static thread_local bool t_side_fork = true;

struct SideFork {
  svlcov_handle* h;
  cudaStream_t st;
  bool on;
  SideFork(svlcov_handle* hh, cudaStream_t s0) : h(hh), st(s0), on(hh->side_st != nullptr && t_side_fork) {
    if (on) {
      cudaEventRecord(h->ev_fork, st);
      cudaStreamWaitEvent(h->side_st, h->ev_fork, 0);
    }
  }
  cudaStream_t stream() const { return on ? h->side_st : st; }
  ~SideFork() {
    if (on) {
      cudaEventRecord(h->ev_join, h->side_st);
      cudaStreamWaitEvent(st, h->ev_join, 0);
    }
  }
};

template <typename TS, typename TC>
static void orthogonalise(svlcov_handle* h, const svlcov_csr& b, int64_t d_len, const TS* Xp, const TC* W, SideBufs& sb,
                          cudaStream_t st, bool r_free = false) {
  int k = h->k, s = b.rows;
  int* status = h->status;
  prepare_side<TS, TC>(h, b, d_len, Xp, W, sb, st);
  if (s == 1 && s1_fast(h)) {
    // one vector: Algorithm 2 is one normalisation, R = sqrt(S) with the
    // deflation rule, X = 1 / R, C_Q = C0 X, in FP64 (one launch)
    launch_s1_orth((const double*)sb.S, (const double*)sb.e2, (const double*)sb.C0, k, h->d.tau, (double*)sb.R,
                   (double*)sb.X, (double*)sb.CQ, sb.defl1, sb.defl2, status, st);
    h->prof.end(st);
    return;
  }
  TC *C0 = (TC*)sb.C0, *e2 = (TC*)sb.e2;
  TC *S = (TC*)sb.S, *L1 = (TC*)sb.L1, *Y1 = (TC*)sb.Y1, *T1 = (TC*)sb.T1, *S2 = (TC*)sb.S2;
  TC *L2 = (TC*)sb.L2, *Y2 = (TC*)sb.Y2, *R = (TC*)sb.R, *X = (TC*)sb.X, *CQ = (TC*)sb.CQ;
  TC tau = (TC)h->d.tau;
  // Scratch of the blocked factorization (batches wider than one CTA's
  // shared memory holds): pass 1 works on a copy of S in S2 (not yet
  // formed), pass 2 on a copy of S2 in S (no longer needed); T1 is free
  // during both.
  if (h->d.small == SVLCOV_SMALL_MIXED) {
    // Pass 1 in FP32 (its pivots resolve only down to ~eps32, hence the
    // FP32 deflation threshold), the pass-2 Gram in FP64, pass 2 in FP32 on
    // the small deviation from the identity (delta form).
    double* Sd = (double*)S;
    double tau1 = std::max(h->d.tau, 1e-6);
    launch_cholinv<float, double, false>(Sd, s, (const double*)e2, (float)tau1, (double*)L1, (double*)Y1, sb.defl1,
                                         (double*)S2, (double*)T1, status, st, r_free);
    if (r_free) {   // L1 (S = L1 L1^T to FP32) is all an R-free add step needs
      h->prof.end(st);
      return;
    }
    gemm<TC>(false, true, s, s, s, (TC)1, S, s, Y1, s, (TC)0, T1, s, status, st, TRI_B_UP);   // T1 = S Y1^T
    gemm<TC>(false, false, s, s, s, (TC)1, Y1, s, T1, s, (TC)0, S2, s, status, st, TRI_A_LO);  // S2 = Y1 S Y1^T
    launch_cholinv<float, double, true>((double*)S2, s, nullptr, (float)h->d.tau, (double*)L2, (double*)Y2,
                                        sb.defl2, (double*)S, (double*)T1, status, st);
    // X = Y1^T Y2^T is R^-1 to ~eps32^2 cond(S), but R2 R1 = L2^T L1^T is not
    // its inverse: Y1 is an FP32 inverse of L1, off by ~eps32 cond(S), and
    // that error would enter K.  The R consistent with the X the folds use is
    // R = Q^T (E - U C0) = X^T S (upper triangular up to ~eps32^2 cond(S)),
    // from S formed again (pass 2 clobbered it; its Gram in S2 is no longer
    // needed) in FP64.
    {
      SideFork fk(h, st);
      gemm<TC>(true, true, s, s, s, (TC)1, Y1, s, Y2, s, (TC)0, X, s, status, fk.stream(),
               TRI_A_UP | TRI_B_UP);                                                                    // X = Y1^T Y2^T
      launch_copy<TC>((TC*)sb.SE, S2, (int64_t)s * s, status, st);
      gemm<TC>(true, false, s, s, k, (TC)-1, C0, k, C0, k, (TC)1, S2, s, status, st);          // S = S_E - C0^T C0
    }
    gemm<TC>(true, false, s, s, s, (TC)1, X, s, S2, s, (TC)0, R, s, status, st, TRI_A_LO);          // R = X^T S
    launch_triu((double*)R, s, status, st);
    gemm<TC>(false, false, k, s, s, (TC)1, C0, k, X, s, (TC)0, CQ, k, status, st, TRI_B_UP);       // C_Q = C0 X
    h->prof.end(st);
    return;
  } else {
    launch_cholinv<TC, TC, false>(S, s, e2, tau, L1, Y1, sb.defl1, S2, T1, status, st);         // S = L1 L1^T, Y1 = L1^-1
    gemm<TC>(false, true, s, s, s, (TC)1, S, s, Y1, s, (TC)0, T1, s, status, st, TRI_B_UP);   // T1 = S Y1^T
    gemm<TC>(false, false, s, s, s, (TC)1, Y1, s, T1, s, (TC)0, S2, s, status, st, TRI_A_LO);  // S2 = Y1 S Y1^T
    launch_cholinv<TC, TC, false>(S2, s, nullptr, tau, L2, Y2, sb.defl2, S, T1, status, st);    // S2 = L2 L2^T
  }
  {
    SideFork fk(h, st);
    gemm<TC>(true, true, s, s, s, (TC)1, L2, s, L1, s, (TC)0, R, s, status, fk.stream(),
             TRI_A_UP | TRI_B_UP);                                                                    // R = L2^T L1^T
    gemm<TC>(true, true, s, s, s, (TC)1, Y1, s, Y2, s, (TC)0, X, s, status, st, TRI_A_UP | TRI_B_UP);  // X = Y1^T Y2^T
    gemm<TC>(false, false, k, s, s, (TC)1, C0, k, X, s, (TC)0, CQ, k, status, st, TRI_B_UP);           // C_Q = C0 X
  }
  h->prof.end(st);
}

// Fold of one projected side (Section 3.2): Xn = W (Fk - C_Q Fs), Winv, and
// Mt = (X Fs Xn^-1)^T, the rows added to X' at the batch's touched rows.
template <typename TC>
static void fold_projected(svlcov_handle* h, SideBufs& sb, const TC* W, const TC* Fbig, int n2, int s, TC* Xtmp,
                           TC* Wn, TC* Winv, int* reset_flag, TC* itmp, cudaStream_t st) {
  int k = h->k;
  int* status = h->status;
  launch_copy2d<TC>(Fbig, n2, Xtmp, k, k, k, status, st);                                             // Fk
  gemm<TC>(false, false, k, k, s, (TC)-1, (TC*)sb.CQ, k, Fbig + k, n2, (TC)1, Xtmp, k, status, st);  // - C_Q Fs
  gemm<TC>(false, false, k, k, k, (TC)1, W, k, Xtmp, k, (TC)0, Wn, k, status, st);
  launch_inverse<TC>(Wn, k, Winv, h->d.reset_threshold, reset_flag, status, st, itmp,
                    inv_newton(h));
  gemm<TC>(false, false, s, k, s, (TC)1, (TC*)sb.X, s, Fbig + k, n2, (TC)0, (TC*)sb.Y, s, status, st);
  gemm<TC>(true, true, k, s, k, (TC)1, Winv, k, (TC*)sb.Y, s, (TC)0, (TC*)sb.Mt, k, status, st);
}

// The same fold without R (mixed R-free steps): Xn = W diag(Sigma) G[:k]
// Theta^-1 and Mt = (G[k:] Theta^-1 Xn^-1)^T, from K G = F Theta.
static void fold_projected_rfree(svlcov_handle* h, SideBufs& sb, const double* W, const double* G, int s, double* Xtmp,
                                 double* Wn, double* Winv, int* reset_flag, double* itmp, cudaStream_t st) {
  int k = h->k;
  int* status = h->status;
  launch_rfree_fold_inputs((const double*)h->sigma, G, (const double*)h->theta, k, s, Xtmp, (double*)sb.Y, status,
                           st);
  gemm<double>(false, false, k, k, k, 1.0, W, k, Xtmp, k, 0.0, Wn, k, status, st);
  launch_inverse<double>(Wn, k, Winv, h->d.reset_threshold, reset_flag, status, st, itmp,
                    inv_newton(h));
  gemm<double>(true, true, k, s, k, 1.0, Winv, k, (double*)sb.Y, s, 0.0, (double*)sb.Mt, k, status, st);
}

// SVD_k of the Rayleigh-Ritz matrix: Jacobi in the small-step precision, or
// FP32 sweeps + FP64 refinement in the mixed mode.
template <typename TC>
static int small_svd_step(svlcov_handle* h, const TC* K, int n2, TC* F, TC* theta, TC* G, cudaStream_t st,
                          const int* n_active = nullptr) {
  cudaEvent_t ja = nullptr, jb = nullptr;
  if (h->prof.nested(PH_JACOBI, ja, jb)) set_jacobi_events(ja, jb);
  int e;
  if (h->d.small == SVLCOV_SMALL_MIXED) {
    const bool fk = t_side_fork && h->side_st;
    e = launch_mixed_svd((const double*)K, n2, h->k, (double*)F, (double*)theta, (double*)G, h->jwork, h->rwork,
                         h->status, st, h->stats, h->d.jacobi_block, n_active, fk ? h->side_st : nullptr,
                         fk ? h->ev_fork : nullptr, fk ? h->ev_join : nullptr);
  }
  else
    e = launch_jacobi<TC>(K, n2, h->k, F, theta, G, h->jwork, h->status, st, h->stats, h->d.jacobi_block,
                          n_active);
  set_jacobi_events(nullptr, nullptr);
  return e;
}

template <typename TS, typename TC>
static int step_add(svlcov_handle* h, const svlcov_csr& b, bool cols, cudaStream_t st) {
  int k = h->k, s = b.rows, n2 = k + s;
  int* status = h->status;
  SideBufs& sb = h->side[0];
  // projected side P and appended side O
  TS* XpP = (TS*)(cols ? h->d.ubuf : h->d.vbuf);
  TS* XpO = (TS*)(cols ? h->d.vbuf : h->d.ubuf);
  TC* WP = (TC*)(cols ? h->Wu : h->Wv);
  TC* WO = (TC*)(cols ? h->Wv : h->Wu);
  TC* WPn = (TC*)(cols ? h->Wu_new : h->Wv_new);
  TC* WOn = (TC*)(cols ? h->Wv_new : h->Wu_new);
  TC* WPi = (TC*)(cols ? h->Wu_inv : h->Wv_inv);
  TC* WOi = (TC*)(cols ? h->Wv_inv : h->Wu_inv);
  int* rP = h->flags + (cols ? 0 : 1);
  int* rO = h->flags + (cols ? 1 : 0);
  int64_t rowsP = cols ? h->m : h->n, rowsO = cols ? h->n : h->m;
  const bool rf = rfree(h, s);
  orthogonalise<TS, TC>(h, b, rowsP, XpP, WP, sb, st, rf);
  TC *K = (TC*)h->K, *F = (TC*)h->F, *G = (TC*)h->G, *theta = (TC*)h->theta;
  h->prof.begin(PH_SVD, st);
  if (rf) {
    // R-free mixed step: FP32 sweeps on [[Sigma, C0], [0, L1^T]], FP64
    // refinement on K^T K = [[Sigma^2, Sigma C0], [C0^T Sigma, S_E]] (held in
    // the K buffer), both with the empty batch vectors' columns moved last.
    launch_active_columns(b.indptr, s, k, h->perm, h->nact, status, st);
    launch_build_K_chol((const double*)h->sigma, (const double*)sb.C0, (const double*)sb.L1, k, s, h->perm,
                        (double*)h->K2, status, st);
    launch_build_M((const double*)h->sigma, (const double*)sb.C0, (const double*)sb.SE, k, s, h->perm, (double*)K,
                   status, st);
    cudaEvent_t ja = nullptr, jb = nullptr;
    if (h->prof.nested(PH_JACOBI, ja, jb)) set_jacobi_events(ja, jb);
    const bool fk = t_side_fork && h->side_st;
    int e = launch_mixed_svd_gram((const double*)h->K2, (const double*)K, n2, k, (double*)theta, (double*)h->G2,
                                  h->jwork, h->rwork, status, st, h->stats, h->d.jacobi_block, h->nact,
                                  fk ? h->side_st : nullptr, fk ? h->ev_fork : nullptr, fk ? h->ev_join : nullptr,
                                  refine_iters(h), sweep_stop(h));
    set_jacobi_events(nullptr, nullptr);
    if (e) return SVLCOV_ERR_CUDA;
    launch_unpermute_rows<TC>((TC*)h->G2, n2, k, k, h->perm, G, status, st);
  } else if (s == 1 && s1_fast(h)) {
    launch_build_K_add<TC>((TC*)h->sigma, (TC*)sb.C0, (TC*)sb.R, k, s, K, status, st);    // K = [[S, C0],[0, R]]
    // K K^T = diag(S^2, 0) + z z^T with z = [C0; R]: the secular-equation SVD
    launch_arrow_svd((const double*)h->sigma, (const double*)sb.C0, (const double*)sb.R, k, (double*)F,
                     (double*)theta, (double*)G, h->awork, status, st);
  } else {
    launch_build_K_add<TC>((TC*)h->sigma, (TC*)sb.C0, (TC*)sb.R, k, s, K, status, st);    // K = [[S, C0],[0, R]]
    // Empty update vectors give zero columns of K: move them last so that the
    // Jacobi's tournament skips them (exact: their right vectors are unit vectors
    // with zero singular values), then put G's rows back in the batch order.
    launch_active_columns(b.indptr, s, k, h->perm, h->nact, status, st);
    launch_permute_cols<TC>(K, n2, k, h->perm, (TC*)h->K2, status, st);
    int e = small_svd_step<TC>(h, (TC*)h->K2, n2, F, theta, (TC*)h->G2, st, h->nact);   // F, Theta, G = SVD_k(K)
    if (e) return SVLCOV_ERR_CUDA;
    launch_unpermute_rows<TC>((TC*)h->G2, n2, k, k, h->perm, G, status, st);
  }
  h->prof.next(PH_FOLD, st);
  {
    SideFork fk(h, st);
    const cudaStream_t so = fk.stream();
    gemm<TC>(false, false, k, k, k, (TC)1, WO, k, G, n2, (TC)0, WOn, k, status, so);      // W_O G[:k]
    launch_inverse<TC>(WOn, k, WOi, h->d.reset_threshold, rO, status, so, (TC*)h->Itmp2,
                      inv_newton(h));
    gemm<TC>(true, true, k, s, k, (TC)1, WOi, k, G + k, n2, (TC)0, (TC*)h->Nt, k, status, so);  // (G[k:] W_O^-1)^T
    if (rf)
      fold_projected_rfree(h, sb, (const double*)WP, (const double*)G, s, (double*)h->Xu, (double*)WPn,
                           (double*)WPi, rP, (double*)h->Itmp, st);
    else
      fold_projected<TC>(h, sb, WP, F, n2, s, (TC*)h->Xu, WPn, WPi, rP, (TC*)h->Itmp, st);
  }
  FiniteSet<TC> fs{};
  fs.ptr[0] = theta; fs.count[0] = k;
  fs.ptr[1] = (TC*)sb.Mt; fs.count[1] = (int64_t)k * s;
  fs.ptr[2] = (TC*)h->Nt; fs.count[2] = (int64_t)k * s;
  fs.ptr[3] = WPn; fs.count[3] = (int64_t)k * k;
  fs.ptr[4] = WOn; fs.count[4] = (int64_t)k * k;
  fs.n = 5;
  h->prof.next(PH_APPLY, st);
  launch_check_finite_multi<TC>(fs, status, st);
  {
    SideFork fk(h, st);
    launch_reset<TS, TC>(XpO, rowsO, k, WOn, rO, status, fk.stream());
    launch_append<TS, TC>(XpO, rowsO, k, s, (TC*)h->Nt, status, fk.stream());
    launch_reset<TS, TC>(XpP, rowsP, k, WPn, rP, status, st);   // only when the guard fired
    launch_scatter<TS, TC>(XpP, k, (TC*)sb.Mt, b.nnz, sb.sc, status, st);
  }
  if (cols)
    launch_commit<TC>((TC*)h->Wu, WPn, rP, (TC*)h->Wv, WOn, rO, (TC*)h->sigma, theta, k, h->counters, 0, s,
                      h->resets, status, st);
  else
    launch_commit<TC>((TC*)h->Wu, WOn, rO, (TC*)h->Wv, WPn, rP, (TC*)h->sigma, theta, k, h->counters, s, 0,
                      h->resets, status, st);
  h->prof.end(st);
  return last_launch();
}

template <typename TS, typename TC>
static int step_weights(svlcov_handle* h, const svlcov_csr& D, const svlcov_csr& E, cudaStream_t st) {
  int k = h->k, s = D.rows, n2 = k + s;
  int* status = h->status;
  SideBufs& sd = h->side[0];
  SideBufs& se = h->side[1];
  orthogonalise<TS, TC>(h, D, h->m, (TS*)h->d.ubuf, (TC*)h->Wu, sd, st);
  orthogonalise<TS, TC>(h, E, h->n, (TS*)h->d.vbuf, (TC*)h->Wv, se, st);
  TC *K = (TC*)h->K, *F = (TC*)h->F, *G = (TC*)h->G, *theta = (TC*)h->theta;
  h->prof.begin(PH_SVD, st);
  launch_build_L<TC>((TC*)sd.C0, (TC*)sd.R, k, s, (TC*)sd.Lm, status, st);
  launch_build_L<TC>((TC*)se.C0, (TC*)se.R, k, s, (TC*)se.Lm, status, st);
  gemm<TC>(false, true, n2, n2, s, (TC)1, (TC*)sd.Lm, n2, (TC*)se.Lm, n2, (TC)0, K, n2, status, st);
  launch_add_diag<TC>(K, n2, (TC*)h->sigma, k, status, st);   // K = diag(S,0) + [C0D;RD][C0E;RE]^T
  int e = small_svd_step<TC>(h, K, n2, F, theta, G, st);
  if (e) return SVLCOV_ERR_CUDA;
  h->prof.next(PH_FOLD, st);
  {
    SideFork fk(h, st);
    fold_projected<TC>(h, se, (TC*)h->Wv, G, n2, s, (TC*)h->Xv, (TC*)h->Wv_new, (TC*)h->Wv_inv, h->flags + 1,
                       (TC*)h->Itmp2, fk.stream());
    fold_projected<TC>(h, sd, (TC*)h->Wu, F, n2, s, (TC*)h->Xu, (TC*)h->Wu_new, (TC*)h->Wu_inv, h->flags + 0,
                       (TC*)h->Itmp, st);
  }
  FiniteSet<TC> fs{};
  fs.ptr[0] = theta; fs.count[0] = k;
  fs.ptr[1] = (TC*)sd.Mt; fs.count[1] = (int64_t)k * s;
  fs.ptr[2] = (TC*)se.Mt; fs.count[2] = (int64_t)k * s;
  fs.ptr[3] = (TC*)h->Wu_new; fs.count[3] = (int64_t)k * k;
  fs.ptr[4] = (TC*)h->Wv_new; fs.count[4] = (int64_t)k * k;
  fs.n = 5;
  h->prof.next(PH_APPLY, st);
  launch_check_finite_multi<TC>(fs, status, st);
  launch_reset<TS, TC>((TS*)h->d.ubuf, h->m, k, (TC*)h->Wu_new, h->flags + 0, status, st);
  launch_scatter<TS, TC>((TS*)h->d.ubuf, k, (TC*)sd.Mt, D.nnz, sd.sc, status, st);
  launch_reset<TS, TC>((TS*)h->d.vbuf, h->n, k, (TC*)h->Wv_new, h->flags + 1, status, st);
  launch_scatter<TS, TC>((TS*)h->d.vbuf, k, (TC*)se.Mt, E.nnz, se.sc, status, st);
  launch_commit<TC>((TC*)h->Wu, (TC*)h->Wu_new, h->flags + 0, (TC*)h->Wv, (TC*)h->Wv_new, h->flags + 1,
                    (TC*)h->sigma, theta, k, h->counters, 0, 0, h->resets, status, st);
  h->prof.end(st);
  return last_launch();
}

template <typename TC>
static int dispatch_add(svlcov_handle* h, const svlcov_csr& b, bool cols, cudaStream_t st) {
  switch (h->d.storage) {
    case SVLCOV_FP64: return step_add<double, TC>(h, b, cols, st);
    case SVLCOV_FP32: return step_add<float, TC>(h, b, cols, st);
    default: return step_add<__nv_bfloat16, TC>(h, b, cols, st);
  }
}

template <typename TC>
static int dispatch_weights(svlcov_handle* h, const svlcov_csr& D, const svlcov_csr& E, cudaStream_t st) {
  switch (h->d.storage) {
    case SVLCOV_FP64: return step_weights<double, TC>(h, D, E, st);
    case SVLCOV_FP32: return step_weights<float, TC>(h, D, E, st);
    default: return step_weights<__nv_bfloat16, TC>(h, D, E, st);
  }
}

static bool csr_ok(const svlcov_csr* b) {
  if (!b) return false;
  if (b->rows < 0 || b->cols < 0 || b->nnz < 0) return false;
  if (b->values_dtype != SVLCOV_FP64 && b->values_dtype != SVLCOV_FP32) return false;
  if (b->rows > 0 && !b->indptr) return false;
  if (b->nnz > 0 && (!b->indices || !b->values)) return false;
  return true;
}

static int do_add(svlcov_handle* h, const svlcov_csr* b, bool cols, void* stream) {
  if (!h || !csr_ok(b)) return SVLCOV_ERR_INVALID_ARG;
  int64_t d_len = cols ? h->m : h->n;
  if (b->cols != d_len) return SVLCOV_ERR_INVALID_ARG;
  if (b->rows > h->d.max_s || b->nnz > h->d.max_nnz) return SVLCOV_ERR_CAPACITY;
  if (cols ? (h->n + b->rows > h->d.max_n) : (h->m + b->rows > h->d.max_m)) return SVLCOV_ERR_CAPACITY;
  if (b->rows == 0) return SVLCOV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  maybe_reorth(h, cols ? 1 : 2, st);
  int rc = small_is_f32(h) ? dispatch_add<float>(h, *b, cols, st) : dispatch_add<double>(h, *b, cols, st);
  if (rc == SVLCOV_OK) {
    if (cols) h->n += b->rows;
    else h->m += b->rows;
    h->last_op = cols ? 0 : 1;
    h->last_s = b->rows;
    h->last_rfree = rfree(h, b->rows);
    ++h->steps;
  }
  return rc;
}

extern "C" int svlcov_add_cols(svlcov_handle* h, const svlcov_csr* Ec_T, void* stream) {
  SplitScope split_scope(h, true);
  return do_add(h, Ec_T, true, stream);
}

extern "C" int svlcov_add_rows(svlcov_handle* h, const svlcov_csr* Er, void* stream) {
  SplitScope split_scope(h, true);
  return do_add(h, Er, false, stream);
}

extern "C" int svlcov_update_weights(svlcov_handle* h, const svlcov_csr* D_T, const svlcov_csr* Em_T, void* stream) {
  SplitScope split_scope(h, true);
  if (!h || !csr_ok(D_T) || !csr_ok(Em_T)) return SVLCOV_ERR_INVALID_ARG;
  if (D_T->cols != h->m || Em_T->cols != h->n || D_T->rows != Em_T->rows) return SVLCOV_ERR_INVALID_ARG;
  if (D_T->rows > h->d.max_s || D_T->nnz > h->d.max_nnz || Em_T->nnz > h->d.max_nnz) return SVLCOV_ERR_CAPACITY;
  if (D_T->rows == 0) return SVLCOV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  maybe_reorth(h, 3, st);
  int rc = small_is_f32(h) ? dispatch_weights<float>(h, *D_T, *Em_T, st)
                           : dispatch_weights<double>(h, *D_T, *Em_T, st);
  if (rc == SVLCOV_OK) {
    h->last_op = 2;
    h->last_s = D_T->rows;
    h->last_rfree = false;
    ++h->steps;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Approximate augmented space (the -GKL / -RPI variants, Appendix algorithms
// "Add columns / Update weights with approximated augmented space").  The
// caller's scratch holds, per projected side, the l-vector basis (W the
// coefficients of Q = E W - U (C0 W), P = Z^T Q) and the step's small dense
// matrices; the rest of the step uses the handle's workspace as the exact
// step does.
namespace {
struct ApproxSide {
  double *P, *W, *T, *T2, *W2, *TE, *Pm, *wr, *u, *ab, *G, *L, *Y, *Aw, *Tw, *e2, *Cq, *Lr;
  unsigned char* defl;
};
struct ApproxBufs {
  ApproxSide side[2];
  double *M, *Lm, *Ym, *Awm, *Twm, *GL;
  unsigned char* deflm;
};
void approx_layout(void* base, int k, int s, int l, ApproxBufs& ab, size_t* total) {
  Carver c(base);
  int64_t n = k + l;
  for (int sd = 0; sd < 2; ++sd) {
    ApproxSide& a = ab.side[sd];
    a.P = c.take<double>((int64_t)s * l);
    a.W = c.take<double>((int64_t)s * l);
    a.T = c.take<double>((int64_t)s * l);
    a.T2 = c.take<double>((int64_t)s * l);
    a.W2 = c.take<double>((int64_t)s * l);
    a.TE = c.take<double>((int64_t)s * l);
    a.Pm = c.take<double>((int64_t)s * (l + 1));
    a.wr = c.take<double>(s);
    a.u = c.take<double>(s);
    a.ab = c.take<double>(2 * l + 2);
    a.G = c.take<double>((int64_t)l * l);
    a.L = c.take<double>((int64_t)l * l);
    a.Y = c.take<double>((int64_t)l * l);
    a.Aw = c.take<double>((int64_t)l * l);
    a.Tw = c.take<double>((int64_t)l * l);
    a.e2 = c.take<double>(l);
    a.Cq = c.take<double>((int64_t)k * l);
    a.Lr = c.take<double>(n * s);
    a.defl = c.take<unsigned char>(l);
  }
  ab.M = c.take<double>(n * n);
  ab.Lm = c.take<double>(n * n);
  ab.Ym = c.take<double>(n * n);
  ab.Awm = c.take<double>(n * n);
  ab.Twm = c.take<double>(n * n);
  ab.GL = c.take<double>(n * k);
  ab.deflm = c.take<unsigned char>(n);
  *total = (c.off + 255) & ~(size_t)255;
}
}  // namespace

// The l-vector basis of one projected side from its residual Gram sb.S:
// GKL (Algorithm 9) or t RPI iterations (Algorithm 10) with an SV-LCOV QR
// that is CholeskyQR2 on W^T S W (same R as Algorithm 2), pass-1 pivots
// tested against the raw norms w^T S_E w (reading R8).
template <typename TC>
static void approx_basis(svlcov_handle* h, SideBufs& sb, int s, const svlcov_approx& a, ApproxSide& x,
                         cudaStream_t st) {
  const int l = a.l;
  int* status = h->status;
  TC *S = (TC*)sb.S, *SE = (TC*)sb.SE;
  TC *P = (TC*)x.P, *W = (TC*)x.W, *T = (TC*)x.T;
  const TC tau = (TC)h->d.tau;
  if (a.method == SVLCOV_APPROX_GKL) {
    const TC* p1 = nullptr;   // NULL: all ones
    if (a.start) {            // the caller's FP64 start, in the small-step type (u is free until the first S w)
      if (sizeof(TC) == 8) p1 = (const TC*)a.start;
      else { launch_cast<double, float>(a.start, (float*)x.u, s, st); p1 = (const TC*)x.u; }
    }
    launch_gkl<TC>(S, s, l, p1, (TC*)x.Pm, W, (TC*)x.wr, (TC*)x.u, (TC*)x.ab, P, status, st);
    return;
  }
  if (sizeof(TC) == 8) launch_copy<TC>((const TC*)a.start, P, (int64_t)s * l, status, st);
  else launch_cast<double, float>(a.start, (float*)P, (int64_t)s * l, st);
  TC *T2 = (TC*)x.T2, *W2 = (TC*)x.W2, *TE = (TC*)x.TE, *G = (TC*)x.G, *L = (TC*)x.L, *Y = (TC*)x.Y;
  for (int it = 0; it < a.t; ++it) {
    launch_mgs_cols<TC>(P, s, l, status, st);                                                   // P orthonormal
    launch_copy<TC>(P, W, (int64_t)s * l, status, st);
    gemm<TC>(false, false, s, l, s, (TC)1, S, s, W, s, (TC)0, T, s, status, st);               // T = S W
    gemm<TC>(false, false, s, l, s, (TC)1, SE, s, W, s, (TC)0, TE, s, status, st);             // S_E W
    launch_diag_quad<TC>(W, TE, s, l, (TC*)x.e2, status, st);                                  // |E w_j|^2
    gemm<TC>(true, false, l, l, s, (TC)1, W, s, T, s, (TC)0, G, l, status, st);                // W^T S W
    launch_cholinv<TC, TC, false>(G, l, (const TC*)x.e2, tau, L, Y, x.defl, (TC*)x.Aw, (TC*)x.Tw, status, st);
    gemm<TC>(false, true, s, l, l, (TC)1, W, s, Y, l, (TC)0, W2, s, status, st, TRI_B_UP);     // W R1^-1
    gemm<TC>(false, true, s, l, l, (TC)1, T, s, Y, l, (TC)0, T2, s, status, st, TRI_B_UP);     // S W R1^-1
    gemm<TC>(true, false, l, l, s, (TC)1, W2, s, T2, s, (TC)0, G, l, status, st);              // pass 2 Gram
    launch_cholinv<TC, TC, false>(G, l, nullptr, tau, L, Y, x.defl, (TC*)x.Aw, (TC*)x.Tw, status, st);
    gemm<TC>(false, true, s, l, l, (TC)1, W2, s, Y, l, (TC)0, W, s, status, st, TRI_B_UP);     // W = W R^-1
    gemm<TC>(false, true, s, l, l, (TC)1, T2, s, Y, l, (TC)0, P, s, status, st, TRI_B_UP);     // P = S W
  }
}

// Fold of one projected side with an approximate basis: Xn = W_X (F[:k] -
// C' F[k:]) with C' = C0 W (k x l), and Mt = (W F[k:] Xn^-1)^T, the rows added
// to X' at the batch's touched rows (F has l + k rows, leading dimension ldf).
template <typename TC>
static void fold_projected_approx(svlcov_handle* h, SideBufs& sb, ApproxSide& x, const TC* Wx, const TC* Fbig,
                                  int ldf, int s, int l, TC* Xtmp, TC* Wn, TC* Winv, int* reset_flag, TC* itmp,
                                  cudaStream_t st) {
  int k = h->k;
  int* status = h->status;
  TC* Cq = (TC*)x.Cq;
  gemm<TC>(false, false, k, l, s, (TC)1, (TC*)sb.C0, k, (TC*)x.W, s, (TC)0, Cq, k, status, st);     // C' = C0 W
  launch_copy2d<TC>(Fbig, ldf, Xtmp, k, k, k, status, st);                                         // F[:k]
  gemm<TC>(false, false, k, k, l, (TC)-1, Cq, k, Fbig + k, ldf, (TC)1, Xtmp, k, status, st);        // - C' F[k:]
  gemm<TC>(false, false, k, k, k, (TC)1, Wx, k, Xtmp, k, (TC)0, Wn, k, status, st);
  launch_inverse<TC>(Wn, k, Winv, h->d.reset_threshold, reset_flag, status, st, itmp,
                    inv_newton(h));
  gemm<TC>(false, false, s, k, l, (TC)1, (TC*)x.W, s, Fbig + k, ldf, (TC)0, (TC*)sb.Y, s, status, st);  // W F[k:]
  gemm<TC>(true, true, k, s, k, (TC)1, Winv, k, (TC*)sb.Y, s, (TC)0, (TC*)sb.Mt, k, status, st);
}

template <typename TS, typename TC>
static int step_add_approx(svlcov_handle* h, const svlcov_csr& b, bool cols, const svlcov_approx& a,
                           cudaStream_t st) {
  const int k = h->k, s = b.rows, l = a.l, nl = k + l, ns = k + s;
  int* status = h->status;
  SideBufs& sb = h->side[0];
  ApproxBufs ab;
  size_t tot = 0;
  approx_layout(a.work, k, s, l, ab, &tot);
  TS* XpP = (TS*)(cols ? h->d.ubuf : h->d.vbuf);
  TS* XpO = (TS*)(cols ? h->d.vbuf : h->d.ubuf);
  TC* WP = (TC*)(cols ? h->Wu : h->Wv);
  TC* WO = (TC*)(cols ? h->Wv : h->Wu);
  TC* WPn = (TC*)(cols ? h->Wu_new : h->Wv_new);
  TC* WOn = (TC*)(cols ? h->Wv_new : h->Wu_new);
  TC* WPi = (TC*)(cols ? h->Wu_inv : h->Wv_inv);
  TC* WOi = (TC*)(cols ? h->Wv_inv : h->Wu_inv);
  int* rP = h->flags + (cols ? 0 : 1);
  int* rO = h->flags + (cols ? 1 : 0);
  int64_t rowsP = cols ? h->m : h->n, rowsO = cols ? h->n : h->m;
  prepare_side<TS, TC>(h, b, rowsP, XpP, WP, sb, st);
  approx_basis<TC>(h, sb, s, a, ab.side[0], st);
  TC *K = (TC*)h->K, *F = (TC*)h->F, *G = (TC*)h->G, *theta = (TC*)h->theta;
  h->prof.begin(PH_SVD, st);
  // SVD_k of the (k+l) x (k+s) K through K K^T = L L^T: the left vectors and
  // singular values of K are those of the square L; G = K^T F Theta^-1.
  launch_build_K_rect<TC>((TC*)h->sigma, (TC*)sb.C0, (TC*)ab.side[0].P, k, s, l, K, status, st);
  gemm<TC>(false, true, nl, nl, ns, (TC)1, K, nl, K, nl, (TC)0, (TC*)ab.M, nl, status, st);
  launch_cholinv<TC, TC, false>((TC*)ab.M, nl, nullptr, (TC)0, (TC*)ab.Lm, (TC*)ab.Ym, ab.deflm, (TC*)ab.Awm,
                                (TC*)ab.Twm, status, st);
  int e = small_svd_step<TC>(h, (TC*)ab.Lm, nl, F, theta, (TC*)ab.GL, st);
  if (e) return SVLCOV_ERR_CUDA;
  gemm<TC>(true, false, ns, k, nl, (TC)1, K, nl, F, nl, (TC)0, G, ns, status, st);          // K^T F
  launch_scale_cols<TC>(G, ns, ns, k, theta, status, st);                                       // Theta^-1
  h->prof.next(PH_FOLD, st);
  {
    SideFork fk(h, st);
    const cudaStream_t so = fk.stream();
    gemm<TC>(false, false, k, k, k, (TC)1, WO, k, G, ns, (TC)0, WOn, k, status, so);      // W_O G[:k]
    launch_inverse<TC>(WOn, k, WOi, h->d.reset_threshold, rO, status, so, (TC*)h->Itmp2,
                      inv_newton(h));
    gemm<TC>(true, true, k, s, k, (TC)1, WOi, k, G + k, ns, (TC)0, (TC*)h->Nt, k, status, so);  // (G[k:] W_O^-1)^T
    fold_projected_approx<TC>(h, sb, ab.side[0], WP, F, nl, s, l, (TC*)h->Xu, WPn, WPi, rP, (TC*)h->Itmp, st);
  }
  FiniteSet<TC> fs{};
  fs.ptr[0] = theta; fs.count[0] = k;
  fs.ptr[1] = (TC*)sb.Mt; fs.count[1] = (int64_t)k * s;
  fs.ptr[2] = (TC*)h->Nt; fs.count[2] = (int64_t)k * s;
  fs.ptr[3] = WPn; fs.count[3] = (int64_t)k * k;
  fs.ptr[4] = WOn; fs.count[4] = (int64_t)k * k;
  fs.n = 5;
  h->prof.next(PH_APPLY, st);
  launch_check_finite_multi<TC>(fs, status, st);
  launch_reset<TS, TC>(XpP, rowsP, k, WPn, rP, status, st);
  launch_scatter<TS, TC>(XpP, k, (TC*)sb.Mt, b.nnz, sb.sc, status, st);
  launch_reset<TS, TC>(XpO, rowsO, k, WOn, rO, status, st);
  launch_append<TS, TC>(XpO, rowsO, k, s, (TC*)h->Nt, status, st);
  if (cols)
    launch_commit<TC>((TC*)h->Wu, WPn, rP, (TC*)h->Wv, WOn, rO, (TC*)h->sigma, theta, k, h->counters, 0, s,
                      h->resets, status, st);
  else
    launch_commit<TC>((TC*)h->Wu, WOn, rO, (TC*)h->Wv, WPn, rP, (TC*)h->sigma, theta, k, h->counters, s, 0,
                      h->resets, status, st);
  h->prof.end(st);
  return last_launch();
}

template <typename TS, typename TC>
static int step_weights_approx(svlcov_handle* h, const svlcov_csr& D, const svlcov_csr& E, const svlcov_approx& a,
                               cudaStream_t st) {
  const int k = h->k, s = D.rows, l = a.l, nl = k + l;
  int* status = h->status;
  SideBufs& sd = h->side[0];
  SideBufs& se = h->side[1];
  ApproxBufs ab;
  size_t tot = 0;
  approx_layout(a.work, k, s, l, ab, &tot);
  prepare_side<TS, TC>(h, D, h->m, (TS*)h->d.ubuf, (TC*)h->Wu, sd, st);
  prepare_side<TS, TC>(h, E, h->n, (TS*)h->d.vbuf, (TC*)h->Wv, se, st);
  approx_basis<TC>(h, sd, s, a, ab.side[0], st);
  approx_basis<TC>(h, se, s, a, ab.side[1], st);
  TC *K = (TC*)h->K, *F = (TC*)h->F, *G = (TC*)h->G, *theta = (TC*)h->theta;
  h->prof.begin(PH_SVD, st);
  launch_build_L_rect<TC>((TC*)sd.C0, (TC*)ab.side[0].P, k, s, l, (TC*)ab.side[0].Lr, status, st);
  launch_build_L_rect<TC>((TC*)se.C0, (TC*)ab.side[1].P, k, s, l, (TC*)ab.side[1].Lr, status, st);
  gemm<TC>(false, true, nl, nl, s, (TC)1, (TC*)ab.side[0].Lr, nl, (TC*)ab.side[1].Lr, nl, (TC)0, K, nl, status, st);
  launch_add_diag<TC>(K, nl, (TC*)h->sigma, k, status, st);   // K = diag(S,0) + [C0D;PD^T][C0E;PE^T]^T
  int e = small_svd_step<TC>(h, K, nl, F, theta, G, st);
  if (e) return SVLCOV_ERR_CUDA;
  h->prof.next(PH_FOLD, st);
  {
    SideFork fk(h, st);
    fold_projected_approx<TC>(h, se, ab.side[1], (TC*)h->Wv, G, nl, s, l, (TC*)h->Xv, (TC*)h->Wv_new,
                              (TC*)h->Wv_inv, h->flags + 1, (TC*)h->Itmp2, fk.stream());
    fold_projected_approx<TC>(h, sd, ab.side[0], (TC*)h->Wu, F, nl, s, l, (TC*)h->Xu, (TC*)h->Wu_new,
                              (TC*)h->Wu_inv, h->flags + 0, (TC*)h->Itmp, st);
  }
  FiniteSet<TC> fs{};
  fs.ptr[0] = theta; fs.count[0] = k;
  fs.ptr[1] = (TC*)sd.Mt; fs.count[1] = (int64_t)k * s;
  fs.ptr[2] = (TC*)se.Mt; fs.count[2] = (int64_t)k * s;
  fs.ptr[3] = (TC*)h->Wu_new; fs.count[3] = (int64_t)k * k;
  fs.ptr[4] = (TC*)h->Wv_new; fs.count[4] = (int64_t)k * k;
  fs.n = 5;
  h->prof.next(PH_APPLY, st);
  launch_check_finite_multi<TC>(fs, status, st);
  launch_reset<TS, TC>((TS*)h->d.ubuf, h->m, k, (TC*)h->Wu_new, h->flags + 0, status, st);
  launch_scatter<TS, TC>((TS*)h->d.ubuf, k, (TC*)sd.Mt, D.nnz, sd.sc, status, st);
  launch_reset<TS, TC>((TS*)h->d.vbuf, h->n, k, (TC*)h->Wv_new, h->flags + 1, status, st);
  launch_scatter<TS, TC>((TS*)h->d.vbuf, k, (TC*)se.Mt, E.nnz, se.sc, status, st);
  launch_commit<TC>((TC*)h->Wu, (TC*)h->Wu_new, h->flags + 0, (TC*)h->Wv, (TC*)h->Wv_new, h->flags + 1,
                    (TC*)h->sigma, theta, k, h->counters, 0, 0, h->resets, status, st);
  h->prof.end(st);
  return last_launch();
}

static bool approx_ok(const svlcov_handle* h, const svlcov_approx* a, int s) {
  if (!a || !a->work) return false;
  if (a->method != SVLCOV_APPROX_GKL && a->method != SVLCOV_APPROX_RPI) return false;
  if (a->l < 1 || a->l > s) return false;
  if (a->method == SVLCOV_APPROX_RPI && (a->t < 1 || !a->start)) return false;
  return true;
}

extern "C" size_t svlcov_approx_work_bytes(const svlcov_handle* h, int32_t l) {
  if (!h || l < 1 || l > h->d.max_s) return 0;
  ApproxBufs ab;
  size_t tot = 0;
  approx_layout(nullptr, h->k, (int)h->d.max_s, l, ab, &tot);
  return tot;
}

template <typename TC>
static int dispatch_add_approx(svlcov_handle* h, const svlcov_csr& b, bool cols, const svlcov_approx& a,
                               cudaStream_t st) {
  switch (h->d.storage) {
    case SVLCOV_FP64: return step_add_approx<double, TC>(h, b, cols, a, st);
    case SVLCOV_FP32: return step_add_approx<float, TC>(h, b, cols, a, st);
    default: return step_add_approx<__nv_bfloat16, TC>(h, b, cols, a, st);
  }
}

template <typename TC>
static int dispatch_weights_approx(svlcov_handle* h, const svlcov_csr& D, const svlcov_csr& E,
                                   const svlcov_approx& a, cudaStream_t st) {
  switch (h->d.storage) {
    case SVLCOV_FP64: return step_weights_approx<double, TC>(h, D, E, a, st);
    case SVLCOV_FP32: return step_weights_approx<float, TC>(h, D, E, a, st);
    default: return step_weights_approx<__nv_bfloat16, TC>(h, D, E, a, st);
  }
}

static int do_add_approx(svlcov_handle* h, const svlcov_csr* b, bool cols, const svlcov_approx* a, void* stream) {
  if (!h || !csr_ok(b)) return SVLCOV_ERR_INVALID_ARG;
  int64_t d_len = cols ? h->m : h->n;
  if (b->cols != d_len) return SVLCOV_ERR_INVALID_ARG;
  if (b->rows > h->d.max_s || b->nnz > h->d.max_nnz) return SVLCOV_ERR_CAPACITY;
  if (cols ? (h->n + b->rows > h->d.max_n) : (h->m + b->rows > h->d.max_m)) return SVLCOV_ERR_CAPACITY;
  if (b->rows == 0) return SVLCOV_OK;
  if (!approx_ok(h, a, b->rows)) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  maybe_reorth(h, cols ? 1 : 2, st);
  int rc = small_is_f32(h) ? dispatch_add_approx<float>(h, *b, cols, *a, st)
                           : dispatch_add_approx<double>(h, *b, cols, *a, st);
  if (rc == SVLCOV_OK) {
    if (cols) h->n += b->rows;
    else h->m += b->rows;
    h->last_op = cols ? 3 : 4;   // no intermediates for the exact-step backward
    h->last_s = b->rows;
    ++h->steps;
  }
  return rc;
}

extern "C" int svlcov_add_cols_approx(svlcov_handle* h, const svlcov_csr* Ec_T, const svlcov_approx* a,
                                      void* stream) {
  SplitScope split_scope(h, true);
  return do_add_approx(h, Ec_T, true, a, stream);
}

extern "C" int svlcov_add_rows_approx(svlcov_handle* h, const svlcov_csr* Er, const svlcov_approx* a, void* stream) {
  SplitScope split_scope(h, true);
  return do_add_approx(h, Er, false, a, stream);
}

extern "C" int svlcov_update_weights_approx(svlcov_handle* h, const svlcov_csr* D_T, const svlcov_csr* Em_T,
                                            const svlcov_approx* a, void* stream) {
  SplitScope split_scope(h, true);
  if (!h || !csr_ok(D_T) || !csr_ok(Em_T)) return SVLCOV_ERR_INVALID_ARG;
  if (D_T->cols != h->m || Em_T->cols != h->n || D_T->rows != Em_T->rows) return SVLCOV_ERR_INVALID_ARG;
  if (D_T->rows > h->d.max_s || D_T->nnz > h->d.max_nnz || Em_T->nnz > h->d.max_nnz) return SVLCOV_ERR_CAPACITY;
  if (D_T->rows == 0) return SVLCOV_OK;
  if (!approx_ok(h, a, D_T->rows)) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  maybe_reorth(h, 3, st);
  int rc = small_is_f32(h) ? dispatch_weights_approx<float>(h, *D_T, *Em_T, *a, st)
                           : dispatch_weights_approx<double>(h, *D_T, *Em_T, *a, st);
  if (rc == SVLCOV_OK) {
    h->last_op = 5;
    h->last_s = D_T->rows;
    ++h->steps;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// Batched runs: a per-device pool of non-blocking streams and events.
namespace {
struct StreamPool {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
};
std::mutex g_pool_mu;
std::unordered_map<int, StreamPool> g_pools;

int pool_for(int need, StreamPool** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SVLCOV_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  StreamPool& p = g_pools[dev];
  if (!p.fork && cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return SVLCOV_ERR_CUDA;
  while ((int)p.streams.size() < need) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SVLCOV_ERR_CUDA;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SVLCOV_ERR_CUDA;
    p.streams.push_back(s);
    p.done.push_back(e);
  }
  *out = &p;
  return SVLCOV_OK;
}
}  // namespace

extern "C" int svlcov_batch_run(svlcov_handle** hs, const svlcov_op* ops, int32_t n_ops, int32_t concurrency,
                                void* stream) {
  if (!hs || (!ops && n_ops > 0) || n_ops < 0) return SVLCOV_ERR_INVALID_ARG;
  if (n_ops == 0) return SVLCOV_OK;
  int P = std::max(1, std::min(64, (int)concurrency));
  StreamPool* pool = nullptr;
  int rc = pool_for(P, &pool);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaEventRecord(pool->fork, st));
  for (int i = 0; i < P; ++i) CUDA_OK(cudaStreamWaitEvent(pool->streams[i], pool->fork, 0));
  std::unordered_map<svlcov_handle*, int> lane;  // handle -> its stream
  int next = 0;
  t_side_fork = false;
  for (int32_t i = 0; i < n_ops && rc == SVLCOV_OK; ++i) {
    svlcov_handle* h = hs[i];
    if (!h) { rc = SVLCOV_ERR_INVALID_ARG; break; }
    auto it = lane.find(h);
    int li = it != lane.end() ? it->second : (lane[h] = next++ % P);
    void* s2 = (void*)pool->streams[li];
    const svlcov_op& op = ops[i];
    if (op.kind == 0) rc = svlcov_add_cols(h, &op.a, s2);
    else if (op.kind == 1) rc = svlcov_add_rows(h, &op.a, s2);
    else if (op.kind == 2) rc = svlcov_update_weights(h, &op.a, &op.b, s2);
    else rc = SVLCOV_ERR_INVALID_ARG;
  }
  t_side_fork = true;
  for (int i = 0; i < P; ++i) {  // join, also after an error
    CUDA_OK(cudaEventRecord(pool->done[i], pool->streams[i]));
    CUDA_OK(cudaStreamWaitEvent(st, pool->done[i], 0));
  }
  return rc;
}

// ---------------------------------------------------------------------------
template <typename TS, typename TC>
static void materialize_side(svlcov_handle* h, int side, void* out, int out_dtype, const int32_t* idx, int64_t cnt,
                             cudaStream_t st) {
  const TS* Xp = (const TS*)(side == 0 ? h->d.ubuf : h->d.vbuf);
  const TC* W = (const TC*)(side == 0 ? h->Wu : h->Wv);
  int64_t rows = side == 0 ? h->m : h->n;
  launch_materialize<TS, TC>(Xp, idx ? cnt : rows, rows, h->k, W, out, out_dtype, idx, st, h->status);
}

template <typename TC>
static void materialize_dispatch(svlcov_handle* h, int side, void* out, int out_dtype, const int32_t* idx,
                                 int64_t cnt, cudaStream_t st) {
  switch (h->d.storage) {
    case SVLCOV_FP64: materialize_side<double, TC>(h, side, out, out_dtype, idx, cnt, st); break;
    case SVLCOV_FP32: materialize_side<float, TC>(h, side, out, out_dtype, idx, cnt, st); break;
    default: materialize_side<__nv_bfloat16, TC>(h, side, out, out_dtype, idx, cnt, st); break;
  }
}

extern "C" int svlcov_get_factors(svlcov_handle* h, void* U, double* sigma, void* V, int32_t out_dtype,
                                  void* stream) {
  if (!h || (out_dtype != SVLCOV_FP64 && out_dtype != SVLCOV_FP32)) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  bool f32 = small_is_f32(h);
  if (U) f32 ? materialize_dispatch<float>(h, 0, U, out_dtype, nullptr, 0, st)
             : materialize_dispatch<double>(h, 0, U, out_dtype, nullptr, 0, st);
  if (V) f32 ? materialize_dispatch<float>(h, 1, V, out_dtype, nullptr, 0, st)
             : materialize_dispatch<double>(h, 1, V, out_dtype, nullptr, 0, st);
  if (sigma) {
    if (f32) launch_cast<float, double>((const float*)h->sigma, sigma, h->k, st);
    else cudaMemcpyAsync(sigma, h->sigma, sizeof(double) * h->k, cudaMemcpyDeviceToDevice, st);
  }
  return last_launch();
}

extern "C" int svlcov_query_rows(svlcov_handle* h, int32_t side, const int32_t* idx, int32_t cnt, void* out,
                                 int32_t out_dtype, void* stream) {
  if (!h || (side != 0 && side != 1) || cnt < 0 || (cnt > 0 && (!idx || !out))) return SVLCOV_ERR_INVALID_ARG;
  if (out_dtype != SVLCOV_FP64 && out_dtype != SVLCOV_FP32) return SVLCOV_ERR_INVALID_ARG;
  if (cnt == 0) return SVLCOV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (small_is_f32(h)) materialize_dispatch<float>(h, side, out, out_dtype, idx, cnt, st);
  else materialize_dispatch<double>(h, side, out, out_dtype, idx, cnt, st);
  return last_launch();
}

template <typename TC>
static void score_dispatch(svlcov_handle* h, const int32_t* rows, const int32_t* cols, int64_t npairs, int symmetric,
                           double* out, cudaStream_t st) {
  const TC *Wu = (const TC*)h->Wu, *Wv = (const TC*)h->Wv, *sg = (const TC*)h->sigma;
  double* Mw = (double*)h->Itmp;   // k x k; step scratch, free between steps
  switch (h->d.storage) {
    case SVLCOV_FP64:
      launch_score_pairs<double, TC>((const double*)h->d.ubuf, (const double*)h->d.vbuf, h->m, h->n, h->k, Wu, Wv, sg,
                                     rows, cols, npairs, symmetric, out, Mw, h->status, st);
      break;
    case SVLCOV_FP32:
      launch_score_pairs<float, TC>((const float*)h->d.ubuf, (const float*)h->d.vbuf, h->m, h->n, h->k, Wu, Wv, sg,
                                    rows, cols, npairs, symmetric, out, Mw, h->status, st);
      break;
    default:
      launch_score_pairs<__nv_bfloat16, TC>((const __nv_bfloat16*)h->d.ubuf, (const __nv_bfloat16*)h->d.vbuf, h->m,
                                            h->n, h->k, Wu, Wv, sg, rows, cols, npairs, symmetric, out, Mw,
                                            h->status, st);
  }
}

extern "C" int svlcov_score_pairs(svlcov_handle* h, const int32_t* rows, const int32_t* cols, int64_t npairs,
                                  int32_t symmetric, double* out, void* stream) {
  if (!h || npairs < 0 || (npairs > 0 && (!rows || !cols || !out))) return SVLCOV_ERR_INVALID_ARG;
  if (npairs == 0) return SVLCOV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (small_is_f32(h)) score_dispatch<float>(h, rows, cols, npairs, symmetric != 0, out, st);
  else score_dispatch<double>(h, rows, cols, npairs, symmetric != 0, out, st);
  return last_launch();
}

extern "C" int svlcov_project(svlcov_handle* h, int32_t side, const svlcov_csr* E, double* P, double* C0,
                              void* stream) {
  if (!h || (side != 0 && side != 1) || !csr_ok(E) || (E->rows > 0 && !P)) return SVLCOV_ERR_INVALID_ARG;
  if (E->cols != (side == 0 ? h->m : h->n) || (h->k & 3) != 0) return SVLCOV_ERR_INVALID_ARG;
  if (E->rows == 0) return SVLCOV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t rows = side == 0 ? h->m : h->n;
  const void* Xp = side == 0 ? h->d.ubuf : h->d.vbuf;
  SplitScope split_scope(h);
  switch (h->d.storage) {
    case SVLCOV_FP64: launch_project<double, double>(*E, (const double*)Xp, rows, h->k, P, h->status, st); break;
    case SVLCOV_FP32: launch_project<float, double>(*E, (const float*)Xp, rows, h->k, P, h->status, st); break;
    default: launch_project<__nv_bfloat16, double>(*E, (const __nv_bfloat16*)Xp, rows, h->k, P, h->status, st);
  }
  if (C0) {   // C0 = W^T P with the side's small factor (FP64; FP32 handles widen it first)
    const int k = h->k;
    const double* W = (const double*)(side == 0 ? h->Wu : h->Wv);
    if (small_is_f32(h)) {
      launch_cast<float, double>((const float*)(side == 0 ? h->Wu : h->Wv), (double*)h->Itmp, (int64_t)k * k, st);
      W = (const double*)h->Itmp;
    }
    gemm<double>(true, false, k, E->rows, k, 1.0, W, k, P, k, 0.0, C0, k, h->status, st);
  }
  return last_launch();
}

extern "C" int svlcov_get_shape(const svlcov_handle* h, int64_t* m, int64_t* n, int32_t* k) {
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  if (m) *m = h->m;
  if (n) *n = h->n;
  if (k) *k = h->k;
  return SVLCOV_OK;
}

extern "C" int svlcov_status(svlcov_handle* h, int32_t* device_code, void* stream) {
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_OK(cudaStreamSynchronize(st));
  int code = 0;
  CUDA_OK(cudaMemcpy(&code, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (code != 0) {
    int64_t c[2];
    CUDA_OK(cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
    h->m = c[0];
    h->n = c[1];
    CUDA_OK(cudaMemset(h->status, 0, sizeof(int)));
  }
  if (device_code) *device_code = code;
  return SVLCOV_OK;
}

static int copy_small_to_host(svlcov_handle* h, const double* src, double* dst, int64_t count) {
  if (!dst) return SVLCOV_OK;
  if (small_is_f32(h)) {
    std::vector<float> tmp(count);
    CUDA_OK(cudaMemcpy(tmp.data(), src, sizeof(float) * count, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < count; ++i) dst[i] = tmp[i];
  } else {
    CUDA_OK(cudaMemcpy(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost));
  }
  return SVLCOV_OK;
}

static int copy_small_from_host(svlcov_handle* h, const double* src, double* dst, int64_t count) {
  if (!src) return SVLCOV_OK;
  if (small_is_f32(h)) {
    std::vector<float> tmp(count);
    for (int64_t i = 0; i < count; ++i) tmp[i] = (float)src[i];
    CUDA_OK(cudaMemcpy(dst, tmp.data(), sizeof(float) * count, cudaMemcpyHostToDevice));
  } else {
    CUDA_OK(cudaMemcpy(dst, src, sizeof(double) * count, cudaMemcpyHostToDevice));
  }
  return SVLCOV_OK;
}

// k x k small matrices are column-major on the device; the host API is row-major.
static void transpose_sq(double* a, int k) {
  for (int i = 0; i < k; ++i)
    for (int j = i + 1; j < k; ++j) std::swap(a[i * k + j], a[j * k + i]);
}

extern "C" int svlcov_get_small_state(svlcov_handle* h, double* Wu, double* Wv, double* sigma, int64_t* resets,
                                      void* stream) {
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  CUDA_OK(cudaStreamSynchronize((cudaStream_t)stream));
  int k = h->k;
  int rc;
  if ((rc = copy_small_to_host(h, h->Wu, Wu, (int64_t)k * k))) return rc;
  if ((rc = copy_small_to_host(h, h->Wv, Wv, (int64_t)k * k))) return rc;
  if ((rc = copy_small_to_host(h, h->sigma, sigma, k))) return rc;
  if (Wu) transpose_sq(Wu, k);
  if (Wv) transpose_sq(Wv, k);
  if (resets) CUDA_OK(cudaMemcpy(resets, h->resets, sizeof(int64_t), cudaMemcpyDeviceToHost));
  return SVLCOV_OK;
}

static size_t storage_elem(const svlcov_handle* h) {
  return h->d.storage == SVLCOV_FP64 ? 8 : (h->d.storage == SVLCOV_FP32 ? 4 : 2);
}

extern "C" int svlcov_get_state(svlcov_handle* h, void* Up_host, void* Vp_host, double* Wu_host, double* Wv_host,
                                double* sigma_host, void* stream) {
  if (!h) return SVLCOV_ERR_INVALID_ARG;
  CUDA_OK(cudaStreamSynchronize((cudaStream_t)stream));
  size_t es = storage_elem(h);
  if (Up_host) CUDA_OK(cudaMemcpy(Up_host, h->d.ubuf, es * h->m * h->k, cudaMemcpyDeviceToHost));
  if (Vp_host) CUDA_OK(cudaMemcpy(Vp_host, h->d.vbuf, es * h->n * h->k, cudaMemcpyDeviceToHost));
  return svlcov_get_small_state(h, Wu_host, Wv_host, sigma_host, nullptr, stream);
}

extern "C" int svlcov_set_state(svlcov_handle* h, int64_t m, int64_t n, const void* Up_host, const void* Vp_host,
                                const double* Wu_host, const double* Wv_host, const double* sigma_host,
                                void* stream) {
  SplitScope split_scope(h);
  if (!h || m < 0 || n < 0 || m > h->d.max_m || n > h->d.max_n) return SVLCOV_ERR_INVALID_ARG;
  if (!Up_host || !Vp_host || !Wu_host || !Wv_host || !sigma_host) return SVLCOV_ERR_INVALID_ARG;
  CUDA_OK(cudaStreamSynchronize((cudaStream_t)stream));
  size_t es = storage_elem(h);
  int k = h->k;
  CUDA_OK(cudaMemcpy(h->d.ubuf, Up_host, es * m * k, cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemcpy(h->d.vbuf, Vp_host, es * n * k, cudaMemcpyHostToDevice));
  std::vector<double> wu(Wu_host, Wu_host + (size_t)k * k), wv(Wv_host, Wv_host + (size_t)k * k);
  transpose_sq(wu.data(), k);
  transpose_sq(wv.data(), k);
  int rc;
  if ((rc = copy_small_from_host(h, wu.data(), h->Wu, (int64_t)k * k))) return rc;
  if ((rc = copy_small_from_host(h, wv.data(), h->Wv, (int64_t)k * k))) return rc;
  if ((rc = copy_small_from_host(h, sigma_host, h->sigma, k))) return rc;
  int64_t c[4] = {m, n, 0, 0};
  CUDA_OK(cudaMemcpy(h->counters, c, sizeof(c), cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemset(h->status, 0, sizeof(int)));
  h->m = m;
  h->n = n;
  h->last_op = -1;  // the step intermediates no longer belong to this state
  return SVLCOV_OK;
}

extern "C" int svlcov_get_intermediate(svlcov_handle* h, int32_t which, int32_t side, double* host_out,
                                       size_t capacity, int32_t* rows, int32_t* cols, void* stream) {
  if (!h || side < 0 || side > 1 || h->last_op < 0) return SVLCOV_ERR_INVALID_ARG;
  if (h->last_op > 2) return SVLCOV_ERR_STATE;   // approximate steps keep other intermediates
  if (h->last_rfree && (which == 3 || which == 4 || which == 6)) return SVLCOV_ERR_STATE;   // R, K, F not formed
  int k = h->k, s = h->last_s, n2 = k + s;
  const SideBufs& sb = h->side[side];
  const double* src = nullptr;
  int r = 0, c = 0;
  switch (which) {
    case 0: src = sb.P; r = k; c = s; break;
    case 1: src = sb.SE; r = s; c = s; break;
    case 2: src = sb.C0; r = k; c = s; break;
    case 3: src = sb.R; r = s; c = s; break;
    case 4: src = h->K; r = n2; c = n2; break;
    case 5: src = h->theta; r = k; c = 1; break;
    case 6: src = h->F; r = n2; c = k; break;
    case 7: src = h->G; r = n2; c = k; break;
    default: return SVLCOV_ERR_INVALID_ARG;
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (!host_out) return SVLCOV_OK;
  if ((size_t)r * c > capacity) return SVLCOV_ERR_CAPACITY;
  CUDA_OK(cudaStreamSynchronize((cudaStream_t)stream));
  return copy_small_to_host(h, src, host_out, (int64_t)r * c);
}

// ---------------------------------------------------------------------------
// Backward of the last add-columns step (FP64 small state).
extern "C" size_t svlcov_add_cols_backward_work_bytes(const svlcov_handle* h) {
  if (!h) return 0;
  int s = (int)h->d.max_s;
  return backward_work_bytes(h->k + s, h->k, s, std::max<int64_t>(h->d.max_nnz, 1));
}

extern "C" int svlcov_add_cols_backward(svlcov_handle* h, const svlcov_csr* E, const int32_t* rows_S, int32_t nS,
                                        const double* U_pre_S, const double* U_pre_nnz, const double* dL_dU_S,
                                        const double* dL_dtheta, double* dL_dvalues, double gap, void* work,
                                        void* stream) {
  SplitScope split_scope(h);
  if (!h || !csr_ok(E) || !work) return SVLCOV_ERR_INVALID_ARG;
  if (h->d.small != SVLCOV_SMALL_FP64 && h->d.small != SVLCOV_SMALL_MIXED) return SVLCOV_ERR_INVALID_ARG;
  if (h->last_op != 0 || E->rows != h->last_s) return SVLCOV_ERR_STATE;
  if (h->last_rfree) return SVLCOV_ERR_STATE;   // needs the literal route (init option literal_steps)
  if (nS < 0 || nS > h->m || (nS > 0 && (!rows_S || !U_pre_S || !dL_dU_S))) return SVLCOV_ERR_INVALID_ARG;
  if (E->nnz > 0 && (!U_pre_nnz || !dL_dvalues)) return SVLCOV_ERR_INVALID_ARG;
  const SideBufs& sb = h->side[0];
  BackwardInputs in{};
  in.C0 = sb.C0; in.R = sb.R; in.X = sb.X; in.CQ = sb.CQ; in.Y = sb.Y;
  in.K = h->K; in.F = h->F; in.G = h->G; in.theta = h->theta;
  in.rowid = sb.sc.rowid; in.slot = sb.sc.slot; in.hstart = sb.sc.hstart; in.hcnt = sb.sc.hcnt;
  in.seg_j = sb.sc.seg_j; in.seg_v = sb.sc.seg_v;
  in.jwork = h->jwork;
  in.mixed = h->d.small == SVLCOV_SMALL_MIXED;
  return launch_add_cols_backward(*E, h->k, in, rows_S, nS, U_pre_S, U_pre_nnz, dL_dU_S, dL_dtheta, dL_dvalues,
                                  gap > 0 ? gap : 1e-6, work, h->status, (cudaStream_t)stream);
}

extern "C" const char* svlcov_strerror(int32_t code) {
  switch (code) {
    case SVLCOV_OK: return "ok";
    case SVLCOV_ERR_INVALID_ARG: return "invalid argument";
    case SVLCOV_ERR_CAPACITY: return "capacity exceeded";
    case SVLCOV_ERR_CUDA: return "CUDA runtime error";
    case SVLCOV_ERR_STATE: return "handle not in the state the call needs";
    case SVLCOV_DEV_BAD_CSR: return "malformed CSR batch";
    case SVLCOV_DEV_NONFINITE: return "non-finite value";
    case SVLCOV_DEV_NOT_PD: return "residual Gram matrix not finite";
    case SVLCOV_DEV_GAP_WARN: return "singular-value gap guard";
    case SVLCOV_DEV_TIMEOUT: return "bounded device wait expired";
    default: return "combination of device status bits";
  }
}

// ---- standalone one-vector SVD ---------------------------------------------------
extern "C" size_t svlcov_small_svd_arrow_work_bytes(void) { return arrow_work_bytes() + 16; }

extern "C" int svlcov_small_svd_arrow(const double* sigma, const double* c, const double* rho, int32_t k, double* F,
                                      double* theta, double* G, void* work, void* stream) {
  if (!sigma || !c || !rho || !F || !theta || !G || !work || k < 1 || k > SVLCOV_MAX_K) return SVLCOV_ERR_INVALID_ARG;
  if (((uintptr_t)work & 255) != 0) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = (int*)((char*)work + arrow_work_bytes());
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SVLCOV_ERR_CUDA;
  launch_arrow_svd(sigma, c, rho, k, F, theta, G, work, status, st);
  return last_launch();
}

// ---- standalone dense product --------------------------------------------------
extern "C" int svlcov_dgemm(int32_t ta, int32_t tb, int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                            int32_t lda, const double* B, int32_t ldb, double beta, double* C, int32_t ldc,
                            int32_t engine, void* stream) {
  if (M < 0 || N < 0 || K < 0 || M > 4096 || N > 4096 || K > 4096 || engine < 0 || engine > 2)
    return SVLCOV_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return SVLCOV_OK;
  if (!C || ldc < M || (K > 0 && (!A || !B))) return SVLCOV_ERR_INVALID_ARG;
  if (K > 0 && (lda < (ta ? K : M) || ldb < (tb ? N : K))) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (engine == 2) {
    gemm_df(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, st);
    return last_launch();
  }
  GemmTcScope tc(engine == 1);
  gemm<double>(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, st);
  return last_launch();
}

// ---- standalone small SVD ----------------------------------------------------
extern "C" size_t svlcov_small_svd_work_bytes(int32_t n) {
  if (n <= 0) return 0;
  return jacobi_work_bytes(n) + 3 * (size_t)n * n * sizeof(double) + 2 * n * sizeof(double) +
         refine_work_bytes(n, n) + 8192;
}

extern "C" int svlcov_small_svd(const double* K, int32_t n, int32_t k, double* F, double* theta, double* G,
                                int32_t precision, void* work, int32_t* sweeps, void* stream) {
  if (!K || !F || !theta || !G || !work || n <= 0 || k <= 0 || k > n) return SVLCOV_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(work);
  int* status = c.take<int>(4);
  char* jw = c.take<char>(jacobi_work_bytes(n));
  cudaMemsetAsync(status, 0, sizeof(int) * 4, st);
  int e = 0;
  if (precision == SVLCOV_SMALL_FP32) {
    float* Kf = c.take<float>((size_t)n * n);
    float* Ff = c.take<float>((size_t)n * k);
    float* Gf = c.take<float>((size_t)n * k);
    float* tf = c.take<float>(k);
    launch_cast<double, float>(K, Kf, (int64_t)n * n, st);
    e = launch_jacobi<float>(Kf, n, k, Ff, tf, Gf, jw, status, st);
    launch_cast<float, double>(Ff, F, (int64_t)n * k, st);
    launch_cast<float, double>(Gf, G, (int64_t)n * k, st);
    launch_cast<float, double>(tf, theta, k, st);
  } else if (precision == SVLCOV_SMALL_MIXED) {
    char* rw = c.take<char>(refine_work_bytes(n, k));
    e = launch_mixed_svd(K, n, k, F, theta, G, jw, rw, status, st, nullptr);
  } else {
    e = launch_jacobi<double>(K, n, k, F, theta, G, jw, status, st);
  }
  if (e) return SVLCOV_ERR_CUDA;
  if (sweeps) {
    CUDA_OK(cudaStreamSynchronize(st));
    int* sw = jacobi_sweeps_ptr(jw, n, precision == SVLCOV_SMALL_FP64 ? 8 : 4);
    CUDA_OK(cudaMemcpy(sweeps, sw, sizeof(int), cudaMemcpyDeviceToHost));
  }
  return last_launch();
}

// Sparse kernels of the SV-LCOV update step: batch validation, the grouped
// (column) view of a batch, the fused gather + Gram kernel that turns the
// batch into SV-LCOV form (Lemma 1: c = U^T b by gathering the rows of U' at
// the nonzeros of b; Lemma 2: the inner products <b_i, b_j>), the sparse
// matrix addition that folds B F[k:] U''^-1 into U' (Section 3.2), the row
// append, the identity reset of the extended decomposition, and the
// materialisation / query U = U' U'' (Theorem 1, Query).
#include <atomic>

#include "kernels.cuh"

namespace svl {

static std::atomic<uint64_t> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

int64_t max_chunks(int64_t max_s, int64_t max_nnz) { return max_s + max_nnz / kChunk + 1; }

// ---------------------------------------------------------------------------
// a0: validation.  One warp per batch row.  Checks indptr (monotone, within
// [0, nnz], indptr[0] = 0, indptr[s] = nnz), indices in [0, d), values finite,
// no duplicate index inside a row (O(deg^2) pairwise scan).  Records the row
// of every nonzero for the later kernels.
__global__ void k_validate(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const void* __restrict__ values, int vdtype, int s, int64_t d, int64_t nnz,
                           int* __restrict__ rowid, int* __restrict__ status) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= s) return;
  int j = warp;
  int64_t a = indptr[j], b = indptr[j + 1];
  if (lane == 0) {
    if (j == 0 && a != 0) flag(status, SVLCOV_DEV_BAD_CSR);
    if (j == s - 1 && b != nnz) flag(status, SVLCOV_DEV_BAD_CSR);
  }
  if (a < 0 || b < a || b > nnz) {
    if (lane == 0) flag(status, SVLCOV_DEV_BAD_CSR);
    return;
  }
  bool bad = false, nonfinite = false;
  for (int64_t e = a + lane; e < b; e += 32) {
    int32_t i = indices[e];
    if (i < 0 || (int64_t)i >= d) bad = true;
    double v = load_val<double>(values, vdtype, e);
    if (!is_finite(v)) nonfinite = true;
    rowid[e] = j;
    for (int64_t f = e + 1; f < b; ++f)
      if (indices[f] == i) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) flag(status, SVLCOV_DEV_BAD_CSR);
  if (__any_sync(0xffffffffu, nonfinite) && lane == 0) flag(status, SVLCOV_DEV_NONFINITE);
}

void launch_validate(const svlcov_csr& b, int64_t d, int* rowid, int* status, cudaStream_t st) {
  if (b.rows <= 0) return;
  int wpb = 8;
  note_launches(1);
  k_validate<<<(int)cdiv(b.rows, wpb), wpb * 32, 0, st>>>(b.indptr, b.indices, b.values, b.values_dtype,
                                                         b.rows, d, b.nnz, rowid, status);
}

// ---------------------------------------------------------------------------
// Grouped view of the batch: all nonzeros that hit the same row i of U' (or
// V') are gathered into one group, ordered by batch row.  Groups are found
// with an open-addressing hash table of size H = 2^logH >= 2 nnz (O(nnz) work,
// no O(m) array), so the step never touches memory proportional to m or n.
__device__ __forceinline__ uint32_t hash_slot(uint32_t i, int logH) {
  return (uint32_t)(i * 2654435761u) >> (32 - logH);
}

__global__ void k_hash_insert(const int32_t* __restrict__ indices, int64_t nnz, int logH, int* hkey, int* hcnt,
                              int* __restrict__ slot, int* __restrict__ rank_tmp, const int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz || failed(status)) return;
  int i = indices[e];
  uint32_t mask = (1u << logH) - 1u;
  uint32_t h = logH > 0 ? hash_slot((uint32_t)i, logH) : 0u;
  for (uint32_t probe = 0; probe <= mask; ++probe) {  // bounded: the table is at most half full
    int prev = atomicCAS(&hkey[h], -1, i);
    if (prev == -1 || prev == i) break;
    h = (h + 1u) & mask;
  }
  slot[e] = (int)h;
  rank_tmp[e] = atomicAdd(&hcnt[h], 1);
}

// Single CTA: exclusive scan of the group sizes, list of occupied slots, and
// the chunk decomposition of the batch rows (ceil(deg / kChunk), at least 1).
__global__ void k_group_scan(const int* __restrict__ hcnt, int H, int* __restrict__ hstart, int* __restrict__ occ,
                             const int32_t* __restrict__ indptr, int s, int* __restrict__ chunk_off,
                             int* __restrict__ chunk_row, int* __restrict__ counts, const int* status) {
  if (failed(status)) return;
  __shared__ int warp_tot[32];
  __shared__ int warp_occ[32];
  __shared__ int carry_sum, carry_occ;
  int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) { carry_sum = 0; carry_occ = 0; }
  __syncthreads();
  // pass over H in tiles of blockDim: scan counts and occupancy together
  for (int base = 0; base < H; base += blockDim.x) {
    int h = base + tid;
    int c = h < H ? hcnt[h] : 0;
    int o = c > 0 ? 1 : 0;
    // pack (count, occupied) scan: two scans
    int vc = c, vo = o;
    for (int d = 1; d < 32; d <<= 1) {
      int tc = __shfl_up_sync(0xffffffffu, vc, d), to = __shfl_up_sync(0xffffffffu, vo, d);
      if (lane >= d) { vc += tc; vo += to; }
    }
    if (lane == 31) { warp_tot[wid] = vc; warp_occ[wid] = vo; }
    __syncthreads();
    if (wid == 0) {
      int xc = lane < nw ? warp_tot[lane] : 0, xo = lane < nw ? warp_occ[lane] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        int tc = __shfl_up_sync(0xffffffffu, xc, d), to = __shfl_up_sync(0xffffffffu, xo, d);
        if (lane >= d) { xc += tc; xo += to; }
      }
      if (lane < nw) { warp_tot[lane] = xc; warp_occ[lane] = xo; }
    }
    __syncthreads();
    int pre_c = (wid > 0 ? warp_tot[wid - 1] : 0) + vc - c + carry_sum;
    int pre_o = (wid > 0 ? warp_occ[wid - 1] : 0) + vo - o + carry_occ;
    if (h < H) {
      hstart[h] = pre_c;
      if (o) occ[pre_o] = h;
    }
    __syncthreads();
    if (tid == 0) { carry_sum += warp_tot[nw - 1]; carry_occ += warp_occ[nw - 1]; }
    __syncthreads();
  }
  if (tid == 0) counts[0] = carry_occ;
  // chunk offsets over the s batch rows (s <= 1024 = blockDim)
  __syncthreads();
  {
    int j = tid;
    int nch = 0;
    if (j < s) {
      int deg = indptr[j + 1] - indptr[j];
      nch = deg > 0 ? (deg + kChunk - 1) / kChunk : 1;
    }
    int v = nch;
    for (int d = 1; d < 32; d <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int x = lane < nw ? warp_tot[lane] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += t;
      }
      if (lane < nw) warp_tot[lane] = x;
    }
    __syncthreads();
    int excl = (wid > 0 ? warp_tot[wid - 1] : 0) + v - nch;
    if (j < s) {
      chunk_off[j] = excl;
      for (int c = 0; c < nch; ++c) chunk_row[excl + c] = j;
    }
    if (j == s - 1) { chunk_off[s] = excl + nch; counts[1] = excl + nch; }
  }
}

__global__ void k_group_fill(const int* __restrict__ slot, const int* __restrict__ rank_tmp,
                             const int* __restrict__ hstart, const int* __restrict__ rowid, int64_t nnz,
                             int* __restrict__ tmp_j, int* __restrict__ tmp_e, const int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz || failed(status)) return;
  int pos = hstart[slot[e]] + rank_tmp[e];
  tmp_j[pos] = rowid[e];
  tmp_e[pos] = (int)e;
}

// Deterministic order inside a group: position = number of entries of the
// group with a smaller batch row (rows are distinct within a group).
__global__ void k_group_rank(const int* __restrict__ tmp_j, const int* __restrict__ tmp_e,
                             const int* __restrict__ slot, const int* __restrict__ hstart,
                             const int* __restrict__ hcnt, const void* __restrict__ values, int vdtype,
                             int64_t nnz, int* __restrict__ seg_j, double* __restrict__ seg_v,
                             const int* status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz || failed(status)) return;
  int e = tmp_e[p];
  int h = slot[e];
  int st = hstart[h], cnt = hcnt[h];
  int j = tmp_j[p];
  int r = 0;
  for (int q = st; q < st + cnt; ++q) r += tmp_j[q] < j;
  seg_j[st + r] = j;
  seg_v[st + r] = load_val<double>(values, vdtype, e);
}

__global__ void k_hash_clear(int* __restrict__ hkey, int* __restrict__ hcnt, int H) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < H) {
    hkey[t] = -1;
    hcnt[t] = 0;
  }
}

void launch_group(const svlcov_csr& b, int logH, const SideScratch& w, int* status, cudaStream_t st) {
  int H = 1 << logH;
  note_launches(1);
  k_hash_clear<<<(int)cdiv(H, 256), 256, 0, st>>>(w.hkey, w.hcnt, H);
  int64_t nnz = b.nnz;
  if (nnz > 0) {   // (no zero-block launch for an empty batch)
    note_launches(1);
    k_hash_insert<<<(int)cdiv(nnz, 256), 256, 0, st>>>(b.indices, nnz, logH, w.hkey, w.hcnt, w.slot,
                                                       w.rank_tmp, status);
  }
  note_launches(1);
  k_group_scan<<<1, 1024, 0, st>>>(w.hcnt, H, w.hstart, w.occ, b.indptr, b.rows, w.chunk_off, w.chunk_row,
                                   w.counts, status);
  if (nnz > 0) {
    note_launches(1);
    k_group_fill<<<(int)cdiv(nnz, 256), 256, 0, st>>>(w.slot, w.rank_tmp, w.hstart, w.rowid, nnz, w.tmp_j,
                                                      w.tmp_e, status);
    note_launches(1);
    k_group_rank<<<(int)cdiv(nnz, 256), 256, 0, st>>>(w.tmp_j, w.tmp_e, w.slot, w.hstart, w.hcnt, b.values,
                                                      b.values_dtype, nnz, w.seg_j, w.seg_v, status);
  }
}

// ---------------------------------------------------------------------------
// a1 + a2, fused: one warp per chunk of <= kChunk nonzeros of one batch row j.
//  * gather (Lemma 1): Ppart[c][:] = sum_e v_e X'[i_e, :], lanes over the k
//    columns, accumulated in the storage's accumulator type (FP32 for FP32 /
//    BF16 storage, FP64 for FP64 storage);
//  * Gram (Lemma 2 inner products): SEpart[c][j'] = sum_e v_e E[j', i_e],
//    walking the group of i_e; products and sums in FP64 (exact products of
//    FP32 values), accumulated in a per-warp shared-memory row.
template <typename TS, int KV>
__global__ void k_gather_gram(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                              const void* __restrict__ values, int vdtype, int s, const TS* __restrict__ Xp,
                              int k, const int* __restrict__ chunk_off, const int* __restrict__ chunk_row,
                              const int* __restrict__ counts, const int* __restrict__ slot,
                              const int* __restrict__ hstart, const int* __restrict__ hcnt,
                              const int* __restrict__ seg_j, const double* __restrict__ seg_v,
                              typename Acc<TS>::type* __restrict__ Ppart, double* __restrict__ SEpart,
                              const int* status) {
  using A = typename Acc<TS>::type;
  extern __shared__ double se_buf_all[];
  if (failed(status)) return;
  int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int c = blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= counts[1]) return;
  double* buf = se_buf_all + (size_t)wib * s;
  int j = chunk_row[c];
  int64_t r0 = indptr[j], r1 = indptr[j + 1];
  int64_t e0 = r0 + (int64_t)(c - chunk_off[j]) * kChunk;
  int64_t e1 = min(e0 + kChunk, r1);
  for (int q = lane; q < s; q += 32) buf[q] = 0.0;
  A acc[KV];
#pragma unroll
  for (int t = 0; t < KV; ++t) acc[t] = (A)0;
  __syncwarp();
  for (int64_t e = e0; e < e1; ++e) {
    int i = indices[e];
    double v = load_val<double>(values, vdtype, e);
    const TS* row = Xp + (int64_t)i * k;
#pragma unroll
    for (int t = 0; t < KV; ++t) {
      int a = lane * KV + t;
      if (a < k) acc[t] += (A)v * (A)to_f64(row[a]);
    }
    int h = slot[e];
    int st = hstart[h], cnt = hcnt[h];
    for (int q = st + lane; q < st + cnt; q += 32) buf[seg_j[q]] += v * seg_v[q];
    __syncwarp();
  }
#pragma unroll
  for (int t = 0; t < KV; ++t) {
    int a = lane * KV + t;
    if (a < k) Ppart[(int64_t)c * k + a] = acc[t];
  }
  for (int q = lane; q < s; q += 32) SEpart[(int64_t)c * s + q] = buf[q];
}

// Per batch row j: P[:, j] = sum of its chunk partials (in chunk order),
// S_E[:, j] = sum of its Gram partials, C0[:, j] = W^T P[:, j], e2[j] = S_E[j,j].
template <typename A, typename TC>
__global__ void k_reduce_c0(const A* __restrict__ Ppart, const double* __restrict__ SEpart,
                            const int* __restrict__ chunk_off, int s, int k, const TC* __restrict__ W,
                            TC* __restrict__ P, TC* __restrict__ SE, TC* __restrict__ C0, TC* __restrict__ e2,
                            const int* status) {
  if (failed(status)) return;
  __shared__ double pj[kMaxK];
  int j = blockIdx.x;
  int c0 = chunk_off[j], c1 = chunk_off[j + 1];
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    A sum = (A)0;
    for (int c = c0; c < c1; ++c) sum += Ppart[(int64_t)c * k + a];
    pj[a] = (double)sum;
    P[(int64_t)j * k + a] = (TC)sum;
  }
  for (int q = threadIdx.x; q < s; q += blockDim.x) {
    double sum = 0.0;
    for (int c = c0; c < c1; ++c) sum += SEpart[(int64_t)c * s + q];
    SE[(int64_t)j * s + q] = (TC)sum;
    if (q == j) e2[j] = (TC)sum;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    TC sum = (TC)0;
    const TC* wa = W + (int64_t)a * k;  // column a of W (col-major)
    for (int b2 = 0; b2 < k; ++b2) sum += wa[b2] * (TC)pj[b2];
    C0[(int64_t)j * k + a] = sum;
  }
}

template <typename TS, typename TC>
void launch_gather_gram(const svlcov_csr& b, const TS* Xp, int k, const TC* W, const SideScratch& w, TC* P,
                        TC* SE, TC* C0, TC* e2, int* status, cudaStream_t st) {
  using A = typename Acc<TS>::type;
  int s = b.rows;
  if (s <= 0) return;
  int wpb = 4;
  int64_t chunks_ub = max_chunks(s, b.nnz);
  size_t smem = (size_t)wpb * s * sizeof(double);
  int grid = (int)cdiv(chunks_ub, wpb);
  int kv = (k + 31) / 32;
#define GG_LAUNCH(KV)                                                                                         \
  {                                                                                                           \
    auto fn = k_gather_gram<TS, KV>;                                                                          \
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    note_launches(1);                                                                                          \
    fn<<<grid, wpb * 32, smem, st>>>(b.indptr, b.indices, b.values, b.values_dtype, s, Xp, k, w.chunk_off,    \
                                     w.chunk_row, w.counts, w.slot, w.hstart, w.hcnt, w.seg_j, w.seg_v,       \
                                     (A*)w.Ppart, w.SEpart, status);                                          \
  }
  if (kv <= 1) GG_LAUNCH(1) else if (kv == 2) GG_LAUNCH(2) else if (kv == 3) GG_LAUNCH(3) else GG_LAUNCH(4)
#undef GG_LAUNCH
  note_launches(1);
  k_reduce_c0<A, TC><<<s, 128, 0, st>>>((const A*)w.Ppart, w.SEpart, w.chunk_off, s, k, W, P, SE, C0, e2, status);
}

// ---------------------------------------------------------------------------
// a7: sparse matrix addition X'[i, :] += sum_j E[j, i] M[j, :] (Eq. 1, second
// term, in the extended decomposition: B F[k:] U''^-1 = E (X F[k:] U''^-1)).
// One warp per touched row i (one group); the group's entries are summed in
// batch-row order, then one read-modify-write of the row.  No atomics.
template <typename TS, typename TC, int KV>
__global__ void k_scatter(TS* __restrict__ Xp, int k, const TC* __restrict__ Mt, const int* __restrict__ occ,
                          const int* __restrict__ counts, const int* __restrict__ hkey,
                          const int* __restrict__ hstart, const int* __restrict__ hcnt,
                          const int* __restrict__ seg_j, const double* __restrict__ seg_v, const int* status) {
  using A = typename Acc<TS>::type;
  if (failed(status)) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= counts[0]) return;
  int h = occ[warp];
  int i = hkey[h];
  int st = hstart[h], cnt = hcnt[h];
  A acc[KV];
#pragma unroll
  for (int t = 0; t < KV; ++t) acc[t] = (A)0;
  for (int q = st; q < st + cnt; ++q) {
    int j = seg_j[q];
    A v = (A)seg_v[q];
    const TC* mj = Mt + (int64_t)j * k;
#pragma unroll
    for (int t = 0; t < KV; ++t) {
      int a = lane * KV + t;
      if (a < k) acc[t] += v * (A)mj[a];
    }
  }
  TS* row = Xp + (int64_t)i * k;
#pragma unroll
  for (int t = 0; t < KV; ++t) {
    int a = lane * KV + t;
    if (a < k) row[a] = from_f64<TS>((double)((A)to_f64(row[a]) + acc[t]));
  }
}

template <typename TS, typename TC>
void launch_scatter(TS* Xp, int k, const TC* Mt, int64_t nnz, const SideScratch& w, const int* status,
                    cudaStream_t st) {
  if (nnz <= 0) return;
  int wpb = 8;
  int grid = (int)cdiv(nnz, wpb);
  int kv = (k + 31) / 32;
#define SC_LAUNCH(KV)                                                                                          \
  {                                                                                                            \
    note_launches(1);                                                                                          \
    k_scatter<TS, TC, KV><<<grid, wpb * 32, 0, st>>>(Xp, k, Mt, w.occ, w.counts, w.hkey, w.hstart, w.hcnt,     \
                                                     w.seg_j, w.seg_v, status);                                \
  }
  if (kv <= 1) SC_LAUNCH(1) else if (kv == 2) SC_LAUNCH(2) else if (kv == 3) SC_LAUNCH(3) else SC_LAUNCH(4)
#undef SC_LAUNCH
}

// ---------------------------------------------------------------------------
// a8: append s new rows (N = rows W^-1) at row offset row0.
template <typename TS, typename TC>
__global__ void k_append(TS* __restrict__ Xp, int64_t row0, int k, int s, const TC* __restrict__ Nt,
                         const int* status) {
  if (failed(status)) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)s * k) return;
  Xp[row0 * k + t] = from_f64<TS>((double)Nt[t]);
}

template <typename TS, typename TC>
void launch_append(TS* Xp, int64_t row0, int k, int s, const TC* Nt, const int* status, cudaStream_t st) {
  if (s <= 0) return;
  int64_t n = (int64_t)s * k;
  note_launches(1);
  k_append<TS, TC><<<(int)cdiv(n, 256), 256, 0, st>>>(Xp, row0, k, s, Nt, status);
}

// ---------------------------------------------------------------------------
// Row times small matrix: out[r, :] = X'[src(r), :] W (k x k, col-major).
// Used for the identity reset (X' <- X' W in place, when *do_reset), for
// materialising U = U' U'' and for row queries.  One warp per row, W staged
// in shared memory.
template <typename TS, typename TC, typename TO>
__global__ void k_rowmul(const TS* __restrict__ Xp, int64_t rows, int k, const TC* __restrict__ W,
                         TO* __restrict__ out, const int32_t* __restrict__ idx, int64_t src_rows,
                         const int* do_reset, const int* status, int* err) {
  using A = typename Acc<TS>::type;  // FP32 math for FP32/BF16 storage, FP64 for FP64 storage
  extern __shared__ __align__(16) unsigned char rm_smem[];
  A* wsm = (A*)rm_smem;
  if (do_reset && *(volatile const int*)do_reset == 0) return;
  if (status && failed(status)) return;
  int nw = blockDim.x >> 5, wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // W row-major in shared memory (wsm[b * k + a] = W(b, a)): lanes, which
  // own consecutive output columns a, then read consecutive words
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int b2 = t / k, a = t - b2 * k;
    wsm[t] = (A)W[(int64_t)a * k + b2];
  }
  A* xrow = wsm + k * k + wib * kMaxK;
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * nw + wib; r < rows; r += (int64_t)gridDim.x * nw) {
    int64_t src = r;
    if (idx) {
      src = idx[r];
      if (src < 0 || src >= src_rows) {
        if (lane == 0 && err) flag(err, SVLCOV_DEV_BAD_CSR);
        for (int a = lane; a < k; a += 32) out[r * k + a] = (TO)0;
        continue;
      }
    }
    for (int a = lane; a < k; a += 32) xrow[a] = (A)to_f64(Xp[src * k + a]);
    __syncwarp();
    for (int a = lane; a < k; a += 32) {
      A sum = (A)0;
      for (int b2 = 0; b2 < k; ++b2) sum = fma(xrow[b2], wsm[(int64_t)b2 * k + a], sum);
      out[r * k + a] = from_f64<TO>((double)sum);
    }
    __syncwarp();
  }
}

template <typename TS, typename TC>
void launch_reset(TS* Xp, int64_t rows, int k, const TC* Wn, const int* do_reset, const int* status,
                  cudaStream_t st) {
  if (rows <= 0) return;
  if constexpr (sizeof(TS) != 8) {
    if (rowmul_tc_ok((int)sizeof(TS), k)) {   // the dense fold X' <- X' W on the tensor cores
      launch_rowmul_tc<TS, TC, TS>(Xp, rows, k, Wn, Xp, do_reset, status, st);
      return;
    }
  }
  int nw = 8;
  size_t smem = sizeof(typename Acc<TS>::type) * ((size_t)k * k + nw * kMaxK);
  auto fn = k_rowmul<TS, TC, TS>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int grid = (int)std::min<int64_t>(cdiv(rows, nw), 152 * 4);
  note_launches(1);
  fn<<<grid, nw * 32, smem, st>>>(Xp, rows, k, Wn, Xp, nullptr, rows, do_reset, status, nullptr);
}

template <typename TS, typename TC>
void launch_materialize(const TS* Xp, int64_t rows, int64_t src_rows, int k, const TC* W, void* out,
                        int out_dtype, const int32_t* idx, cudaStream_t st, int* err) {
  if (rows <= 0) return;
  if constexpr (sizeof(TS) != 8) {
    if (!idx && rowmul_tc_ok((int)sizeof(TS), k)) {   // every row: U = U' W on the tensor cores
      // as on the other path, a status bit set earlier (e.g. by a query) does not stop the write-out
      if (out_dtype == SVLCOV_FP64) launch_rowmul_tc<TS, TC, double>(Xp, rows, k, W, (double*)out, nullptr, nullptr, st);
      else launch_rowmul_tc<TS, TC, float>(Xp, rows, k, W, (float*)out, nullptr, nullptr, st);
      return;
    }
  }
  int nw = 8;
  size_t smem = sizeof(typename Acc<TS>::type) * ((size_t)k * k + nw * kMaxK);
  int grid = (int)std::min<int64_t>(cdiv(rows, nw), 152 * 8);
  if (out_dtype == SVLCOV_FP64) {
    auto fn = k_rowmul<TS, TC, double>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launches(1);
    fn<<<grid, nw * 32, smem, st>>>(Xp, rows, k, W, (double*)out, idx, src_rows, nullptr, nullptr, err);
  } else {
    auto fn = k_rowmul<TS, TC, float>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    note_launches(1);
    fn<<<grid, nw * 32, smem, st>>>(Xp, rows, k, W, (float*)out, idx, src_rows, nullptr, nullptr, err);
  }
}

template <typename TS>
__global__ void k_convert_in(const void* __restrict__ src, int src_dtype, TS* __restrict__ dst, int64_t count) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double v = src_dtype == SVLCOV_FP64 ? ((const double*)src)[t] : (double)((const float*)src)[t];
  dst[t] = from_f64<TS>(v);
}

template <typename TS>
void launch_convert_in(const void* src, int src_dtype, TS* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return;
  note_launches(1);
  k_convert_in<TS><<<(int)cdiv(count, 256), 256, 0, st>>>(src, src_dtype, dst, count);
}

// ---- explicit instantiations ------------------------------------------------
#define INST_TS_TC(TS, TC)                                                                                     \
  template void launch_gather_gram<TS, TC>(const svlcov_csr&, const TS*, int, const TC*, const SideScratch&,   \
                                           TC*, TC*, TC*, TC*, int*, cudaStream_t);                            \
  template void launch_scatter<TS, TC>(TS*, int, const TC*, int64_t, const SideScratch&, const int*,           \
                                       cudaStream_t);                                                          \
  template void launch_append<TS, TC>(TS*, int64_t, int, int, const TC*, const int*, cudaStream_t);           \
  template void launch_reset<TS, TC>(TS*, int64_t, int, const TC*, const int*, const int*, cudaStream_t);     \
  template void launch_materialize<TS, TC>(const TS*, int64_t, int64_t, int, const TC*, void*, int,         \
                                           const int32_t*, cudaStream_t, int*);
INST_TS_TC(double, double)
INST_TS_TC(double, float)
INST_TS_TC(float, double)
INST_TS_TC(float, float)
INST_TS_TC(__nv_bfloat16, double)
INST_TS_TC(__nv_bfloat16, float)
template void launch_convert_in<double>(const void*, int, double*, int64_t, cudaStream_t);
template void launch_convert_in<float>(const void*, int, float*, int64_t, cudaStream_t);
template void launch_convert_in<__nv_bfloat16>(const void*, int, __nv_bfloat16*, int64_t, cudaStream_t);

}  // namespace svl

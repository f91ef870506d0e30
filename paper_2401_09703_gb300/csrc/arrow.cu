// SVD_k of the Rayleigh-Ritz matrix of a one-vector step (s = 1, the
// streaming granularity of Section 4): K = [[Sigma, c], [0, rho]] with
// Sigma = diag(sigma_1 >= ... >= sigma_k >= 0), c = C0 (k) and rho = R (the
// scalar residual norm; Algorithm 3 with s = 1, Algorithm 11 as Algorithm 3
// on A^T).  Then K K^T = D + z z^T with D = diag(sigma^2, 0) and z = [c; rho]:
// a rank-one change of a diagonal matrix, whose eigenvalues are the roots of
// the secular equation 1 + sum_i z_i^2 / (d_i - lambda) = 0 (Bunch, Nielsen &
// Sorensen, Numer. Math. 31, 1978), one in each interval between poles.
// Instead of (k+1)^3 Jacobi sweeps: O(k) work per root, all roots at once.
//
// Steps (FP64 throughout):
//  1. deflation (one CTA): z_i negligible -> (sigma_i, e_i, e_i) is a
//     singular triplet; two poles closer than the tolerance -> a rotation in
//     their plane zeroes one z component (on both sides when both are Sigma
//     directions with equal sigma; on the left only when the pole is 0, i.e.
//     sigma_i ~ 0 against the new direction);
//  2. roots (one warp per root, many CTAs): lambda_j = pole + tau with tau
//     solved by safeguarded Newton / bisection on the secular function in the
//     shifted variable, so that every difference d_i - lambda_j is formed
//     from the exact pole differences (no cancellation);
//  3. the vector of z that the computed roots make exact (Loewner's formula,
//     as in Gu & Eisenstat, SIAM J. Matrix Anal. Appl. 16, 1995), which keeps
//     the eigenvectors numerically orthogonal; ranks of all values;
//  4. vectors: u_j = (z^_i / (d_i - lambda_j))_i and, from K^T u = theta v,
//     v_j = ((sigma_i z^_i / (d_i - lambda_j))_{i<k}, -1), both normalised,
//     rotated back; the leading k triplets are written out (F, Theta, G as
//     the Jacobi path writes them: (k+1) x k column-major, Theta descending).
//  5. a kept zero value whose right vector is not defined by the formula (a
//     zero sigma_i together with rho = 0) gets the orthogonal complement of
//     the other kept right vectors (a null vector of K).
#include <cmath>

#include "kernels.cuh"

namespace svl {

namespace {

constexpr int AR_MAXN = SVLCOV_MAX_K + 1;
constexpr double AR_EPS = 2.220446049250313e-16;

// kind of a reduced index: a Sigma direction (0..k-1) or the new direction k
struct ArrowWork {
  int n;                  // k + 1
  int m;                  // non-deflated count
  int degenerate;         // a kept zero value needs the complement (step 5)
  int nrot;               // rotations recorded
  int idx[AR_MAXN];       // reduced index r -> original index (non-deflated first, descending d)
  double d[AR_MAXN];      // poles of the non-deflated indices (descending)
  double z[AR_MAXN];      // z after the rotations, non-deflated indices
  double zh[AR_MAXN];     // Loewner z
  double lam[AR_MAXN];    // eigenvalues: roots (r < m), deflated values (r >= m)
  double tau[AR_MAXN];    // root r = d[org[r]] + tau[r]
  int org[AR_MAXN];       // pole index of the shift of root r
  int rank[AR_MAXN];      // output position of value r (descending), >= k: dropped
  int rot_p[AR_MAXN], rot_q[AR_MAXN], rot_two[AR_MAXN];
  double rot_c[AR_MAXN], rot_s[AR_MAXN];
};

// At shift tau from pole o: the pole's own term -z_o^2 / tau, and the sum psi
// of the other terms z_i^2 / ((d_i - d_o) - tau) with its derivative, by one
// warp; f = 1 + psi - z_o^2 / tau is the secular function.
__device__ __forceinline__ void secular(const ArrowWork& w, int o, double tau, int lane, double& psi, double& dpsi) {
  double s = 0.0, ds = 0.0;
  for (int i = lane; i < w.m; i += 32) {
    if (i == o) continue;
    const double del = (w.d[i] - w.d[o]) - tau;
    const double q = w.z[i] / del;
    s = fma(q, w.z[i], s);     // z^2 / del
    ds = fma(q, q, ds);        // z^2 / del^2
  }
  psi = warp_sum(s);
  dpsi = warp_sum(ds);
}

}  // namespace

// ---- 1. deflation -------------------------------------------------------------
__global__ void k_arrow_setup(const double* __restrict__ sigma, const double* __restrict__ c,
                              const double* __restrict__ rho, int k, ArrowWork* __restrict__ w,
                              const int* status) {
  if (failed(status)) return;
  if (threadIdx.x != 0) return;
  const int n = k + 1;
  double d[AR_MAXN], z[AR_MAXN];
  int def[AR_MAXN];
  double zn2 = 0.0;
  for (int i = 0; i < n; ++i) {
    d[i] = i < k ? sigma[i] * sigma[i] : 0.0;
    z[i] = i < k ? c[i] : *rho;
    zn2 = fma(z[i], z[i], zn2);
    def[i] = 0;
  }
  // Deflation in the scale of K (so that it perturbs K, not only K K^T, by at
  // most the tolerance): z_i with |z_i| <= tol, and poles whose singular
  // values differ by at most tol, are treated as exact deflations.
  const double zn = sqrt(zn2);
  const double s1 = k > 0 ? fmax(sigma[0], 0.0) : 0.0;
  const double tol = 8.0 * AR_EPS * fmax(s1, zn);
  for (int i = 0; i < n; ++i)
    if (!(fabs(z[i]) > tol)) def[i] = 1;       // also z = 0 overall
  // Close poles, in order: the previous kept index p and the next kept i.  d is
  // descending (sigma descending, the new direction's pole 0 last).
  int nrot = 0;
  int p = -1;
  for (int i = 0; i < n; ++i) {
    if (def[i]) continue;
    const double sp = p >= 0 ? sigma[p] : 0.0, si = i < k ? sigma[i] : 0.0;
    if (p >= 0 && sp - si <= tol) {
      // rotate in the (p, i) plane so that z_i takes the norm and z_p = 0:
      // the rotation moves K by at most (sigma_p - sigma_i) |cs sn| <= tol
      const double r = hypot(z[p], z[i]);
      const double cs = z[i] / r, sn = z[p] / r;
      w->rot_p[nrot] = p;
      w->rot_q[nrot] = i;
      w->rot_c[nrot] = cs;
      w->rot_s[nrot] = sn;
      w->rot_two[nrot] = i < k ? 1 : 0;   // both Sigma directions: the right side turns too
      ++nrot;
      z[i] = r;
      z[p] = 0.0;
      def[p] = 1;
    }
    p = i;
  }
  int m = 0;
  for (int i = 0; i < n; ++i)
    if (!def[i]) {
      w->idx[m] = i;
      w->d[m] = d[i];
      w->z[m] = z[i];
      ++m;
    }
  int r = m;
  for (int i = 0; i < n; ++i)
    if (def[i]) {
      w->idx[r] = i;
      w->lam[r] = d[i];
      w->z[r] = 0.0;
      ++r;
    }
  w->n = n;
  w->m = m;
  w->nrot = nrot;
  w->degenerate = 0;
}

// ---- 2. roots: one warp per root ----------------------------------------------
__global__ void __launch_bounds__(32) k_arrow_roots(ArrowWork* __restrict__ w, double* __restrict__ dlt,
                                                    const int* status) {
  if (failed(status)) return;
  const int j = blockIdx.x, lane = threadIdx.x;
  const int m = w->m;
  if (j >= m) return;
  // root j lies in (d_j, d_{j-1}) (descending), the first one in (d_0, d_0 + |z|^2)
  double zn2 = 0.0;
  for (int i = lane; i < m; i += 32) zn2 = fma(w->z[i], w->z[i], zn2);
  zn2 = warp_sum(zn2);
  const double width = j == 0 ? zn2 : w->d[j - 1] - w->d[j];
  // which pole is the root closer to: the sign of f at the midpoint
  double psi, dpsi;
  int o = j;
  double lo = 0.0, hi = width;          // tau bracket relative to pole o
  if (j > 0) {
    secular(*w, j, 0.5 * width, lane, psi, dpsi);
    const double fm = 1.0 + psi - w->z[j] * w->z[j] / (0.5 * width);
    if (fm < 0.0) {                     // f increases on the interval: root above the midpoint
      o = j - 1;                        // shift to the upper pole
      lo = -0.5 * width;
      hi = 0.0;
    } else {
      lo = 0.0;
      hi = 0.5 * width;
    }
  }
  // Iteration exact in the pole's own term (Bunch, Nielsen & Sorensen's
  // osculatory idea): psi is linearised around the current tau and
  // 1 + psi + psi' (t - tau) - z_o^2 / t = 0 solved for t (the root of the
  // right sign of a quadratic), safeguarded by the bracket [lo, hi].
  const double zo2 = w->z[o] * w->z[o];
  double t = 0.5 * (lo + hi);
  for (int it = 0; it < 80; ++it) {
    secular(*w, o, t, lane, psi, dpsi);
    const double f = 1.0 + psi - zo2 / t;
    if (f == 0.0) break;
    if (f < 0.0) lo = t;
    else hi = t;
    const double b = 1.0 + psi - dpsi * t;
    double tn;
    if (!(dpsi > 0.0)) tn = zo2 / b;
    else {
      const double disc = sqrt(fma(b, b, 4.0 * dpsi * zo2));
      if (o == j)   // positive root
        tn = b > 0.0 ? 2.0 * zo2 / (b + disc) : (disc - b) / (2.0 * dpsi);
      else          // negative root
        tn = b > 0.0 ? -(b + disc) / (2.0 * dpsi) : 2.0 * zo2 / (b - disc);
    }
    if (fabs(tn - t) <= 4.0 * AR_EPS * fabs(t)) break;   // converged: the step is rounding (t stays)
    // outside the bracket (or NaN): bisect; the first root may sit on its
    // upper end d_0 + |z|^2 (a single non-deflated pole)
    if (!(tn > lo && (tn < hi || (j == 0 && tn == hi)))) tn = 0.5 * (lo + hi);
    t = tn;
    if (hi - lo <= 4.0 * AR_EPS * fmax(fabs(lo), fabs(hi))) break;
  }
  if (lane == 0) {
    w->tau[j] = t;
    w->org[j] = o;
    w->lam[j] = w->d[o] + t;
  }
  const double dorg = w->d[o];
  for (int i = lane; i < m; i += 32) dlt[(size_t)j * AR_MAXN + i] = (w->d[i] - dorg) - t;   // d_i - lambda_j
}

// ---- 3. Loewner z and ranks (one CTA) -----------------------------------------
__global__ void k_arrow_zhat(ArrowWork* __restrict__ w, const double* __restrict__ dlt, int k, const int* status) {
  if (failed(status)) return;
  const int m = w->m, n = w->n;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    // z^_i^2 = prod_j (lambda_j - d_i) / prod_{j != i} (d_j - d_i), as a product
    // of ratios of interlaced factors (each O(1))
    double pr = -dlt[(size_t)i * AR_MAXN + i];
    for (int j = 0; j < m; ++j) {
      if (j == i) continue;
      pr *= -dlt[(size_t)j * AR_MAXN + i] / (w->d[j] - w->d[i]);
    }
    const double a = sqrt(fmax(pr, 0.0));
    w->zh[i] = w->z[i] >= 0.0 ? a : -a;
  }
  // rank of every value, descending, ties by reduced index
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = w->lam[r];
    int rk = 0;
    for (int q = 0; q < n; ++q) {
      const double u = w->lam[q];
      rk += (u > v) || (u == v && q < r);
    }
    w->rank[r] = rk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // a kept zero value whose right vector the formulas leave undefined: a
    // deflated new direction (rho ~ 0) ranked among the leading k
    int deg = 0;
    for (int r = m; r < n; ++r)
      if (w->idx[r] == k && w->rank[r] < k && !(w->lam[r] > 0.0)) deg = 1;
    w->degenerate = deg;
  }
}

// ---- 4. vectors: one CTA of 128 threads per value -----------------------------
__global__ void __launch_bounds__(128) k_arrow_vectors(const ArrowWork* __restrict__ w, const double* __restrict__ dlt,
                                                       const double* __restrict__ sigma, int k, double* __restrict__ F,
                                                       double* __restrict__ theta, double* __restrict__ G,
                                                       const int* status) {
  if (failed(status)) return;
  const int r = blockIdx.x;
  const int n = w->n, m = w->m;
  if (r >= n) return;
  const int rk = w->rank[r];
  if (rk >= k) return;   // not among the leading k
  __shared__ double u[AR_MAXN], v[AR_MAXN], red[2][4];
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) {
    u[i] = 0.0;
    // a root's right vector has -1 at the new direction, deflated or not
    // (K^T u there is sum_i z_i u_i = -1 by the secular equation)
    v[i] = (r < m && i == k) ? -1.0 : 0.0;
  }
  __syncthreads();
  if (r < m) {
    // u (in the reduced order) = z^ / (d - lambda_r); v = sigma z^ / (d - lambda_r) on the Sigma directions
    for (int i = tid; i < m; i += blockDim.x) {
      const double del = dlt[(size_t)r * AR_MAXN + i];
      const int oi = w->idx[i];
      const double q = w->zh[i] / del;
      u[oi] = q;
      if (oi < k) v[oi] = sigma[oi] * q;
    }
  } else {
    const int oi = w->idx[r];
    if (tid == 0) {
      u[oi] = 1.0;
      if (oi < k) v[oi] = 1.0;   // (sigma_i, e_i, e_i); the new direction's right vector: step 5
    }
  }
  __syncthreads();
  // rotations back, last recorded first: (p, q) with e_p' = cs e_p - sn e_q ... the
  // forward rotation mapped (z_p, z_q) to (0, r): [z_p'; z_q'] = [cs -sn; sn cs] [z_p; z_q]
  if (tid == 0) {
    for (int t = w->nrot - 1; t >= 0; --t) {
      const int p = w->rot_p[t], q = w->rot_q[t];
      const double cs = w->rot_c[t], sn = w->rot_s[t];
      const double up = u[p], uq = u[q];
      u[p] = cs * up + sn * uq;
      u[q] = -sn * up + cs * uq;
      if (w->rot_two[t]) {
        const double vp = v[p], vq = v[q];
        v[p] = cs * vp + sn * vq;
        v[q] = -sn * vp + cs * vq;
      }
    }
  }
  __syncthreads();
  double su = 0.0, sv = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    su = fma(u[i], u[i], su);
    sv = fma(v[i], v[i], sv);
  }
  su = warp_sum(su);
  sv = warp_sum(sv);
  if ((tid & 31) == 0) { red[0][tid >> 5] = su; red[1][tid >> 5] = sv; }
  __syncthreads();
  const int nw = (int)(blockDim.x >> 5);
  double nu = 0.0, nv = 0.0;
  for (int q = 0; q < nw; ++q) { nu += red[0][q]; nv += red[1][q]; }
  const double iu = nu > 0.0 ? 1.0 / sqrt(nu) : 0.0;
  const double iv = nv > 0.0 ? 1.0 / sqrt(nv) : 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    F[(size_t)rk * n + i] = u[i] * iu;
    G[(size_t)rk * n + i] = v[i] * iv;
  }
  if (tid == 0) theta[rk] = sqrt(fmax(w->lam[r], 0.0));
}

// ---- 5. the complement for a kept zero value (one CTA; usually returns at once)
__global__ void k_arrow_complement(const ArrowWork* __restrict__ w, int k, double* __restrict__ G,
                                   const int* status) {
  if (failed(status) || !w->degenerate) return;
  const int n = w->n;
  int rk = -1;
  for (int r = w->m; r < n; ++r)
    if (w->idx[r] == k) rk = w->rank[r];
  if (rk < 0 || rk >= k) return;
  __shared__ double v[AR_MAXN];
  __shared__ double dot;
  // the unit vector least covered by the other kept right vectors, then
  // Gram-Schmidt (twice) against them
  if (threadIdx.x == 0) {
    int best = 0;
    double bcov = 2.0;
    for (int i = 0; i < n; ++i) {
      double cov = 0.0;
      for (int c = 0; c < k; ++c)
        if (c != rk) cov += G[(size_t)c * n + i] * G[(size_t)c * n + i];
      if (cov < bcov) { bcov = cov; best = i; }
    }
    for (int i = 0; i < n; ++i) v[i] = i == best ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < k; ++c) {
      if (c == rk) continue;
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += G[(size_t)c * n + i] * v[i];
        dot = s;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] -= dot * G[(size_t)c * n + i];
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    dot = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) G[(size_t)rk * n + i] = v[i] * dot;
}

// ---- Algorithm 2 for one vector ------------------------------------------------
__global__ void k_s1_orth(const double* __restrict__ S, const double* __restrict__ e2, const double* __restrict__ C0,
                          int k, double tau, double* __restrict__ R, double* __restrict__ X, double* __restrict__ CQ,
                          unsigned char* defl1, unsigned char* defl2, int* status) {
  if (failed(status)) return;
  const double s0 = S[0], r0 = e2[0];
  const bool finite = isfinite(s0);
  // R8: the direction is dropped when its residual is at most tau of its norm
  const bool drop = !finite || !(s0 > tau * r0) || !(r0 > 0.0);
  const double rr = drop ? 0.0 : sqrt(s0);
  const double x = drop ? 0.0 : 1.0 / rr;
  for (int i = threadIdx.x; i < k; i += blockDim.x) CQ[i] = C0[i] * x;
  if (threadIdx.x == 0) {
    if (!finite) flag(status, SVLCOV_DEV_NOT_PD);
    R[0] = rr;
    X[0] = x;
    defl1[0] = defl2[0] = drop ? 1 : 0;
  }
}

void launch_s1_orth(const double* S, const double* e2, const double* C0, int k, double tau, double* R, double* X,
                    double* CQ, unsigned char* defl1, unsigned char* defl2, int* status, cudaStream_t st) {
  note_launches(1);
  k_s1_orth<<<1, 128, 0, st>>>(S, e2, C0, k, tau, R, X, CQ, defl1, defl2, status);
}

size_t arrow_work_bytes() {
  return ((sizeof(ArrowWork) + 255) & ~(size_t)255) + sizeof(double) * (size_t)AR_MAXN * AR_MAXN + 256;
}

// F, theta, G = SVD_k of K = [[diag(sigma), c], [0, rho]] (sigma, c: device, k;
// rho: device scalar), F and G (k+1) x k column-major.
void launch_arrow_svd(const double* sigma, const double* c, const double* rho, int k, double* F, double* theta,
                      double* G, void* work, const int* status, cudaStream_t st) {
  ArrowWork* w = (ArrowWork*)work;
  double* dlt = (double*)((char*)work + ((sizeof(ArrowWork) + 255) & ~(size_t)255));
  const int n = k + 1;
  note_launches(5);
  k_arrow_setup<<<1, 32, 0, st>>>(sigma, c, rho, k, w, status);
  k_arrow_roots<<<n, 32, 0, st>>>(w, dlt, status);
  k_arrow_zhat<<<1, 128, 0, st>>>(w, dlt, k, status);
  k_arrow_vectors<<<n, 128, 0, st>>>(w, dlt, sigma, k, F, theta, G, status);
  k_arrow_complement<<<1, 128, 0, st>>>(w, k, G, status);
}

}  // namespace svl

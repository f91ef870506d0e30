"""The -GKL and -RPI variants of the sparse update, FP64 (TEST INFRASTRUCTURE
ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
leg, never by the product path).

Appendix "Approximating the Augmented Space": instead of an orthonormal basis
of the whole residual Z = (I - U U^T) E (Algorithm 2, s vectors), an l-vector
basis Q of a Krylov (Golub-Kahan-Lanczos, Algorithm 9) or power-iteration
(RPI, Algorithm 10) subspace of Z is built in SV-LCOV form, together with
P = Z^T Q (s x l).  The update then takes SVD_k of

    K = [[Sigma, U^T E], [0, P^T]]        ((k + l) x (k + s))

and folds it as Algorithm 3 does (appendix "Add columns with approximated
augmented space"); the weight update (appendix "Update weights with
approximated augmented space") uses
    K = diag(Sigma, 0) + [U^T D; P_D^T] [V^T E; P_E^T]^T   ((k + l) square).
With l = rank(Z) the subspace is all of range(Z) and the update is exact.

The random quantities of the methods are inputs: GKL's starting vector p_1
(s) and RPI's starting matrix (s x l, orthonormalised here before use).

Readings (also listed in the design notes):
* R18  breakdown: a zero alpha_i or beta_i (the Krylov space is exhausted) ends
       the recurrence; the remaining Lanczos vectors are zero and contribute
       nothing.  "Zero" is below 1e-13 times the largest alpha/beta so far.
* R19  Algorithm 10 orthonormalises P after forming Q = Z P; Q's span does not
       depend on it, so P is orthonormalised first, as in the dense RPI listing.
* R20  the right factor of K holds V's k columns and s identity columns, so the
       appended rows are G[k:] V''^-1 exactly as in Algorithm 3; the U side adds
       B' F[k:] U''^-1, with B' the l SV-LCOV vectors of Q.
"""
from __future__ import annotations

import numpy as np

from .dense import svd_k
from .svlcov import Batch, State, svlcov_qr

_BREAKDOWN = 1e-13


def gkl_svlcov(B0: np.ndarray, C0: np.ndarray, l: int, p1: np.ndarray):
    """Algorithm 9: l Golub-Kahan-Lanczos steps on the tuples (b, c).

    B0 (r x s) and C0 (k x s) hold the batch E and U^T E.  Step i:
      b'_i = B0 p_i - beta_{i-1} b'_{i-1},   c'_i = C0 p_i - beta_{i-1} c'_{i-1}
      alpha_i = sqrt(<b'_i, b'_i> - <c'_i, c'_i>)            (Lemma 2)
      (b'_i, c'_i) /= alpha_i
      p_{i+1} = B0^T b'_i - C0^T c'_i - alpha_i p_i
      p_{i+1} orthogonalised against p_1..p_i (Gram-Schmidt, one pass)
      beta_i = |p_{i+1}|,  p_{i+1} /= beta_i
    Returns B' (r x l), C' (k x l) -- Q = B' - U C' -- and
    P = P_{l+1} H^T with H = diag(alpha) + superdiag(beta)  (l x (l + 1)).
    """
    r, s = B0.shape
    k = C0.shape[0]
    Bq = np.zeros((r, l))
    Cq = np.zeros((k, l))
    Pm = np.zeros((s, l + 1))
    alpha = np.zeros(l)
    beta = np.zeros(l)
    Pm[:, 0] = p1 / np.linalg.norm(p1)
    scale = 0.0
    beta_prev = 0.0
    stopped = False
    for i in range(l):
        if stopped:
            break
        b = B0 @ Pm[:, i]
        c = C0 @ Pm[:, i]
        if i > 0:
            b = b - beta_prev * Bq[:, i - 1]
            c = c - beta_prev * Cq[:, i - 1]
        a2 = b @ b - c @ c
        a = np.sqrt(max(a2, 0.0))
        scale = max(scale, a)
        if a <= _BREAKDOWN * scale or a == 0.0:      # R18
            stopped = True
            break
        alpha[i] = a
        Bq[:, i] = b / a
        Cq[:, i] = c / a
        p = B0.T @ Bq[:, i] - C0.T @ Cq[:, i] - a * Pm[:, i]
        for j in range(i + 1):
            p = p - (Pm[:, j] @ p) * Pm[:, j]
        bt = np.linalg.norm(p)
        scale = max(scale, bt)
        if bt <= _BREAKDOWN * scale:                  # R18
            beta[i] = 0.0
            stopped = True
        else:
            beta[i] = bt
            Pm[:, i + 1] = p / bt
        beta_prev = beta[i]
    H = np.zeros((l, l + 1))
    H[np.arange(l), np.arange(l)] = alpha
    H[np.arange(l), np.arange(1, l + 1)] = beta
    P = Pm @ H.T
    return Bq, Cq, P, dict(alpha=alpha, beta=beta, Pm=Pm)


def rpi_svlcov(B0: np.ndarray, C0: np.ndarray, l: int, t: int, P0: np.ndarray, tau: float = 1e-12):
    """Algorithm 10: t randomized power iterations on the tuples (b, c).

    Each iteration: P <- orthonormal basis of P (library QR; R19);
    (B', C') = (B0 P, C0 P); (B', C') <- Algorithm 2 on them (SV-LCOV QR);
    P <- B0^T B' - C0^T C' (= Z^T Q).  Returns B' (r x l), C' (k x l), P (s x l).
    """
    P = np.array(P0, dtype=np.float64, copy=True)
    Bq = Cq = None
    for _ in range(t):
        P, _ = np.linalg.qr(P)
        Bq, Cq, _, _ = svlcov_qr(B0 @ P, C0 @ P, tau)
        P = B0.T @ Bq - C0.T @ Cq
    return Bq, Cq, P


def _basis(method: str, B0, C0, l: int, t: int, start):
    if method == "gkl":
        Bq, Cq, P, _ = gkl_svlcov(B0, C0, l, start)
    elif method == "rpi":
        Bq, Cq, P = rpi_svlcov(B0, C0, l, t, start)
    else:
        raise ValueError(method)
    return Bq, Cq, P


class ApproxState(State):
    """The extended decomposition updated with an approximate augmented space."""

    @staticmethod
    def init(U, sigma, V, tau=1e-12, reset_threshold=1e8) -> "ApproxState":
        st = State.init(U, sigma, V, tau, reset_threshold)
        return ApproxState(st.Up, st.Wu, st.sigma, st.Wv, st.Vp, st.tau, st.reset_threshold)

    def add_cols_approx(self, indptr, indices, values, s: int, method: str, l: int, start, t: int = 3):
        """Appendix "Add columns with approximated augmented space"."""
        k = self.k
        bt = Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Up, self.Wu, bt)                  # U^T E_c
        Bq, Cq, P = _basis(method, bt.B0, C0, l, t, start)
        K = np.zeros((k + l, k + s))
        K[:k, :k] = np.diag(self.sigma)
        K[:k, k:] = C0
        K[k:, k:] = P.T
        F, th, G = svd_k(K, k)
        self._fold("u", F[:k] - Cq @ F[k:], bt.support, Bq @ F[k:])
        self.sigma = th
        self._append("v", G[:k], G[k:])                           # R20
        self.log.append(dict(op="cols_" + method, K=K, P=P, C0=C0, F=F, G=G, theta=th))

    def add_rows_approx(self, indptr, indices, values, s: int, method: str, l: int, start, t: int = 3):
        """Add rows: the add-columns variant on A^T (as Algorithm 11 is Algorithm 3 on A^T)."""
        k = self.k
        bt = Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Vp, self.Wv, bt)                  # V^T E_r^T
        Bq, Cq, P = _basis(method, bt.B0, C0, l, t, start)
        K = np.zeros((k + s, k + l))                              # K of A^T, transposed
        K[:k, :k] = np.diag(self.sigma)
        K[k:, :k] = C0.T
        K[k:, k:] = P
        F, th, G = svd_k(K, k)
        self._append("u", F[:k], F[k:])
        self.sigma = th
        self._fold("v", G[:k] - Cq @ G[k:], bt.support, Bq @ G[k:])
        self.log.append(dict(op="rows_" + method, K=K, P=P, C0=C0, F=F, G=G, theta=th))

    def update_weights_approx(self, D, E, s: int, method: str, l: int, start, t: int = 3):
        """Appendix "Update weights with approximated augmented space"; the
        same start serves both sides."""
        k = self.k
        bd = Batch.from_csr(*D, s)
        be = Batch.from_csr(*E, s)
        C0d = self._project(self.Up, self.Wu, bd)
        Bd, Cd, Pd = _basis(method, bd.B0, C0d, l, t, start)
        C0e = self._project(self.Vp, self.Wv, be)
        Be, Ce, Pe = _basis(method, be.B0, C0e, l, t, start)
        K = np.zeros((k + l, k + l))
        K[:k, :k] = np.diag(self.sigma)
        K += np.vstack([C0d, Pd.T]) @ np.vstack([C0e, Pe.T]).T
        F, th, G = svd_k(K, k)
        self._fold("u", F[:k] - Cd @ F[k:], bd.support, Bd @ F[k:])
        self.sigma = th
        self._fold("v", G[:k] - Ce @ G[k:], be.support, Be @ G[k:])
        self.log.append(dict(op="weights_" + method, K=K, F=F, G=G, theta=th))

    def apply_approx(self, op: str, batch, method: str, l: int, start, t: int = 3):
        if op == "cols":
            self.add_cols_approx(batch.indptr, batch.indices, batch.values, batch.rows, method, l, start, t)
        elif op == "rows":
            self.add_rows_approx(batch.indptr, batch.indices, batch.values, batch.rows, method, l, start, t)
        elif op == "weights":
            D, E = batch
            self.update_weights_approx((D.indptr, D.indices, D.values), (E.indptr, E.indices, E.values), D.rows,
                                       method, l, start, t)
        else:
            raise ValueError(op)

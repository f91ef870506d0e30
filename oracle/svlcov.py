"""The paper's sparse update (SV-LCOV), FP64, written for checking by eye.

Section 3.1: a vector z = (I - U U^T) b of the augmented matrix is held as
the tuple (b, c) with c = U^T b (Definition 1).  Scaling, addition and the
inner product <(b1,c1),(b2,c2)> = <b1,b2> - <c1,c2> (Lemma 2) act on the
tuple; by Lemma 3 this inner product equals the one of the vectors it stands
for, so Gram-Schmidt can run on tuples (Algorithm 2).

Section 3.2: the factors are kept as U = U' U'' and V = V' V'' (U' m x k,
U'' k x k; only the products are orthonormal).  Algorithms 3 (add columns),
11 (add rows) and 4 (update weights) update U'', V'', Sigma, add a sparse
matrix to U' or V' and append rows, never rewriting all of U' or V'.

Sparse vectors.  All b-vectors of one batch live on the union of the batch's
nonzero positions (its support, r positions).  They are stored as a dense
r x s array over that support: every operation then costs O(r) per vector,
which is the O(nnz) cost Lemma 2 states.

Readings where the paper is silent or inconsistent (the same list is kept in
the design notes):
* R1  the K block of Algorithms 3/4/11 is the projection C0 = U^T E; the folds
      use the C returned by Algorithm 2 (rescaled during Gram-Schmidt).
* R2  the sparse add of Algorithms 3 and 11 uses the *updated* U''/V'' inverse.
* R3  "append new columns G[k:] V''^-1 to V'" appends s *rows* to V'.
* R4  Algorithm 4 writes its SVD output as Sigma_k (it is Theta_k) and uses
      U''^-1 in its V-side sparse add; the V side uses the updated V''^-1.
* R5  Algorithm 11's block "E_r^T V_k" is dimensionally E_r V_k = C0^T.
* R8  Gram-Schmidt deflation: when alpha^2 <= tau * <e_i, e_i> (or e_i = 0)
      the vector is dropped: R's row i is 0, b_i and c_i are set to 0.
* R9  the extended decomposition is reset (U' <- U' U'', U'' <- I) when
      cond_1(U'') exceeds a threshold (Section 3.2 names resetting to the
      identity as the remedy for ill-conditioning, without a rule).
* R17 the new U'' = U'' (F[:k] - C F[k:]) (or V'' G[:k]) can be singular --
      e.g. when an old direction leaves the top k entirely -- and then the
      U''^-1 of Algorithm 3's sparse add does not exist.  The check of R9 is made on the new
      factor before it is inverted; if it fails, the fold is done as a reset
      (U' <- U' U''_new, then the sparse add without U''^-1, U'' <- I).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dense import svd_k


def _xinv(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    """X W^-1 by an LU solve (library routine)."""
    return np.linalg.solve(W.T, X.T).T


def cond1(W: np.ndarray) -> float:
    return float(np.linalg.norm(W, 1) * np.linalg.norm(np.linalg.inv(W), 1))


@dataclass
class Batch:
    """Update vectors e_1..e_s restricted to their joint support.

    ``support`` (r,) are the positions (rows of U' or V'); ``B0`` (r x s) holds
    e_j on the support (column j = update vector j)."""
    support: np.ndarray
    B0: np.ndarray

    @staticmethod
    def from_csr(indptr, indices, values, s: int) -> "Batch":
        indptr = np.asarray(indptr, dtype=np.int64)
        indices = np.asarray(indices, dtype=np.int64)
        values = np.asarray(values, dtype=np.float64)
        support = np.unique(indices)
        pos = np.searchsorted(support, indices)
        B0 = np.zeros((support.shape[0], s))
        for j in range(s):
            a, b = indptr[j], indptr[j + 1]
            B0[pos[a:b], j] = values[a:b]
        return Batch(support, B0)


def svlcov_qr(B0: np.ndarray, C0: np.ndarray, tau: float = 1e-12):
    """Algorithm 2: modified Gram-Schmidt on the tuples (b_j, c_j).

    For i = 1..s: alpha = sqrt(<b_i,b_i> - <c_i,c_i>), R_ii = alpha, scale the
    tuple by 1/alpha; then for every later j: beta = <b_i,b_j> - <c_i,c_j>,
    R_ij = beta, (b_j, c_j) -= beta (b_i, c_i).  The loop over j is written as
    array operations over all later j at once (same operations, same order
    for each j).  Deflation R8 as described in the module header.

    Returns B (r x s), C (k x s) with Q = B - U C orthonormal (up to dropped
    columns), R (s x s upper triangular) with (I - U U^T) E = Q R, and the list
    of dropped indices.
    """
    B = np.array(B0, dtype=np.float64, copy=True)
    C = np.array(C0, dtype=np.float64, copy=True)
    s = B.shape[1]
    R = np.zeros((s, s))
    e2 = np.einsum("ij,ij->j", B0, B0)            # <e_i, e_i>
    dropped = []
    for i in range(s):
        alpha2 = B[:, i] @ B[:, i] - C[:, i] @ C[:, i]
        if e2[i] == 0.0 or alpha2 <= tau * e2[i]:
            B[:, i] = 0.0
            C[:, i] = 0.0
            dropped.append(i)
            continue
        alpha = np.sqrt(alpha2)
        R[i, i] = alpha
        B[:, i] /= alpha
        C[:, i] /= alpha
        if i + 1 < s:
            beta = B[:, i] @ B[:, i + 1:] - C[:, i] @ C[:, i + 1:]
            R[i, i + 1:] = beta
            B[:, i + 1:] -= np.outer(B[:, i], beta)
            C[:, i + 1:] -= np.outer(C[:, i], beta)
    return B, C, R, dropped


@dataclass
class State:
    """Extended decomposition U' U'' Sigma V''^T V'^T (Section 3.2), FP64."""
    Up: np.ndarray
    Wu: np.ndarray
    sigma: np.ndarray
    Wv: np.ndarray
    Vp: np.ndarray
    tau: float = 1e-12
    reset_threshold: float = 1e8
    resets: int = 0
    log: list = field(default_factory=list)

    @staticmethod
    def init(U, sigma, V, tau=1e-12, reset_threshold=1e8) -> "State":
        """U' <- U, V' <- V, U'' = V'' = I (Section 3.2)."""
        k = U.shape[1]
        return State(np.array(U, dtype=np.float64, copy=True), np.eye(k),
                     np.array(sigma, dtype=np.float64, copy=True), np.eye(k),
                     np.array(V, dtype=np.float64, copy=True), tau, reset_threshold)

    @property
    def k(self) -> int:
        return self.Wu.shape[0]

    # Query (Theorem 1): a row of U is U'[i] U'' in O(k^2)
    def query_u(self, idx):
        return self.Up[np.asarray(idx)] @ self.Wu

    def query_v(self, idx):
        return self.Vp[np.asarray(idx)] @ self.Wv

    def factors(self):
        return self.Up @ self.Wu, self.sigma.copy(), self.Vp @ self.Wv

    # Turning a batch into SV-LCOV form (Lemma 1): c = U^T b gathers the rows
    # of U' at the batch's nonzeros, then multiplies by U''.
    @staticmethod
    def _project(Xp, W, batch: Batch):
        return W.T @ (Xp[batch.support].T @ batch.B0)

    def _ill(self, W: np.ndarray) -> bool:
        """R9/R17: a small factor is ill-conditioned when it is singular,
        non-finite or cond_1 exceeds the reset threshold."""
        if not np.all(np.isfinite(W)):
            return True
        try:
            return cond1(W) > self.reset_threshold
        except np.linalg.LinAlgError:
            return True

    def _fold(self, side: str, X: np.ndarray, support: np.ndarray, Badd: np.ndarray):
        """W <- W X, then X'[support] += Badd W^-1 (Section 3.2, Eq. 1 split).

        R17: when the new W is ill-conditioned (R9) the fold is done as a
        reset instead -- X' <- X' (W X), X'[support] += Badd, W <- I -- which
        gives the same product X' W."""
        if side == "u":
            Wn = self.Wu @ X
            if self._ill(Wn):
                self.Up = self.Up @ Wn
                self.Up[support] += Badd
                self.Wu = np.eye(self.k)
                self.resets += 1
            else:
                self.Wu = Wn
                self.Up[support] += _xinv(Badd, Wn)
        else:
            Wn = self.Wv @ X
            if self._ill(Wn):
                self.Vp = self.Vp @ Wn
                self.Vp[support] += Badd
                self.Wv = np.eye(self.k)
                self.resets += 1
            else:
                self.Wv = Wn
                self.Vp[support] += _xinv(Badd, Wn)

    def _append(self, side: str, X: np.ndarray, rows: np.ndarray):
        """W <- W X, then append the rows ``rows W^-1`` (the append step of
        Algorithms 3 and 11); reset variant as in ``_fold`` (R17)."""
        if side == "u":
            Wn = self.Wu @ X
            if self._ill(Wn):
                self.Up = np.vstack([self.Up @ Wn, rows])
                self.Wu = np.eye(self.k)
                self.resets += 1
            else:
                self.Wu = Wn
                self.Up = np.vstack([self.Up, _xinv(rows, Wn)])
        else:
            Wn = self.Wv @ X
            if self._ill(Wn):
                self.Vp = np.vstack([self.Vp @ Wn, rows])
                self.Wv = np.eye(self.k)
                self.resets += 1
            else:
                self.Wv = Wn
                self.Vp = np.vstack([self.Vp, _xinv(rows, Wn)])

    def add_cols(self, indptr, indices, values, s: int):
        """Algorithm 3 (add columns E_c, m x s; row j of the CSR is column j)."""
        k = self.k
        bt = Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Up, self.Wu, bt)                  # U^T E_c
        B, C, R, dropped = svlcov_qr(bt.B0, C0, self.tau)
        K = np.zeros((k + s, k + s))
        K[:k, :k] = np.diag(self.sigma)
        K[:k, k:] = C0
        K[k:, k:] = R
        F, th, G = svd_k(K, k)
        self._fold("u", F[:k] - C @ F[k:], bt.support, B @ F[k:])  # R2
        self.sigma = th
        self._append("v", G[:k], G[k:])  # R3
        self.log.append(dict(op="cols", K=K, R=R, C0=C0, C=C, F=F, G=G, theta=th, dropped=dropped))

    def add_rows(self, indptr, indices, values, s: int):
        """Algorithm 11 (add rows E_r, s x n; row j of the CSR is new row j)."""
        k = self.k
        bt = Batch.from_csr(indptr, indices, values, s)           # columns of E_r^T
        C0 = self._project(self.Vp, self.Wv, bt)                  # V^T E_r^T
        B, C, R, dropped = svlcov_qr(bt.B0, C0, self.tau)
        K = np.zeros((k + s, k + s))  # R5
        K[:k, :k] = np.diag(self.sigma)
        K[k:, :k] = C0.T
        K[k:, k:] = R.T
        F, th, G = svd_k(K, k)
        self._append("u", F[:k], F[k:])
        self.sigma = th
        self._fold("v", G[:k] - C @ G[k:], bt.support, B @ G[k:])
        self.log.append(dict(op="rows", K=K, R=R, C0=C0, C=C, F=F, G=G, theta=th, dropped=dropped))

    def update_weights(self, D, E, s: int):
        """Algorithm 4 (A + D E_m^T; D and E are CSR triples (indptr, indices,
        values) holding D^T and E_m^T)."""
        k = self.k
        bd = Batch.from_csr(*D, s)
        be = Batch.from_csr(*E, s)
        C0d = self._project(self.Up, self.Wu, bd)
        Bd, Cd, Rd, dd = svlcov_qr(bd.B0, C0d, self.tau)
        C0e = self._project(self.Vp, self.Wv, be)
        Be, Ce, Re, de = svlcov_qr(be.B0, C0e, self.tau)
        K = np.zeros((k + s, k + s))
        K[:k, :k] = np.diag(self.sigma)
        K += np.vstack([C0d, Rd]) @ np.vstack([C0e, Re]).T
        F, th, G = svd_k(K, k)
        self._fold("u", F[:k] - Cd @ F[k:], bd.support, Bd @ F[k:])
        self.sigma = th
        self._fold("v", G[:k] - Ce @ G[k:], be.support, Be @ G[k:])  # R4
        self.log.append(dict(op="weights", K=K, Rd=Rd, Re=Re, C0d=C0d, C0e=C0e, F=F, G=G,
                             theta=th, dropped=(dd, de)))

    def apply(self, op: str, batch):
        """Dispatch one (op, batch) item as produced by ``synth``."""
        if op == "cols":
            self.add_cols(batch.indptr, batch.indices, batch.values, batch.rows)
        elif op == "rows":
            self.add_rows(batch.indptr, batch.indices, batch.values, batch.rows)
        elif op == "weights":
            D, E = batch
            self.update_weights((D.indptr, D.indices, D.values), (E.indptr, E.indices, E.values), D.rows)
        else:
            raise ValueError(op)

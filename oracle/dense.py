"""Dense FP64 references: the definition of the update and Zha-Simon.

Orientation of the batches (see ``synth.generators``): a batch of ``s`` update
vectors is given as an (s x d) array whose row ``j`` is update vector ``j``.
For new columns this is E_c^T, for new rows E_r, for a weight update D^T and
E_m^T.
"""
from __future__ import annotations

import numpy as np


def svd_k(K: np.ndarray, k: int):
    """Rank-k truncated SVD (Section 2: SVD_k keeps the k largest singular
    values with their vectors).

    Canonical form (the paper leaves order, sign and ties open): singular
    values descending, ties kept in their original order (stable sort); each
    left vector is signed so that its largest-magnitude entry is positive
    (the lowest index wins a tie in magnitude), and the right vector is
    flipped with it.  Returns F (rows x k), theta (k,), G (cols x k).
    """
    F, th, Gt = np.linalg.svd(K, full_matrices=False)
    order = np.argsort(-th, kind="stable")
    F, th, G = F[:, order], th[order], Gt[order].T
    F, th, G = F[:, :k].copy(), th[:k].copy(), G[:, :k].copy()
    for j in range(F.shape[1]):
        i = int(np.argmax(np.abs(F[:, j])))
        if F[i, j] < 0:
            F[:, j] *= -1.0
            G[:, j] *= -1.0
    return F, th, G


def qr_nonneg(Z: np.ndarray):
    """Reduced Householder QR with the sign of each R_ii made non-negative
    (the QR with R_ii > 0 is unique for full column rank)."""
    Q, R = np.linalg.qr(Z, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d, R * d[:, None]


# ---------------------------------------------------------------------------
# The definition (Section 3.3, "maintaining an approximate rank-k truncated
# SVD"; Theorem 1): the result of an update is the rank-k truncated SVD of the
# modification applied to A_k = U diag(sigma) V^T.
# ---------------------------------------------------------------------------
def define_add_cols(U, sigma, V, EcT, k=None):
    k = U.shape[1] if k is None else k
    Ak = (U * sigma) @ V.T
    return svd_k(np.hstack([Ak, np.asarray(EcT).T]), k)


def define_add_rows(U, sigma, V, Er, k=None):
    k = U.shape[1] if k is None else k
    Ak = (U * sigma) @ V.T
    return svd_k(np.vstack([Ak, np.asarray(Er)]), k)


def define_update_weights(U, sigma, V, DT, EmT, k=None):
    k = U.shape[1] if k is None else k
    Ak = (U * sigma) @ V.T
    return svd_k(Ak + np.asarray(DT).T @ np.asarray(EmT), k)


# ---------------------------------------------------------------------------
# Zha-Simon (Section 2.1): augment with an orthonormal basis of the augmented
# matrix (I - U U^T) E obtained by a dense QR, take the SVD of the small
# projected matrix, rotate.
# ---------------------------------------------------------------------------
def zha_simon_add_cols(U, sigma, V, EcT):
    """[A_k E_c] = [U Q] [[Sigma, U^T E_c], [0, R]] blockdiag(V, I)^T."""
    E = np.asarray(EcT, dtype=np.float64).T          # m x s
    k = U.shape[1]
    s = E.shape[1]
    C = U.T @ E
    Q, R = qr_nonneg(E - U @ C)
    K = np.zeros((k + s, k + s))
    K[:k, :k] = np.diag(sigma)
    K[:k, k:] = C
    K[k:, k:] = R
    F, th, G = svd_k(K, k)
    Un = np.hstack([U, Q]) @ F
    n = V.shape[0]
    Vn = np.vstack([V @ G[:k], G[k:]])                # blockdiag(V, I) G
    assert Vn.shape[0] == n + s
    return Un, th, Vn, dict(K=K, C=C, R=R, Q=Q, F=F, G=G)


def zha_simon_add_rows(U, sigma, V, Er):
    """[A_k; E_r] = blockdiag(U, I) [[Sigma, 0], [E_r V, R^T]] [V Q]^T with
    Q R = (I - V V^T) E_r^T."""
    Er = np.asarray(Er, dtype=np.float64)              # s x n
    k = U.shape[1]
    s = Er.shape[0]
    C = V.T @ Er.T                                     # k x s
    Q, R = qr_nonneg(Er.T - V @ C)
    K = np.zeros((k + s, k + s))
    K[:k, :k] = np.diag(sigma)
    K[k:, :k] = C.T
    K[k:, k:] = R.T
    F, th, G = svd_k(K, k)
    Un = np.vstack([U @ F[:k], F[k:]])                 # blockdiag(U, I) F
    Vn = np.hstack([V, Q]) @ G
    return Un, th, Vn, dict(K=K, C=C, R=R, Q=Q, F=F, G=G)


def zha_simon_update_weights(U, sigma, V, DT, EmT):
    """A_k + D E_m^T = [U Q_D] (diag(Sigma, 0) + [U^T D; R_D][V^T E_m; R_E]^T) [V Q_E]^T."""
    D = np.asarray(DT, dtype=np.float64).T              # m x s
    E = np.asarray(EmT, dtype=np.float64).T             # n x s
    k = U.shape[1]
    s = D.shape[1]
    assert E.shape[1] == s
    CD = U.T @ D
    CE = V.T @ E
    QD, RD = qr_nonneg(D - U @ CD)
    QE, RE = qr_nonneg(E - V @ CE)
    K = np.zeros((k + s, k + s))
    K[:k, :k] = np.diag(sigma)
    K += np.vstack([CD, RD]) @ np.vstack([CE, RE]).T
    F, th, G = svd_k(K, k)
    Un = np.hstack([U, QD]) @ F
    Vn = np.hstack([V, QE]) @ G
    return Un, th, Vn, dict(K=K, CD=CD, CE=CE, RD=RD, RE=RE, F=F, G=G)

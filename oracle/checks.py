"""Error measures for comparing truncated SVDs (FP64, numpy).

TEST INFRASTRUCTURE ONLY (part of the oracle): the rulers every parity test
uses.  Their definitions follow the tolerance reading of the step's result
(a truncated SVD is compared by its singular values and, across a gap in the
spectrum, by the principal angles between singular subspaces).  Each is
pinned against known answers in tests/test_oracle_checks.py.
"""
from __future__ import annotations

import numpy as np


def orth_err(X: np.ndarray) -> float:
    """max |X^T X - I|."""
    return float(np.max(np.abs(X.T @ X - np.eye(X.shape[1]))))


def sigma_rel_err(s: np.ndarray, s_ref: np.ndarray, floor: float = 1e-12) -> float:
    """max_i |s_i - s_ref_i| / s_ref_i over s_ref_i > floor * s_ref_1."""
    s = np.asarray(s, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    keep = s_ref > floor * s_ref[0]
    if not keep.any():
        return 0.0
    return float(np.max(np.abs(s[keep] - s_ref[keep]) / s_ref[keep]))


def gapped_prefix(s_ref: np.ndarray, rel_gap: float = 1e-3) -> int:
    """Largest k' such that (s_k' - s_k'+1) / s_1 >= rel_gap (k' = k when the
    last value clears the gap against zero).  Subspace angles are only
    defined across such a gap."""
    s_ref = np.asarray(s_ref, dtype=np.float64)
    k = s_ref.shape[0]
    ext = np.append(s_ref, 0.0)
    for kp in range(k, 0, -1):
        if (ext[kp - 1] - ext[kp]) >= rel_gap * s_ref[0]:
            return kp
    return 0


def max_sin_angle(X: np.ndarray, Xref: np.ndarray, rank_tol: float = 1e-10) -> float:
    """Sine of the largest principal angle between range(X) and range(Xref),
    two blocks of the same width k'.  The columns need not be orthonormal:
    both blocks are orthonormalised first (the angles belong to the
    subspaces).  The sine is the 2-norm of (I - Qr Qr^T) Q.  A block whose
    columns do not span k' dimensions (a zero or dependent column) has lost a
    direction, and the angle to it is taken as 90 degrees: 1.0 is returned.
    An empty block (k' = 0) compares nothing and returns 0."""
    if X.shape[1] != Xref.shape[1]:
        raise ValueError("blocks of different width")
    if X.shape[1] == 0:
        return 0.0
    Q, R = np.linalg.qr(X)
    Qr, Rr = np.linalg.qr(Xref)
    for r in (np.abs(np.diag(R)), np.abs(np.diag(Rr))):
        if r.min() <= rank_tol * max(r.max(), np.finfo(float).tiny):
            return 1.0
    res = Q - Qr @ (Qr.T @ Q)
    return float(np.linalg.norm(res, 2))


def compare(U, s, V, Uref, sref, Vref, rel_gap: float = 1e-3) -> dict:
    """Singular-value error and subspace sines on the gapped leading block."""
    kp = gapped_prefix(sref, rel_gap)
    return dict(sigma=sigma_rel_err(s, sref), k_prime=kp,
                sin_u=max_sin_angle(U[:, :kp], Uref[:, :kp]),
                sin_v=max_sin_angle(V[:, :kp], Vref[:, :kp]))


def projector_err(X: np.ndarray, Y: np.ndarray) -> float:
    """max |X X^T - Y Y^T| (sign- and rotation-invariant comparison)."""
    return float(np.max(np.abs(X @ X.T - Y @ Y.T)))

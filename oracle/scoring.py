"""Scores of index pairs from a truncated SVD (FP64, numpy).

TEST INFRASTRUCTURE ONLY (part of the oracle).  The inference step of the
paper's downstream tasks (Section 4, task setup of link prediction and
collaborative filtering): a pair (i, j) is scored by the inner product
U[i]^T Sigma V[j] of its two representations; for an undirected graph the
larger of the two directions is taken.  Pinned in tests/test_oracle_scoring.py
(exact-rank reconstruction: the scores are the matrix entries themselves).
"""
from __future__ import annotations

import numpy as np


def score_pairs(U, sigma, V, rows, cols, symmetric=False):
    """out[p] = sum_l U[rows[p], l] sigma[l] V[cols[p], l] (and the max with
    the (cols[p], rows[p]) direction when symmetric)."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    out = np.array([float(np.sum(U[i] * s * V[j])) for i, j in zip(rows, cols)])
    if symmetric:
        rev = np.array([float(np.sum(U[j] * s * V[i])) for i, j in zip(rows, cols)])
        out = np.maximum(out, rev)
    return out

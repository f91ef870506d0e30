"""Pins of the oracle's pair scores (oracle/scoring.py): for a matrix of
exact rank <= k its rank-k SVD reproduces it, so the score of (i, j) is the
entry A[i, j] itself -- before and after an update step that keeps the rank
within k (the exact-recovery property of the update).  A planted mistake
(Sigma^1/2 instead of Sigma, the roles of U and V swapped, no max over the
two directions) fails one of them."""
import numpy as np
import pytest

import synth
from oracle import scoring, svlcov


def _low_rank(m, n, r, g):
    return g.standard_normal((m, r)) @ g.standard_normal((r, n))


def test_scores_reproduce_an_exact_rank_matrix():
    g = synth.rng(41)
    A = _low_rank(30, 20, 4, g)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    k = 6
    rows = g.integers(0, 30, 200)
    cols = g.integers(0, 20, 200)
    out = scoring.score_pairs(U[:, :k], s[:k], Vt[:k].T, rows, cols)
    assert np.max(np.abs(out - A[rows, cols])) < 1e-12 * np.abs(A).max()


def test_scores_after_an_update_that_keeps_the_rank():
    g = synth.rng(42)
    A = _low_rank(25, 18, 3, g)
    k = 5
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    st = svlcov.State.init(U[:, :k], s[:k], Vt[:k].T)
    # two new columns: one in range(A), one new direction (rank 3 -> 4 <= k)
    E = np.zeros((25, 2))
    E[:, 0] = A @ g.standard_normal(18)
    E[[2, 7, 11], 1] = [1.0, -2.0, 0.5]
    b = synth.csr_from_coo(*np.nonzero(E.T), E.T[np.nonzero(E.T)], 2, 25)
    st.apply("cols", b)
    Uo, so, Vo = st.factors()
    B = np.hstack([A, E])
    rows = g.integers(0, 25, 300)
    cols = g.integers(0, 20, 300)
    out = scoring.score_pairs(Uo, so, Vo, rows, cols)
    assert np.max(np.abs(out - B[rows, cols])) < 1e-10 * np.abs(B).max()


def test_symmetric_scores_take_the_larger_direction():
    g = synth.rng(43)
    X = _low_rank(12, 12, 3, g)
    U, s, Vt = np.linalg.svd(X)
    rows = np.arange(12).repeat(12)
    cols = np.tile(np.arange(12), 12)
    out = scoring.score_pairs(U[:, :3], s[:3], Vt[:3].T, rows, cols, symmetric=True)
    assert np.max(np.abs(out - np.maximum(X[rows, cols], X[cols, rows]))) < 1e-12 * np.abs(X).max()
    S = X + X.T                                             # symmetric: both directions agree
    U, s, Vt = np.linalg.svd(S)
    out = scoring.score_pairs(U[:, :6], s[:6], Vt[:6].T, rows, cols, symmetric=True)
    assert np.max(np.abs(out - S[rows, cols])) < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("wrong", ["sqrt_sigma", "swap", "no_max"])
def test_planted_scoring_mistakes_fail_a_pin(wrong):
    g = synth.rng(44)
    X = _low_rank(12, 10, 3, g)
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    U, s, V = U[:, :3], s[:3], Vt[:3].T
    rows = np.arange(10).repeat(10)
    cols = np.tile(np.arange(10), 10)
    if wrong == "sqrt_sigma":
        out = np.array([np.sum(U[i] * np.sqrt(s) * V[j]) for i, j in zip(rows, cols)])
        ref = X[rows, cols]
    elif wrong == "swap":
        out = np.array([np.sum(V[i] * s * U[j]) for i, j in zip(rows, cols)])
        ref = X[rows, cols]
    else:
        out = np.array([np.sum(U[i] * s * V[j]) for i, j in zip(rows, cols)])
        ref = np.maximum(X[rows, cols], X[cols, rows])
    assert np.max(np.abs(out - ref)) > 1e-6

"""Pins for the oracle of the -GKL and -RPI variants (approximate augmented
space, Appendix Algorithms 9 and 10 and the add-columns / update-weights
algorithms built on them), independent of the oracle's own code path:

* with l = s (the whole residual space) both variants are the exact update,
  so they must reproduce the exact sparse method step by step;
* the Lanczos relations of Golub-Kahan bidiagonalisation hold for the dense
  vectors the SV-LCOV tuples stand for (Z p_i = alpha_i q_i + beta_{i-1}
  q_{i-1}, Q orthonormal, P = Z^T Q);
* one approximate step equals the same step written densely: the textbook
  GKL / RPI on the explicit residual Z = (I - U U^T) E, then the SVD of
  [[Sigma, U^T E], [0, Q^T Z]] and U_new = [U Q] F, V_new = [[V, 0], [0, I]] G.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import approx, checks, svlcov

from tests.test_oracle_pins import _mixed_problem


def _starts(g, s, l):
    return g.standard_normal(s), g.standard_normal((s, l))


@pytest.mark.parametrize("method,t", [("gkl", 0), ("rpi", 1), ("rpi", 3)])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_full_rank_approximation_is_exact(method, t, seed):
    """l = s: Q spans all of range(Z), so every step equals the exact one."""
    U, s, V, ops = _mixed_problem(seed)
    ex = svlcov.State.init(U, s, V)
    ap = approx.ApproxState.init(U, s, V)
    g = synth.rng(100 + seed)
    for kind, b in ops:
        ss = b[0].rows if kind == "weights" else b.rows
        p1, P0 = _starts(g, ss, ss)
        ex.apply(kind, b)
        ap.apply_approx(kind, b, method, ss, p1 if method == "gkl" else P0, t=t)
        Ue, se, Ve = ex.factors()
        Ua, sa, Va = ap.factors()
        assert np.max(np.abs(sa - se)) < 1e-10 * se[0], (kind, np.max(np.abs(sa - se)))
        kp = checks.gapped_prefix(se, 1e-6)
        assert checks.projector_err(Ua[:, :kp], Ue[:, :kp]) < 1e-8
        assert checks.projector_err(Va[:, :kp], Ve[:, :kp]) < 1e-8


def _one_batch(seed, m=60, n=45, k=5, s=9, per_vec=4):
    g = synth.rng(seed)
    A = sp.random(m, n, density=0.2, random_state=seed, data_rvs=lambda x: g.standard_normal(x)).toarray()
    U, sg, V = synth.init_factors(A, k, seed)
    b = synth.random_csr_batch(s, m, per_vec, g)
    return U, sg, V, b, g


def test_gkl_lanczos_relations():
    U, sg, V, b, g = _one_batch(7)
    E = b.dense().T                                   # m x s
    st = svlcov.State.init(U, sg, V)
    bt = svlcov.Batch.from_csr(b.indptr, b.indices, b.values, b.rows)
    C0 = U.T @ E
    l = 5
    Bq, Cq, P, info = approx.gkl_svlcov(bt.B0, C0, l, g.standard_normal(b.rows))
    Q = -U @ Cq
    Q[bt.support] += Bq
    Z = E - U @ C0
    Pm, a, be = info["Pm"], info["alpha"], info["beta"]
    assert checks.orth_err(Q) < 1e-12
    assert checks.orth_err(Pm) < 1e-12
    for i in range(l):
        lhs = Z @ Pm[:, i]
        rhs = a[i] * Q[:, i] + (be[i - 1] * Q[:, i - 1] if i > 0 else 0.0)
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.linalg.norm(Z)
    assert np.max(np.abs(P - Z.T @ Q)) < 1e-12 * np.linalg.norm(Z)
    del st


def _dense_gkl(Z, l, p1):
    """Textbook Golub-Kahan-Lanczos bidiagonalisation of the explicit Z with
    full reorthogonalisation of the right vectors."""
    m, s = Z.shape
    Q = np.zeros((m, l))
    Pm = np.zeros((s, l + 1))
    Pm[:, 0] = p1 / np.linalg.norm(p1)
    beta = 0.0
    for i in range(l):
        q = Z @ Pm[:, i] - (beta * Q[:, i - 1] if i > 0 else 0.0)
        alpha = np.linalg.norm(q)
        Q[:, i] = q / alpha
        p = Z.T @ Q[:, i] - alpha * Pm[:, i]
        p -= Pm[:, :i + 1] @ (Pm[:, :i + 1].T @ p)
        beta = np.linalg.norm(p)
        Pm[:, i + 1] = p / beta
    return Q


def _dense_rpi(Z, t, P0):
    P = P0
    Q = None
    for _ in range(t):
        P, _ = np.linalg.qr(P)
        Q, _ = np.linalg.qr(Z @ P)
        P = Z.T @ Q
    return Q


@pytest.mark.parametrize("method", ["gkl", "rpi"])
def test_one_step_matches_the_dense_formulation(method):
    U, sg, V, b, g = _one_batch(11)
    k, l = U.shape[1], 4
    p1, P0 = _starts(g, b.rows, l)
    E = b.dense().T
    Z = E - U @ (U.T @ E)
    Q = _dense_gkl(Z, l, p1) if method == "gkl" else _dense_rpi(Z, 3, P0)
    K = np.zeros((k + l, k + b.rows))
    K[:k, :k] = np.diag(sg)
    K[:k, k:] = U.T @ E
    K[k:, k:] = Q.T @ Z
    Fu, th, Gt = np.linalg.svd(K)
    Fu, th, G = Fu[:, :k], th[:k], Gt[:k].T
    Ud = np.hstack([U, Q]) @ Fu
    Vbig = np.zeros((V.shape[0] + b.rows, k + b.rows))
    Vbig[:V.shape[0], :k] = V
    Vbig[V.shape[0]:, k:] = np.eye(b.rows)
    Vd = Vbig @ G
    ap = approx.ApproxState.init(U, sg, V)
    ap.add_cols_approx(b.indptr, b.indices, b.values, b.rows, method, l, p1 if method == "gkl" else P0, t=3)
    Ua, sa, Va = ap.factors()
    assert np.max(np.abs(sa - th)) < 1e-12 * th[0]
    kp = checks.gapped_prefix(th, 1e-6)
    assert checks.projector_err(Ua[:, :kp], Ud[:, :kp]) < 1e-10
    assert checks.projector_err(Va[:, :kp], Vd[:, :kp]) < 1e-10
    assert checks.orth_err(Ua) < 1e-12 and checks.orth_err(Va) < 1e-12


def test_gkl_error_shrinks_with_l():
    """Smaller approximate space, larger departure from the exact update: the
    error of the leading singular values is largest at l = 1 and zero at l = s."""
    U, sg, V, b, g = _one_batch(13, s=12)
    ex = svlcov.State.init(U, sg, V)
    ex.add_cols(b.indptr, b.indices, b.values, b.rows)
    p1 = g.standard_normal(b.rows)
    errs = []
    for l in (1, 4, b.rows):
        ap = approx.ApproxState.init(U, sg, V)
        ap.add_cols_approx(b.indptr, b.indices, b.values, b.rows, "gkl", l, p1)
        errs.append(checks.sigma_rel_err(ap.sigma, ex.sigma))
    assert errs[0] > errs[1] and errs[2] < 1e-12, errs

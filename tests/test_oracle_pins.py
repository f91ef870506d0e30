"""Pins for the FP64 CPU oracle: facts fixed by the paper and by mathematics,
independent of the oracle's own code path.

* closed-form cases of the update definition (tests/golden/);
* Lemma 3 (isometry of the SV-LCOV inner product);
* Algorithm 2's R equals the unique Householder R (R_ii > 0) of the dense
  augmented matrix;
* definition (full dense SVD) = Zha-Simon = sparse method on tiny inputs, over
  mixed trajectories of all three update kinds;
* exact recovery when the total rank stays <= k;
* orthonormality of U' U'' and V' V'' after every step;
* residuals of the updated triplets against the matrix-free operator;
* planted mistakes in the oracle are caught by these pins.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import checks, dense, svlcov

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cases.json")


def _csr(d):
    return synth.CSR(np.array(d["indptr"], dtype=np.int32), np.array(d["indices"], dtype=np.int32),
                     np.array(d["values"], dtype=np.float64), d["rows"], d["cols"])


def _apply_dense(kind, U, s, V, batch):
    if kind == "cols":
        return dense.define_add_cols(U, s, V, batch.dense())
    if kind == "rows":
        return dense.define_add_rows(U, s, V, batch.dense())
    D, E = batch
    return dense.define_update_weights(U, s, V, D.dense(), E.dense())


def _apply_zs(kind, U, s, V, batch):
    if kind == "cols":
        return dense.zha_simon_add_cols(U, s, V, batch.dense())[:3]
    if kind == "rows":
        return dense.zha_simon_add_rows(U, s, V, batch.dense())[:3]
    D, E = batch
    return dense.zha_simon_update_weights(U, s, V, D.dense(), E.dense())[:3]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_closed_form_cases(case):
    U = np.array(case["U"]); s = np.array(case["sigma"]); V = np.array(case["V"])
    if case["op"] == "weights":
        batch = (_csr(case["D"]), _csr(case["E"]))
    else:
        batch = _csr(case["batch"])
    Ue, se, Ve = np.array(case["U_out"]), np.array(case["sigma_out"]), np.array(case["V_out"])
    for impl in ("def", "zs", "sv"):
        if impl == "def":
            Uo, so, Vo = _apply_dense(case["op"], U, s, V, batch)
        elif impl == "zs":
            Uo, so, Vo = _apply_zs(case["op"], U, s, V, batch)
        else:
            st = svlcov.State.init(U, s, V)
            st.apply(case["op"], batch)
            Uo, so, Vo = st.factors()
        assert np.allclose(so, se, rtol=0, atol=1e-12), (impl, so, se)
        assert checks.projector_err(Uo, Ue) < 1e-12, impl
        assert checks.projector_err(Vo, Ve) < 1e-12, impl


# ---------------------------------------------------------------------------
def _orthonormal(m, k, g):
    Q, _ = np.linalg.qr(g.standard_normal((m, k)))
    return Q


def test_lemma3_isometry():
    """<(b1,c1),(b2,c2)> = <b1,b2> - <c1,c2> equals the inner product of the
    projected vectors (I - U U^T) b (Lemma 3)."""
    g = synth.rng(11)
    m, k = 200, 7
    U = _orthonormal(m, k, g)
    for _ in range(20):
        b1 = sp.random(m, 1, density=0.05, random_state=int(g.integers(1 << 30))).toarray().ravel()
        b2 = sp.random(m, 1, density=0.05, random_state=int(g.integers(1 << 30))).toarray().ravel()
        b2[np.nonzero(b1)[0][:2]] = 1.5          # force shared support
        c1, c2 = U.T @ b1, U.T @ b2
        z1, z2 = b1 - U @ c1, b2 - U @ c2
        assert abs((b1 @ b2 - c1 @ c2) - z1 @ z2) <= 1e-13 * max(1.0, abs(b1 @ b2))


def test_alg2_matches_householder_qr():
    """Algorithm 2's R is the unique QR factor (R_ii > 0) of the dense
    augmented matrix (I - U U^T) E, and B - U C is orthonormal."""
    g = synth.rng(12)
    m, k, s = 300, 6, 9
    U = _orthonormal(m, k, g)
    batch = synth.random_csr_batch(s, m, 8, g)
    bt = svlcov.Batch.from_csr(batch.indptr, batch.indices, batch.values, s)
    C0 = U[bt.support].T @ bt.B0
    B, C, R, dropped = svlcov.svlcov_qr(bt.B0, C0)
    assert dropped == []
    E = batch.dense().T
    Qh, Rh = dense.qr_nonneg(E - U @ (U.T @ E))
    assert np.max(np.abs(R - Rh)) < 1e-12 * np.abs(Rh).max()
    Q = -U @ C
    Q[bt.support] += B
    assert checks.orth_err(Q) < 1e-12
    assert np.max(np.abs(Q - Qh)) < 1e-11


def _mixed_problem(seed, m=36, n=28, k=4, steps=9, s_max=4):
    g = synth.rng(seed)
    A = sp.random(m, n, density=0.25, random_state=seed,
                  data_rvs=lambda x: g.standard_normal(x)).toarray()
    U, s, V = synth.init_factors(A, k, seed)
    ops = []
    mm, nn = m, n
    for t in range(steps):
        kind = ("cols", "rows", "weights")[t % 3]
        ss = int(g.integers(1, s_max + 1))
        if kind == "cols":
            b = synth.random_csr_batch(ss, mm, 3, g); nn += ss
        elif kind == "rows":
            b = synth.random_csr_batch(ss, nn, 3, g); mm += ss
        else:
            b = (synth.random_csr_batch(ss, mm, 2, g), synth.random_csr_batch(ss, nn, 2, g))
        ops.append((kind, b))
    return U, s, V, ops


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_definition_zhasimon_sparse_agree(seed):
    """Tiny mixed trajectories: the definition (dense full SVD of the updated
    matrix), Zha-Simon and the sparse method give the same triplets
    (Theorem 1 and the remark that the method reproduces Zha-Simon)."""
    U, s, V, ops = _mixed_problem(seed)
    Ud, sd, Vd = U, s, V
    Uz, sz, Vz = U, s, V
    st = svlcov.State.init(U, s, V)
    for kind, b in ops:
        Ud, sd, Vd = _apply_dense(kind, Ud, sd, Vd, b)
        Uz, sz, Vz = _apply_zs(kind, Uz, sz, Vz, b)
        st.apply(kind, b)
        Us, ss, Vs = st.factors()
        assert np.max(np.abs(sd - sz)) < 1e-12 * sd[0]
        assert np.max(np.abs(sd - ss)) < 1e-12 * sd[0]
        kp = checks.gapped_prefix(sd, 1e-6)
        for X in (Uz, Us):
            assert checks.projector_err(X[:, :kp], Ud[:, :kp]) < 1e-9
        for Y in (Vz, Vs):
            assert checks.projector_err(Y[:, :kp], Vd[:, :kp]) < 1e-9
        assert checks.orth_err(Us) < 1e-12 and checks.orth_err(Vs) < 1e-12


# ---------------------------------------------------------------------------
def _disjoint_rank_k(m, n, k, g, rank):
    """A = sum of ``rank`` sparse outer products with disjoint supports, with
    exact rank-k factors (zero singular values padded with unit vectors on
    rows/cols outside every support)."""
    rows = g.permutation(m)
    cols = g.permutation(n)
    rs = np.array_split(rows[: m // 2], rank)
    cs = np.array_split(cols[: n // 2], rank)
    U = np.zeros((m, k)); V = np.zeros((n, k)); s = np.zeros(k)
    for l in range(rank):
        a = np.zeros(m); a[rs[l]] = g.standard_normal(rs[l].shape[0])
        b = np.zeros(n); b[cs[l]] = g.standard_normal(cs[l].shape[0])
        s[l] = np.linalg.norm(a) * np.linalg.norm(b)
        U[:, l] = a / np.linalg.norm(a); V[:, l] = b / np.linalg.norm(b)
    for l in range(rank, k):
        U[rows[m - k + l], l] = 1.0
        V[cols[n - k + l], l] = 1.0
    order = np.argsort(-s, kind="stable")
    return U[:, order], s[order], V[:, order], rows, cols, rs


def test_exact_recovery_in_range():
    """E_c inside range(U): every Gram-Schmidt vector is dropped (reading R8),
    and U Theta V^T reproduces [A E] exactly."""
    g = synth.rng(21)
    m, n, k = 60, 40, 4
    U, s, V, rows, cols, rs = _disjoint_rank_k(m, n, k, g, rank=k)
    A = (U * s) @ V.T
    coef = g.standard_normal((k, 3))
    E = U @ coef                                   # m x 3, sparse (supports of U)
    Ec = synth.csr_from_coo(*np.nonzero(E.T), E.T[np.nonzero(E.T)], 3, m)
    st = svlcov.State.init(U, s, V)
    st.add_cols(Ec.indptr, Ec.indices, Ec.values, 3)
    assert st.log[-1]["dropped"] == [0, 1, 2]
    Un, sn, Vn = st.factors()
    M = np.hstack([A, E])
    assert np.linalg.norm((Un * sn) @ Vn.T - M) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(sn, np.linalg.svd(M, compute_uv=False)[:k], rtol=1e-12, atol=1e-12)


def test_exact_recovery_new_directions():
    """rank(A) = k - 2 and E adds two new directions: [A E] (columns) and
    [A; E] (rows) have rank k and are reproduced exactly."""
    g = synth.rng(22)
    m, n, k = 60, 40, 5
    U, s, V, rows, cols, rs = _disjoint_rank_k(m, n, k, g, rank=k - 2)
    A = (U * s) @ V.T
    # two new columns on rows outside every support and padding vector
    used = set(np.nonzero(np.abs(U).sum(1))[0].tolist())
    fresh = [r for r in range(m) if r not in used][:4]
    E = np.zeros((m, 2))
    E[fresh[0], 0] = 2.0; E[fresh[1], 0] = -1.0
    E[fresh[2], 1] = 0.5; E[fresh[3], 1] = 3.0
    E[:, 1] += 0.7 * E[:, 0]
    Ec = synth.csr_from_coo(*np.nonzero(E.T), E.T[np.nonzero(E.T)], 2, m)
    st = svlcov.State.init(U, s, V)
    st.add_cols(Ec.indptr, Ec.indices, Ec.values, 2)
    Un, sn, Vn = st.factors()
    M = np.hstack([A, E])
    assert np.linalg.norm((Un * sn) @ Vn.T - M) <= 1e-12 * np.linalg.norm(M)
    assert np.allclose(sn, np.linalg.svd(M, compute_uv=False)[:k], rtol=0, atol=1e-12 * sn[0])
    # rows: the same new directions appended as rows of A
    usedc = set(np.nonzero(np.abs(V).sum(1))[0].tolist())
    freshc = [c for c in range(n) if c not in usedc][:2]
    Er = np.zeros((2, n)); Er[0, freshc[0]] = 1.5; Er[1, freshc[1]] = -2.5; Er[1, freshc[0]] = 0.25
    Erc = synth.csr_from_coo(*np.nonzero(Er), Er[np.nonzero(Er)], 2, n)
    st = svlcov.State.init(U, s, V)
    st.add_rows(Erc.indptr, Erc.indices, Erc.values, 2)
    Un, sn, Vn = st.factors()
    M = np.vstack([A, Er])
    assert np.linalg.norm((Un * sn) @ Vn.T - M) <= 1e-12 * np.linalg.norm(M)


# ---------------------------------------------------------------------------
def test_c1_trajectory_residuals_and_orthonormality():
    """C1 (2000 x 1000, k = 16, 10 batches of 10 columns): after every step
    the triplets satisfy M v_i = theta_i u_i and M^T u_i = theta_i v_i for the
    matrix-free M = [U S V^T, E_c] (relative 1e-12), U and V stay orthonormal
    to 1e-12, and the definition (dense SVD of M) agrees."""
    p = synth.c1_problem()
    U, s, V = p["U"], p["sigma"], p["V"]
    st = svlcov.State.init(U, s, V)
    for kind, b in p["batches"]:
        E = b.dense().T                            # m x s
        st.apply(kind, b)
        Un, sn, Vn = st.factors()
        # M v and M^T u without forming M
        Mv = U @ (s[:, None] * (V.T @ Vn[: V.shape[0]])) + E @ Vn[V.shape[0]:]
        Mtu = np.vstack([V @ (s[:, None] * (U.T @ Un)), E.T @ Un])
        assert np.max(np.linalg.norm(Mv - Un * sn, axis=0)) <= 1e-12 * sn[0]
        assert np.max(np.linalg.norm(Mtu - Vn * sn, axis=0)) <= 1e-12 * sn[0]
        assert checks.orth_err(Un) < 1e-12 and checks.orth_err(Vn) < 1e-12
        Ud, sd, Vd = dense.define_add_cols(U, s, V, b.dense())
        assert checks.sigma_rel_err(sn, sd) < 1e-12
        cmp = checks.compare(Un, sn, Vn, Ud, sd, Vd)
        assert cmp["sin_u"] < 1e-9 and cmp["sin_v"] < 1e-9
        U, s, V = Un, sn, Vn


def test_query_rows_match_materialised_factors():
    """Theorem 1 Query: row i of U is U'[i] U''."""
    U, s, V, ops = _mixed_problem(7)
    st = svlcov.State.init(U, s, V)
    for kind, b in ops:
        st.apply(kind, b)
    Uf, sf, Vf = st.factors()
    idx = np.array([0, 3, Uf.shape[0] - 1])
    assert np.array_equal(st.query_u(idx), Uf[idx])
    idx = np.array([1, Vf.shape[0] - 1])
    assert np.array_equal(st.query_v(idx), Vf[idx])


def test_reset_is_a_noop_on_the_factors():
    """Resetting U'' to I after folding it into U' does not change U' U''."""
    U, s, V, ops = _mixed_problem(8)
    a = svlcov.State.init(U, s, V)
    b = svlcov.State.init(U, s, V, reset_threshold=1.0)   # reset at every fold
    for kind, bt in ops:
        a.apply(kind, bt)
        b.apply(kind, bt)
    assert b.resets > 0
    for x, y in zip(a.factors(), b.factors()):
        assert np.max(np.abs(x - y)) < 1e-12


def test_empty_and_duplicate_columns_are_dropped():
    g = synth.rng(31)
    m, n, k = 50, 30, 3
    A = g.standard_normal((m, n))
    U, s, V = synth.init_factors(A, k, 0)
    col = np.zeros(m); col[[3, 7, 9]] = [1.0, -2.0, 0.5]
    E = np.stack([col, np.zeros(m), col], axis=1)   # second empty, third duplicate
    Ec = synth.csr_from_coo(*np.nonzero(E.T), E.T[np.nonzero(E.T)], 3, m)
    st = svlcov.State.init(U, s, V)
    st.add_cols(Ec.indptr, Ec.indices, Ec.values, 3)
    assert st.log[-1]["dropped"] == [1, 2]
    Ud, sd, Vd = dense.define_add_cols(U, s, V, E.T)
    Us, ss, Vs = st.factors()
    assert checks.sigma_rel_err(ss, sd) < 1e-12
    assert checks.projector_err(Us, Ud) < 1e-10


# ---------------------------------------------------------------------------
# Planted mistakes: each variant breaks one step in a plausible way; the pins
# above must reject it.
class _KUsesRescaledC(svlcov.State):
    def add_cols(self, indptr, indices, values, s):
        k = self.k
        bt = svlcov.Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Up, self.Wu, bt)
        B, C, R, _ = svlcov.svlcov_qr(bt.B0, C0, self.tau)
        K = np.zeros((k + s, k + s)); K[:k, :k] = np.diag(self.sigma); K[:k, k:] = C; K[k:, k:] = R
        F, th, G = dense.svd_k(K, k)
        self.Wu = self.Wu @ (F[:k] - C @ F[k:])
        self.Up[bt.support] += svlcov._xinv(B @ F[k:], self.Wu)
        self.sigma = th; self.Wv = self.Wv @ G[:k]
        self.Vp = np.vstack([self.Vp, svlcov._xinv(G[k:], self.Wv)])


class _OldInverse(svlcov.State):
    def add_cols(self, indptr, indices, values, s):
        k = self.k
        bt = svlcov.Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Up, self.Wu, bt)
        B, C, R, _ = svlcov.svlcov_qr(bt.B0, C0, self.tau)
        K = np.zeros((k + s, k + s)); K[:k, :k] = np.diag(self.sigma); K[:k, k:] = C0; K[k:, k:] = R
        F, th, G = dense.svd_k(K, k)
        old = self.Wu
        self.Wu = self.Wu @ (F[:k] - C @ F[k:])
        self.Up[bt.support] += svlcov._xinv(B @ F[k:], old)
        self.sigma = th; self.Wv = self.Wv @ G[:k]
        self.Vp = np.vstack([self.Vp, svlcov._xinv(G[k:], self.Wv)])


class _NoCorrectionTerm(svlcov.State):
    def add_cols(self, indptr, indices, values, s):
        k = self.k
        bt = svlcov.Batch.from_csr(indptr, indices, values, s)
        C0 = self._project(self.Up, self.Wu, bt)
        B, C, R, _ = svlcov.svlcov_qr(bt.B0, C0, self.tau)
        K = np.zeros((k + s, k + s)); K[:k, :k] = np.diag(self.sigma); K[:k, k:] = C0; K[k:, k:] = R
        F, th, G = dense.svd_k(K, k)
        self.Wu = self.Wu @ F[:k]
        self.Up[bt.support] += svlcov._xinv(B @ F[k:], self.Wu)
        self.sigma = th; self.Wv = self.Wv @ G[:k]
        self.Vp = np.vstack([self.Vp, svlcov._xinv(G[k:], self.Wv)])


def _wrong_sign_qr(B0, C0, tau=1e-12):
    B = B0.copy(); C = C0.copy(); s = B.shape[1]; R = np.zeros((s, s))
    for i in range(s):
        a = np.sqrt(B[:, i] @ B[:, i] + C[:, i] @ C[:, i])
        R[i, i] = a; B[:, i] /= a; C[:, i] /= a
        beta = B[:, i] @ B[:, i + 1:] + C[:, i] @ C[:, i + 1:]
        R[i, i + 1:] = beta
        B[:, i + 1:] -= np.outer(B[:, i], beta); C[:, i + 1:] -= np.outer(C[:, i], beta)
    return B, C, R, []


@pytest.mark.parametrize("variant", ["K_uses_rescaled_C", "old_inverse", "no_correction_term",
                                     "inner_product_sign"])
def test_planted_mistakes_are_caught(variant, monkeypatch):
    g = synth.rng(41)
    m, n, k, s = 40, 30, 4, 3
    A = sp.random(m, n, density=0.3, random_state=3, data_rvs=lambda x: g.standard_normal(x)).toarray()
    U, sg, V = synth.init_factors(A, k, 0)
    Ec = synth.random_csr_batch(s, m, 5, g)
    cls = {"K_uses_rescaled_C": _KUsesRescaledC, "old_inverse": _OldInverse,
           "no_correction_term": _NoCorrectionTerm, "inner_product_sign": svlcov.State}[variant]
    if variant == "inner_product_sign":
        monkeypatch.setattr(svlcov, "svlcov_qr", _wrong_sign_qr)
    st = cls.init(U, sg, V) if cls is svlcov.State else cls(*svlcov.State.init(U, sg, V).__dict__.values())
    st.add_cols(Ec.indptr, Ec.indices, Ec.values, s)
    Us, ss, Vs = st.factors()
    Ud, sd, Vd = dense.define_add_cols(U, sg, V, Ec.dense())
    err = max(checks.sigma_rel_err(ss, sd), checks.projector_err(Us, Ud), checks.projector_err(Vs, Vd),
              checks.orth_err(Us), checks.orth_err(Vs))
    assert err > 1e-6, (variant, err)


# ---------------------------------------------------------------------------
def nonempty_columns(b):
    """The batch without its empty update vectors (the gradient of a
    deflated direction does not exist; the differentiation workload uses
    batches with none, reading R14)."""
    keep = [j for j in range(b.rows) if b.indptr[j + 1] > b.indptr[j]]
    r, c, v = [], [], []
    for jj, j in enumerate(keep):
        a, e = b.indptr[j], b.indptr[j + 1]
        r.extend([jj] * (e - a)); c.extend(b.indices[a:e].tolist()); v.extend(b.values[a:e].tolist())
    return synth.csr_from_coo(np.array(r, dtype=np.int64), np.array(c, dtype=np.int64), np.array(v), len(keep), b.cols)


def _c5_small(seed=51, N=1200, k=8, s=12):
    p = synth.c2_problem(seed=seed, N=N, k=k, s=s, n_batches=2, power_iters=2)
    kind, b = p["batches"][1]          # a column step
    assert kind == "cols"
    b = nonempty_columns(b)
    st = svlcov.State.init(p["U"], p["sigma"], p["V"])
    st.apply(*p["batches"][0])         # the row step before it
    U, sg, V = st.factors()
    g = synth.rng(seed)
    S_rows = np.sort(g.choice(U.shape[0], size=200, replace=False))
    return U, sg, V, b, S_rows


def test_gradient_autograd_matches_finite_differences():
    """The reference gradient of the C5 loss (torch float64 autograd on the
    dense Zha-Simon step) equals central finite differences of the sparse
    oracle's loss (h = 1e-3) on random nonzeros, to 1e-5 normwise."""
    from oracle import backward
    U, sg, V, b, S_rows = _c5_small()
    ga = backward.grad_autograd(U, sg, b.indptr, b.indices, b.values, b.rows, S_rows)
    g = synth.rng(3)
    which = g.choice(b.nnz, size=min(16, b.nnz), replace=False)
    gf = backward.grad_fd(U, sg, V, b.indptr, b.indices, b.values, b.rows, S_rows, which)
    assert np.linalg.norm(ga[which] - gf) <= 1e-5 * np.linalg.norm(gf)
    assert np.linalg.norm(gf) > 0

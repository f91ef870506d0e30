"""GPU parity: the CUDA path (called through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (singular values relative, subspaces as the sine of the largest
principal angle on the gapped leading block):
  FP64 storage, FP64 small steps : 1e-10 / 1e-8  (rounding of the FP64 path)
  FP32 storage                   : 1e-5  / 1e-4
  BF16 storage                   : 1e-3  / 1e-2
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import checks, dense, svlcov as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import compare, dev_batch, make_gpu, run_gpu, run_oracle, to_dev  # noqa: E402


def _mixed_problem(seed, m=60, n=45, k=6, steps=12, s_max=7, per_vec=4):
    g = synth.rng(seed)
    A = sp.random(m, n, density=0.2, random_state=seed, data_rvs=lambda x: g.standard_normal(x)).toarray()
    U, s, V = synth.init_factors(A, k, seed)
    ops, mm, nn = [], m, n
    for t in range(steps):
        kind = ("cols", "rows", "weights")[t % 3]
        ss = int(g.integers(1, s_max + 1))
        if kind == "cols":
            b = synth.random_csr_batch(ss, mm, per_vec, g); nn += ss
        elif kind == "rows":
            b = synth.random_csr_batch(ss, nn, per_vec, g); mm += ss
        else:
            b = (synth.random_csr_batch(ss, mm, per_vec, g), synth.random_csr_batch(ss, nn, per_vec, g))
        ops.append((kind, b))
    return U, s, V, ops


@pytest.mark.parametrize("n,k", [(8, 3), (26, 16), (70, 10), (129, 32), (320, 64)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("mixed", 1e-10)])
def test_small_svd_matches_lapack(n, k, precision, tol):
    from paper_2401_09703_gb300 import small_svd
    g = synth.rng(n * 7 + k)
    K = np.triu(g.standard_normal((n, n)))
    K[:k, :k] = np.diag(np.sort(np.abs(g.standard_normal(k)))[::-1] * 5)
    Kt = torch.as_tensor(K, device="cuda")
    F, th, G, sweeps = small_svd(Kt, k, precision)
    F, th, G = F.cpu().numpy(), th.cpu().numpy(), G.cpu().numpy()
    Fo, tho, Go = dense.svd_k(K, k)
    assert checks.sigma_rel_err(th, tho) < tol
    kp = checks.gapped_prefix(tho, 1e-3)
    if precision == "fp32":
        # Wedin's sin-theta bound: a backward error of c sqrt(n) eps32 ||K|| (K rounded to FP32,
        # rotations in FP32, sweeps stopped at 4 sqrt(n) eps32 off-diagonality) moves the leading
        # k' singular subspaces by at most that over the gap to the next value of the full
        # spectrum; c = 20
        full = np.linalg.svd(K, compute_uv=False)
        vtol = 20 * np.sqrt(n) * 2.0 ** -24 / ((full[kp - 1] - full[kp]) / full[0])
    else:
        vtol = 100 * tol
    assert checks.max_sin_angle(F[:, :kp], Fo[:, :kp]) < vtol
    assert checks.max_sin_angle(G[:, :kp], Go[:, :kp]) < vtol
    assert np.max(np.abs(K @ G - F * th)) < 10 * tol * th[0]
    assert 0 < sweeps < 40


def test_mixed_svd_close_pair_streaming_k():
    """The Rayleigh-Ritz matrix of update 222 of the streaming node insertion
    (C2 graph, s = 1), built by the oracle: its leading values include a pair
    5e-4 apart (relative).  The mixed SVD (FP32 sweeps with the early stop,
    three FP64 first-order steps) must reach FP64 accuracy on it; with a stop
    of 1e-2 instead of 1e-3 the steps could not remove the coupling the sweeps
    left between that pair (one value off by 1e-4)."""
    from paper_2401_09703_gb300 import small_svd
    p = synth.c2_problem(s=1, n_batches=112)
    st = osv.State.init(p["U"], p["sigma"], p["V"])
    for kind, b in p["batches"][:223]:
        st.apply(kind, b)
    # a rows step: the oracle logs K in the orientation of A, the GPU factors
    # that of A^T (Algorithm 11 as Algorithm 3 on A^T), i.e. the transpose
    K = np.ascontiguousarray(st.log[-1]["K"].T)
    k = 64
    Fo, tho, Go = dense.svd_k(K, k)
    gaps = (tho[:-1] - tho[1:]) / tho[0]
    assert gaps.min() < 1e-3            # the close pair is there
    F, th, G, sweeps = small_svd(torch.as_tensor(K, device="cuda"), k, "mixed")
    F, th, G = F.cpu().numpy(), th.cpu().numpy(), G.cpu().numpy()
    assert checks.sigma_rel_err(th, tho) < 1e-12
    assert np.max(np.abs(G.T @ G - np.eye(k))) < 1e-10
    kp = checks.gapped_prefix(tho, 1e-6)
    assert checks.max_sin_angle(G[:, :kp], Go[:, :kp]) < 1e-8


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mixed_trajectory_fp64(seed):
    """Add columns, add rows and weight updates in FP64: GPU = oracle."""
    U, s, V, ops = _mixed_problem(seed)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp64", small="fp64")
    assert code == 0
    st = run_oracle(U, s, V, ops)
    c = compare(Ug, sg, Vg, st)
    assert c["sigma"] < 1e-10, c
    assert c["sin_u"] < 1e-8 and c["sin_v"] < 1e-8, c
    assert checks.orth_err(Ug) < 1e-10 and checks.orth_err(Vg) < 1e-10


def test_c1_fp64_full_trajectory_and_intermediates():
    """C1: 2000 x 1000 binary, k = 16, ten batches of ten new columns, FP64.
    Every step's intermediates match the oracle: P and S_E exactly (integer
    data), R to rounding, Theta to 1e-12; final factors to 1e-10."""
    p = synth.c1_problem()
    U, s, V, ops = p["U"], p["sigma"], p["V"], p["batches"]
    g = make_gpu(U, s, V, ops, storage="fp64", small="fp64")
    st = osv.State.init(U, s, V)
    for t, (kind, b) in enumerate(ops):
        Xp = st.Up.copy()
        g.apply(kind, dev_batch(kind, b))
        st.apply(kind, b)
        log = st.log[-1]
        bt = osv.Batch.from_csr(b.indptr, b.indices, b.values, b.rows)
        if t == 0:   # afterwards U' is only defined up to the small factor
            P_ref = Xp[bt.support].T @ bt.B0
            assert np.max(np.abs(g.intermediate(0) - P_ref)) <= 1e-12 * max(1.0, np.abs(P_ref).max())
        SE_ref = bt.B0.T @ bt.B0
        assert np.array_equal(g.intermediate(1), SE_ref)
        # C0 = U^T E: rows follow the singular vectors, whose signs are free
        C0g, C0o = g.intermediate(2), log["C0"]
        sgn = np.sign(np.sum(C0g * C0o, axis=1, keepdims=True))
        sgn[sgn == 0] = 1.0
        assert np.max(np.abs(C0g * sgn - C0o)) < 1e-11
        assert np.max(np.abs(g.intermediate(3) - log["R"])) < 1e-10 * max(1.0, np.abs(log["R"]).max())
        assert np.max(np.abs(g.intermediate(5).ravel() - log["theta"])) < 1e-12 * log["theta"][0]
    assert g.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    c = compare(Ug, sg, Vg, st)
    assert c["sigma"] < 1e-10 and c["sin_u"] < 1e-8 and c["sin_v"] < 1e-8, c


def _small_c2(N=3000, k=16, s=64, n_batches=6, seed=1002):
    p = synth.c2_problem(seed=seed, N=N, k=k, s=s, n_batches=n_batches, power_iters=2)
    return p["U"], p["sigma"], p["V"], p["batches"]


@pytest.mark.parametrize("small", ["fp64", "mixed", "fp32"])
def test_c2_like_fp32_storage(small):
    """Graph node insertion (Chung-Lu, rows then columns), FP32 factors."""
    U, s, V, ops = _small_c2()
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp32", small=small, values_dtype=torch.float32,
                                  init_dtype=torch.float32)
    assert code == 0
    st = run_oracle(U, s, V, ops)
    c = compare(Ug, sg, Vg, st)
    tol = 1e-5 if small != "fp32" else 1e-4
    assert c["sigma"] < tol, c
    assert c["sin_u"] < 10 * tol and c["sin_v"] < 10 * tol, c


def test_c2_like_bf16_storage():
    U, s, V, ops = _small_c2(n_batches=4)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="bf16", small="mixed", values_dtype=torch.float32,
                                  init_dtype=torch.float32)
    assert code == 0
    st = run_oracle(U, s, V, ops)
    c = compare(Ug, sg, Vg, st)
    assert c["sigma"] < 1e-3, c
    assert c["sin_u"] < 1e-2 and c["sin_v"] < 1e-2, c


def _small_c3(n_users=20000, n_items=5000, k=32, s=512, n_batches=2):
    p = synth.c3_problem(n_users=n_users, n_items=n_items, k=k, s=s, n_batches=n_batches, power_iters=2)
    return p["U"], p["sigma"], p["V"], p["batches"]


@pytest.mark.parametrize("storage,small,tol,literal", [("fp64", "fp64", 1e-10, 0), ("fp64", "mixed", 1e-7, 1),
                                                       ("fp64", "mixed", 1e-7, 0), ("fp32", "mixed", 1e-5, 0),
                                                       ("bf16", "mixed", 1e-3, 0)])
def test_c3_like_wide_batches(storage, small, tol, literal):
    """Rating matrix (Zipf item popularity), users appended in batches of
    s = 512: wider than the one-CTA shared-memory Cholesky in FP64 and in the
    FP32 first pass, so the blocked factorization runs.  R of the first step
    equals the oracle's (it is unique: positive diagonal); a mixed step on the
    default R-free route forms no R and says so."""
    from paper_2401_09703_gb300 import SvlcovError
    U, s, V, ops = _small_c3()
    vdt = torch.float64 if storage == "fp64" else torch.float32
    idt = torch.float64 if storage == "fp64" else torch.float32
    g = make_gpu(U, s, V, ops, storage=storage, small=small, init_dtype=idt, literal_steps=literal)
    st = osv.State.init(U, s, V)
    for t, (kind, b) in enumerate(ops):
        g.apply(kind, dev_batch(kind, b, vdt))
        st.apply(kind, b)
        if t == 0 and storage == "fp64":
            if small == "mixed" and not literal:
                for which in (3, 4, 6):   # R, K, F
                    with pytest.raises(SvlcovError):
                        g.intermediate(which)
                continue
            Rg, Ro = g.intermediate(3), st.log[-1]["R"]
            rtol = 1e-10 if small == "fp64" else 1e-7
            assert np.max(np.abs(Rg - Ro)) < rtol * np.abs(Ro).max()
    assert g.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    c = compare(Ug, sg, Vg, st)
    assert c["sigma"] < tol, c
    stol = 1e-8 if tol < 1e-9 else 10 * tol
    assert c["sin_u"] < stol and c["sin_v"] < stol, c


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_rfree_and_literal_mixed_steps_agree(storage):
    """The mixed step without R (folds from Sigma, G and Theta; SVD_k refined
    on K^T K = [[Sigma^2, Sigma C0], [C0^T Sigma, E^T E]]) and the literal
    Algorithm 2 / 3 / 11 step reach the same factors: both against the oracle
    over a node-insertion trajectory (rows and columns steps, k = 16, s = 64),
    and against each other."""
    U, s, V, ops = _small_c2()
    vdt = torch.float64 if storage == "fp64" else torch.float32
    idt = torch.float64 if storage == "fp64" else torch.float32
    st = osv.State.init(U, s, V)
    for kind, b in ops:
        st.apply(kind, b)
    out = []
    for literal in (0, 1):
        g = make_gpu(U, s, V, ops, storage=storage, small="mixed", init_dtype=idt, literal_steps=literal)
        for kind, b in ops:
            g.apply(kind, dev_batch(kind, b, vdt))
        assert g.status() == 0
        out.append([x.cpu().numpy().astype(np.float64) for x in g.get_factors()])
        c = compare(*out[-1], st)
        tol = 1e-9 if storage == "fp64" else 1e-5
        assert c["sigma"] < tol, (literal, c)
        assert c["sin_u"] < 100 * tol and c["sin_v"] < 100 * tol, (literal, c)
    (Ua, sa, Va), (Ub, sb, Vb) = out
    assert np.max(np.abs(sa - sb)) / sa[0] < (1e-9 if storage == "fp64" else 1e-5)


def test_reorthonormalisation_keeps_fp64_parity():
    """Forcing the re-orthonormalisation of the projected factor before every
    step on FP64 storage changes nothing beyond rounding: U'W is orthonormal
    to FP64 accuracy there, so the correction is ~eps."""
    U, s, V, ops = _mixed_problem(4)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp64", small="fp64", reorth=1)
    assert code == 0
    c = compare(Ug, sg, Vg, run_oracle(U, s, V, ops))
    assert c["sigma"] < 1e-10 and c["sin_u"] < 1e-8 and c["sin_v"] < 1e-8, c
    assert checks.orth_err(Ug) < 1e-10 and checks.orth_err(Vg) < 1e-10


def test_bf16_reorthonormalisation_reduces_drift():
    """BF16 factors drift from orthonormal with every rounding; the default
    re-orthonormalisation (every step) keeps Sigma closer to the oracle than
    no correction, and within the BF16 target."""
    U, s, V, ops = _small_c3(n_batches=4)
    st = run_oracle(U, s, V, ops)
    errs = {}
    for ro in (-1, 0):
        g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="bf16", small="mixed", values_dtype=torch.float32,
                                      init_dtype=torch.float32, reorth=ro)
        assert code == 0
        errs[ro] = compare(Ug, sg, Vg, st)["sigma"]
    assert errs[0] < errs[-1] and errs[0] < 1e-3, errs


def test_maximum_rank_and_batch_width():
    """k = 128 and s = 1024 (the largest the library takes; K is 1152^2):
    one add-rows step of a rating matrix, mixed small steps, FP32 factors."""
    U, s, V, ops = _small_c3(n_users=40000, n_items=10000, k=128, s=1024, n_batches=1)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp32", small="mixed", values_dtype=torch.float32,
                                  init_dtype=torch.float32)
    assert code == 0
    st = run_oracle(U, s, V, ops)
    c = compare(Ug, sg, Vg, st)
    assert c["sigma"] < 1e-5, c
    assert c["sin_u"] < 1e-4 and c["sin_v"] < 1e-4, c


def test_query_rows_and_determinism():
    U, s, V, ops = _mixed_problem(5)
    g1, c1, U1, s1, V1 = run_gpu(U, s, V, ops)
    g2, c2, U2, s2, V2 = run_gpu(U, s, V, ops)
    assert np.array_equal(U1, U2) and np.array_equal(s1, s2) and np.array_equal(V1, V2)
    idx = torch.tensor([0, 3, U1.shape[0] - 1], dtype=torch.int32)
    q = g1.query_rows(0, idx).cpu().numpy()
    assert np.array_equal(q, U1[idx.numpy()])
    qv = g1.query_rows(1, torch.tensor([1, V1.shape[0] - 1], dtype=torch.int32)).cpu().numpy()
    assert np.array_equal(qv, V1[[1, V1.shape[0] - 1]])


def test_checkpoint_resume_is_bit_exact():
    U, s, V, ops = _mixed_problem(6)
    g, code, Ua, sa, Va = run_gpu(U, s, V, ops)
    h = make_gpu(U, s, V, ops)
    half = len(ops) // 2
    for kind, b in ops[:half]:
        h.apply(kind, dev_batch(kind, b))
    state = h.get_state()
    h2 = make_gpu(U, s, V, ops)
    h2.set_state(state)
    for kind, b in ops[half:]:
        h2.apply(kind, dev_batch(kind, b))
    Ub, sb, Vb = (x.cpu().numpy() for x in h2.get_factors())
    assert np.array_equal(Ua, Ub) and np.array_equal(sa, sb) and np.array_equal(Va, Vb)


def test_empty_rows_and_empty_batch_deflate():
    """Update vectors with no nonzeros (and a batch with nnz = 0) are dropped
    by the deflation rule and the result equals the definition."""
    g0 = synth.rng(9)
    m, n, k = 50, 40, 5
    A = g0.standard_normal((m, n))
    U, s, V = synth.init_factors(A, k, 0)
    E = np.zeros((4, m)); E[1, [2, 5]] = [1.0, 2.0]; E[3, [7]] = [3.0]
    b = synth.csr_from_coo(*np.nonzero(E), E[np.nonzero(E)], 4, m)
    empty = synth.CSR(np.zeros(3, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), 2, m + 0)
    ops = [("cols", b)]
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops)
    assert code == 0
    Ud, sd, Vd = dense.define_add_cols(U, s, V, E)
    assert checks.sigma_rel_err(sg, sd) < 1e-10
    g2 = make_gpu(U, s, V, [("rows", synth.CSR(np.zeros(3, dtype=np.int32), np.zeros(0, dtype=np.int32),
                                               np.zeros(0), 2, n))])
    g2.add_rows(to_dev(synth.CSR(np.zeros(3, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0), 2, n)))
    assert g2.status() == 0
    U2, s2, V2 = (x.cpu().numpy() for x in g2.get_factors())
    Ud, sd, Vd = dense.define_add_rows(U, s, V, np.zeros((2, n)))
    assert checks.sigma_rel_err(s2, sd) < 1e-12 and U2.shape[0] == m + 2


@pytest.mark.parametrize("bad", ["duplicate", "out_of_range", "nan", "indptr"])
def test_bad_batches_flag_status_and_leave_state_unchanged(bad):
    from paper_2401_09703_gb300 import _abi
    U, s, V, ops = _mixed_problem(4, steps=3)
    g = make_gpu(U, s, V, ops)
    U0, s0, V0 = (x.cpu().numpy() for x in g.get_factors())
    m = U.shape[0]
    indptr = np.array([0, 2, 4], dtype=np.int32)
    indices = np.array([1, 5, 7, 9], dtype=np.int32)
    values = np.array([1.0, 2.0, 3.0, 4.0])
    if bad == "duplicate":
        indices[1] = 1
    elif bad == "out_of_range":
        indices[2] = m + 3
    elif bad == "nan":
        values[3] = np.nan
    else:
        indptr = np.array([0, 3, 2], dtype=np.int32)
        indptr[2] = 4; indptr[1] = 5
    b = synth.CSR(indptr, indices, values, 2, m)
    g.add_cols(to_dev(b))
    code = g.status()
    expect = _abi.SVLCOV_DEV_NONFINITE if bad == "nan" else _abi.SVLCOV_DEV_BAD_CSR
    assert code & expect
    U1, s1, V1 = (x.cpu().numpy() for x in g.get_factors())
    assert g.shape()[1] == V.shape[0]
    assert np.array_equal(U0, U1) and np.array_equal(s0, s1) and np.array_equal(V0, V1[: V0.shape[0]])


def test_capacity_is_a_host_error():
    from paper_2401_09703_gb300 import SvlcovError, _abi
    U, s, V, ops = _mixed_problem(7, steps=1)
    g = make_gpu(U, s, V, ops)
    big = synth.random_csr_batch(g._desc.max_s + 1, U.shape[0], 2, synth.rng(1))
    with pytest.raises(SvlcovError) as ei:
        g.add_cols(to_dev(big))
    assert ei.value.code == _abi.SVLCOV_ERR_CAPACITY

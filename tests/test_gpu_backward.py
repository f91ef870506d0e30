"""GPU backward of one add-columns step (svlcov_add_cols_backward) against
the FP64 oracle gradient.

The loss is L = sum_{r in S} sum_i U_new[r, i]^2 theta_i (the squared norms
of the updated embeddings U Theta^(1/2) over a row set S), differentiated
with respect to the stored values of the batch.  The reference gradient is
torch float64 autograd of the dense Zha-Simon step (oracle.backward), itself
pinned to finite differences of the sparse oracle on the CPU; here the GPU
gradient is also checked against central differences (h = 1e-3) of the
sparse oracle's loss on sampled nonzeros.

Tolerances (normwise relative):
  FP64 storage, FP64 small steps : 1e-8  (rounding of the FP64 path, amplified
                                          by 1 / min gap of the spectrum of K)
  FP64 storage, mixed small steps: 1e-5  (the mixed SVD refines vectors from
                                          FP32 sweeps; for pairs ~1e-4 theta_1
                                          apart its individual vectors keep
                                          ~1e-10 errors, which the pair terms
                                          amplify by 1 / gap; measured 3e-8 to
                                          5e-7 depending on the sweep order)
  FP32 storage, mixed small steps: 1e-4  (U' rounded to FP32 perturbs U by
                                          ~1e-7; the adjoint amplifies it by the
                                          same gap factor)
  against finite differences     : 1e-5 + the path's own tolerance (the
                                          O(h^2) truncation of the difference)
The start state of every case is the oracle's, so both sides differentiate
the same step.
"""
import numpy as np
import pytest

import synth
from oracle import backward, svlcov as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import to_dev  # noqa: E402

GAP_WARN = 0x80


def _case(N, k, s, n_loss, seed=1002):
    p = synth.c5_problem(seed=seed, N=N, k=k, s=s, n_loss=n_loss, power_iters=2 if N < 20000 else 4)
    st = osv.State.init(p["U"], p["sigma"], p["V"])
    st.apply("rows", p["rows"])
    U, sg, V = st.factors()
    return U, sg, V, p["cols"], p["S_rows"]


def _gpu_model(U, sg, V, b, storage, small):
    from paper_2401_09703_gb300 import SVLCOV
    dev = torch.device("cuda")
    return SVLCOV(torch.as_tensor(U, device=dev), torch.as_tensor(sg, device=dev), torch.as_tensor(V, device=dev),
                  max_m=U.shape[0] + 8, max_n=V.shape[0] + b.rows + 8, max_s=b.rows, max_nnz=b.nnz,
                  storage=storage, small=small, literal_steps=1)


def _gpu_grad(U, sg, V, b, S_rows, storage, small, gap=1e-6):
    """The GPU gradient through the autograd Function, and the status word."""
    from paper_2401_09703_gb300 import add_cols_with_grad
    g = _gpu_model(U, sg, V, b, storage, small)
    batch = to_dev(b, torch.float64)
    batch.values.requires_grad_(True)
    U_S, th = add_cols_with_grad(g, batch, torch.as_tensor(S_rows), gap=gap)
    L = (U_S * U_S * th).sum()
    (gv,) = torch.autograd.grad(L, batch.values)
    code = g.status()
    return gv.cpu().numpy(), float(L.detach()), code, g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,k,s,n_loss", [(1200, 8, 12, 200), (6000, 16, 64, 1000), (20000, 32, 128, 2048)])
@pytest.mark.parametrize("storage,small,tol", [("fp64", "fp64", 1e-8), ("fp64", "mixed", 1e-5),
                                               ("fp32", "mixed", 1e-4)])
def test_backward_matches_oracle_gradient(N, k, s, n_loss, storage, small, tol):
    U, sg, V, b, S_rows = _case(N, k, s, n_loss)
    ga = backward.grad_autograd(U, sg, b.indptr, b.indices, b.values, b.rows, S_rows)
    gv, L, code, _ = _gpu_grad(U, sg, V, b, S_rows, storage, small)
    assert code == 0, code
    Lo = backward.loss_oracle(U, sg, V, b.indptr, b.indices, b.values, b.rows, S_rows)
    assert abs(L - Lo) <= tol * abs(Lo)
    assert _rel(gv, ga) <= tol, _rel(gv, ga)


@pytest.mark.slow
def test_backward_c5_full_size():
    """C5: C2's first column step (k = 64, N = 1e5, the distinct non-empty
    update vectors of s = 256), loss over 4096 existing nodes, FP32 storage
    with mixed small steps and FP64 storage with FP64 small steps; the FP32
    gradient against the oracle's autograd gradient and against finite
    differences on 64 sampled nonzeros (h = 1e-3)."""
    U, sg, V, b, S_rows = _case(100_000, 64, 256, 4096)
    ga = backward.grad_autograd(U, sg, b.indptr, b.indices, b.values, b.rows, S_rows)
    g32, _, code32, _ = _gpu_grad(U, sg, V, b, S_rows, "fp32", "mixed")
    g64, _, code64, _ = _gpu_grad(U, sg, V, b, S_rows, "fp64", "fp64")
    assert code32 == 0 and code64 == 0, (code32, code64)
    assert _rel(g64, ga) <= 1e-8, _rel(g64, ga)
    assert _rel(g32, ga) <= 1e-4, _rel(g32, ga)
    which = synth.rng(7).choice(b.nnz, size=min(64, b.nnz), replace=False)
    gf = backward.grad_fd(U, sg, V, b.indptr, b.indices, b.values, b.rows, S_rows, which)
    assert _rel(g32[which], gf) <= 1e-4 + 1e-5, _rel(g32[which], gf)
    assert _rel(g64[which], gf) <= 1e-5, _rel(g64[which], gf)


def test_backward_matches_finite_differences_small():
    U, sg, V, b, S_rows = _case(6000, 16, 64, 1000)
    gv, _, code, _ = _gpu_grad(U, sg, V, b, S_rows, "fp64", "fp64")
    assert code == 0
    which = synth.rng(11).choice(b.nnz, size=min(24, b.nnz), replace=False)
    gf = backward.grad_fd(U, sg, V, b.indptr, b.indices, b.values, b.rows, S_rows, which)
    assert _rel(gv[which], gf) <= 1e-5, _rel(gv[which], gf)


def test_backward_theta_only_and_empty_row_set():
    """dL/dtheta alone (no rows in S): L = sum of the k kept singular values,
    against torch autograd of the same loss on the dense step."""
    U, sg, V, b, _ = _case(1200, 8, 12, 10)
    from paper_2401_09703_gb300 import add_cols_with_grad
    g = _gpu_model(U, sg, V, b, "fp64", "fp64")
    batch = to_dev(b, torch.float64)
    batch.values.requires_grad_(True)
    _, th = add_cols_with_grad(g, batch, torch.zeros(0, dtype=torch.int32))
    (gv,) = torch.autograd.grad(th.sum(), batch.values)
    assert g.status() == 0
    v = torch.tensor(b.values, dtype=torch.float64, requires_grad=True)
    # the oracle's dense step: sum of the kept singular values of K
    Ut, s_t = torch.as_tensor(U), torch.as_tensor(sg)
    E = backward._dense_E(b.indptr, b.indices, v, b.rows, U.shape[0])
    C = Ut.T @ E
    Q, R = torch.linalg.qr(E - Ut @ C)
    k = len(sg)
    K = torch.cat([torch.cat([torch.diag(s_t), C], 1), torch.cat([torch.zeros(b.rows, k, dtype=torch.float64), R], 1)])
    (go,) = torch.autograd.grad(torch.linalg.svdvals(K)[:k].sum(), v)
    assert _rel(gv.cpu().numpy(), go.numpy()) <= 1e-9


def test_backward_gap_guard_reports_warning():
    """A gap threshold above every singular-value gap guards every pair: the
    status word carries SVLCOV_DEV_GAP_WARN after the backward (and the
    gradient keeps only the dL/dtheta and direct terms)."""
    U, sg, V, b, S_rows = _case(1200, 8, 12, 200)
    _, _, code, _ = _gpu_grad(U, sg, V, b, S_rows, "fp64", "fp64", gap=2.0)
    assert code & GAP_WARN


def test_backward_host_errors():
    from paper_2401_09703_gb300 import SvlcovError
    U, sg, V, b, S_rows = _case(1200, 8, 12, 50)
    S = torch.as_tensor(S_rows, dtype=torch.int32, device="cuda")
    z = torch.zeros((len(S_rows), len(sg)), dtype=torch.float64, device="cuda")
    zn = torch.zeros((b.nnz, len(sg)), dtype=torch.float64, device="cuda")
    # no step yet
    g = _gpu_model(U, sg, V, b, "fp64", "fp64")
    batch = to_dev(b)
    with pytest.raises(SvlcovError):
        g.add_cols_backward(batch, S, z, zn, z, None)
    # FP32 small steps keep no FP64 intermediates
    g32 = _gpu_model(U, sg, V, b, "fp64", "fp32")
    g32.add_cols(batch)
    with pytest.raises(SvlcovError):
        g32.add_cols_backward(batch, S, z, zn, z, None)
    # a step in between
    g.add_cols(batch)
    rb = synth.random_csr_batch(3, g.shape()[1], 2, synth.rng(1))
    g.add_rows(to_dev(rb))
    with pytest.raises(SvlcovError):
        g.add_cols_backward(batch, S, z, zn, z, None)
    assert g.status() == 0

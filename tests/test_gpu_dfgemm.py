"""The FP64 products in double-float arithmetic on the FP32 pipe
(svlcov_dgemm, engine 2), the refinement products of steps whose factors
are stored in FP32 / BF16, against numpy's FP64 product through the C ABI.

Bound: an operand x splits as hi + lo with hi its top 24 significant bits,
so |lo| < 2^-23 |x| and lo carries x - hi to 2^-24 of itself; the hi
products are exact, the dropped lo lo term and the rounding of the cross
terms stay within 2^-45 |a b| per term, and the FP32 sum of the error parts
adds at most K 2^-47 of sum_k |a_ik b_kj| -- so |C_df - AB| <=
4 (K + 4) 2^-46 (|A| |B|)_ij, beside the FP64 rounding of the reference."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _bound(a, b):
    K = a.shape[1]
    ab = np.abs(a) @ np.abs(b)
    return 4 * (K + 4) * 2.0 ** -46 * ab + 2 * K * EPS * ab


SHAPES = [(1, 1, 1), (7, 5, 3), (64, 64, 64), (320, 72, 320), (256, 256, 64), (200, 130, 1100),
          (129, 65, 1152), (1152, 128, 64), (33, 300, 17), (72, 72, 320)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_df_dgemm_matches_fp64(M, N, K, ta, tb):
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(M * 137 + N * 11 + K + 5 * ta + 2 * tb)
    A = g.standard_normal((K, M) if ta else (M, K)) * np.exp(g.uniform(-3, 3, size=(K, M) if ta else (M, K)))
    B = g.standard_normal((N, K) if tb else (K, N))
    a = A.T if ta else A
    b = B.T if tb else B
    C = a @ b
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), ta=ta, tb=tb,
                engine="df32").cpu().numpy()
    bnd = _bound(a, b)
    assert np.all(np.abs(out - C) <= bnd), float(np.max(np.abs(out - C) / bnd))
    # and far beyond FP32: a plain FP32 product misses the bound
    if K >= 64:
        c32 = (a.astype(np.float32) @ b.astype(np.float32)).astype(np.float64)
        assert np.max(np.abs(c32 - C) / bnd) > 100.0


def test_df_dgemm_alpha_beta_and_cancellation():
    """alpha op(A) op(B) + beta C, and a Gram difference that cancels to
    ~1e-6 of its terms (the residual Gram of a batch nearly in the span of
    the factors) keeps its small entries to the bound."""
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(21)
    A = g.standard_normal((150, 300))
    B = g.standard_normal((300, 90))
    C0 = g.standard_normal((150, 90))
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), alpha=2.0, beta=-3.0,
                C=torch.as_tensor(C0, device="cuda"), engine="df32").cpu().numpy()
    ref = 2.0 * (A @ B) - 3.0 * C0
    assert np.all(np.abs(out - ref) <= 2.0 * _bound(A, B) + 4 * EPS * np.abs(3.0 * C0))
    # E^T E - C0^T C0 with E = U C0 + 1e-3 noise: the difference is ~1e-6 of the Gram
    U, _ = np.linalg.qr(g.standard_normal((400, 64)))
    Cq = g.standard_normal((64, 48))
    E = U @ Cq + 1e-3 * g.standard_normal((400, 48))
    SE = E.T @ E
    S = dgemm(torch.as_tensor(Cq, device="cuda"), torch.as_tensor(Cq, device="cuda"), ta=True, alpha=-1.0, beta=1.0,
              C=torch.as_tensor(SE, device="cuda"), engine="df32").cpu().numpy()
    ref = SE - Cq.T @ Cq
    assert np.all(np.abs(S - ref) <= _bound(Cq.T, Cq) + 4 * EPS * np.abs(SE))
    assert np.max(np.abs(S - ref)) < 1e-6 * np.max(np.abs(ref))


def test_df_dgemm_zero_k_and_exact_small_integers():
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(22)
    A = g.integers(-1000, 1001, size=(40, 70)).astype(np.float64)
    B = g.integers(-1000, 1001, size=(70, 30)).astype(np.float64)
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), engine="df32").cpu().numpy()
    assert np.array_equal(out, A @ B)   # |a b| < 2^20: exact products, sums below 2^27: exact
    Z = torch.zeros((5, 0), dtype=torch.float64, device="cuda")
    C0 = torch.full((5, 4), 2.0, dtype=torch.float64, device="cuda")
    out = dgemm(Z, torch.zeros((0, 4), dtype=torch.float64, device="cuda"), beta=0.5, C=C0, engine="df32")
    assert torch.equal(out.cpu(), torch.full((5, 4), 1.0, dtype=torch.float64))

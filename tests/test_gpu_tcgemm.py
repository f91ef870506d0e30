"""The FP64 products on the tensor cores (svlcov_dgemm, engine 1: Ozaki
digit splitting, exact BF16 digit products in FP32 tensor memory) against
numpy's FP64 product and the FP64-pipe engine, through the C ABI.

Bound: the eight digits represent every element exactly on the grid of its
row's (column's) largest exponent, and the dropped digit pairs (s + t >= 8)
stay below 2^-53 of the product of the two scales per term, so
|C_tc - AB| <= c K 2^-52 max|a_i.| max|b_.j| beside the FP64 rounding
K eps |A||B| of the reference itself (c = 4)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _ref(A, B, ta, tb):
    a = A.T if ta else A
    b = B.T if tb else B
    return a, b, a @ b


def _bound(a, b):
    K = a.shape[1]
    rm = np.abs(a).max(axis=1)[:, None]
    cm = np.abs(b).max(axis=0)[None, :]
    return 4 * K * 2.0 ** -52 * rm * cm + 2 * K * EPS * (np.abs(a) @ np.abs(b))


SHAPES = [(1, 1, 1), (7, 5, 3), (64, 64, 64), (320, 72, 320), (256, 256, 256), (200, 130, 1100),
          (129, 65, 1152), (1152, 128, 64), (33, 300, 17)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_tensor_dgemm_matches_fp64(M, N, K, ta, tb):
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(M * 131 + N * 7 + K + 3 * ta + tb)
    A = g.standard_normal((K, M) if ta else (M, K)) * np.exp(g.uniform(-3, 3, size=(K, M) if ta else (M, K)))
    B = g.standard_normal((N, K) if tb else (K, N))
    a, b, C = _ref(A, B, ta, tb)
    At, Bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
    Ctc = dgemm(At, Bt, ta=ta, tb=tb, engine="tensor").cpu().numpy()
    C64 = dgemm(At, Bt, ta=ta, tb=tb, engine="fp64").cpu().numpy()
    bnd = _bound(a, b)
    assert np.all(np.abs(Ctc - C) <= bnd), float(np.max(np.abs(Ctc - C) / bnd))
    assert np.all(np.abs(C64 - C) <= bnd)


def test_tensor_dgemm_alpha_beta_and_exact_integers():
    """Small integers are single digits: their products come out exact."""
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(7)
    A = g.integers(-127, 128, size=(150, 300)).astype(np.float64)
    B = g.integers(-127, 128, size=(300, 90)).astype(np.float64)
    C0 = g.integers(-5, 6, size=(150, 90)).astype(np.float64)
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), alpha=2.0, beta=-3.0,
                C=torch.as_tensor(C0, device="cuda"), engine="tensor").cpu().numpy()
    assert np.array_equal(out, 2.0 * (A @ B) - 3.0 * C0)


def test_tensor_dgemm_wide_dynamic_range_and_nonfinite():
    from paper_2401_09703_gb300 import dgemm
    g = synth.rng(8)
    A = g.standard_normal((96, 80))
    A[3, :] *= 1e200
    A[5, :] *= 1e-200
    A[7, 10] = 0.0
    B = g.standard_normal((80, 40))
    B[:, 2] *= 1e-150
    C = A @ B
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), engine="tensor").cpu().numpy()
    assert np.all(np.abs(out - C) <= _bound(A, B))
    A[11, 4] = np.nan
    B[9, 30] = np.inf
    out = dgemm(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda"), engine="tensor").cpu().numpy()
    assert np.all(np.isnan(out[11, :])) and np.all(np.isnan(out[:, 30]))
    ok = np.ones_like(out, dtype=bool)
    ok[11, :] = False
    ok[:, 30] = False
    assert np.all(np.isfinite(out[ok]))


def test_tensor_dgemm_rejects_bad_sizes():
    from paper_2401_09703_gb300 import _abi
    L = _abi.lib()
    assert L.svlcov_dgemm(0, 0, 5000, 4, 4, 1.0, None, 5000, None, 4, 0.0, None, 5000, 1, None) == \
        _abi.SVLCOV_ERR_INVALID_ARG
    assert L.svlcov_dgemm(0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 3, None) == _abi.SVLCOV_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_trajectory_with_tensor_products(seed):
    """A mixed-mode trajectory (all three step kinds) whose FP64 small
    products run on the tensor cores (init option tensor_gemm = 1) matches
    the FP64 oracle as the FP64-pipe products do."""
    from tests.gpu_util import compare, run_gpu, run_oracle
    from tests.test_gpu_parity import _mixed_problem
    U, s, V, ops = _mixed_problem(seed)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp64", small="mixed", tensor_gemm=1)
    assert code == 0
    c = compare(Ug, sg, Vg, run_oracle(U, s, V, ops))
    assert c["sigma"] < 1e-10 and c["sin_u"] < 1e-8 and c["sin_v"] < 1e-8, c

"""Projection of update vectors without updating (svlcov_project: P =
X'^T E^T, C0 = X^T E^T, Lemma 1's gather) against the oracle's factors, on
all storage types and both sides; out-of-range indices."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import run_gpu, run_oracle, to_dev  # noqa: E402
from tests.test_gpu_parity import _mixed_problem  # noqa: E402


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 1e-6), ("bf16", 1e-2)])
@pytest.mark.parametrize("side", [0, 1])
def test_projection_matches_oracle(storage, tol, side):
    U, s, V, ops = _mixed_problem(5, k=8)
    small = "fp64" if storage == "fp64" else "mixed"
    idt = torch.float64 if storage == "fp64" else torch.float32
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage=storage, small=small, init_dtype=idt, values_dtype=idt)
    assert code == 0
    X = Ug if side == 0 else Vg
    rng = synth.rng(77 + side)
    E = synth.random_csr_batch(300, X.shape[0], 6, rng)
    P, C0 = g.project(side, to_dev(E))
    C0 = C0.cpu().numpy()
    ref = X.T @ E.dense().T           # k x s, from the library's own factors (U = U' U'')
    assert np.max(np.abs(C0 - ref)) < tol * max(1.0, np.abs(ref).max())
    st = run_oracle(U, s, V, ops)
    Uo, so, Vo = st.factors()
    Xo = Uo if side == 0 else Vo
    refo = Xo.T @ E.dense().T         # against the oracle: the same up to the columns' signs
    sgn = np.sign(np.sum(C0 * refo, axis=1, keepdims=True))
    sgn[sgn == 0] = 1.0
    assert np.max(np.abs(C0 * sgn - refo)) < max(10 * tol, 1e-8) * max(1.0, np.abs(refo).max())
    assert g.status() == 0


def test_projection_bad_index_and_k_multiple_of_four():
    from paper_2401_09703_gb300 import _abi
    U, s, V, ops = _mixed_problem(6, k=8, steps=2)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops)
    m = Ug.shape[0]
    E = synth.CSR(np.array([0, 2], dtype=np.int32), np.array([1, m + 5], dtype=np.int32), np.ones(2), 1, m)
    g.project(0, to_dev(E))
    assert g.status() & _abi.SVLCOV_DEV_BAD_CSR
    U, s, V, ops = _mixed_problem(6, k=6, steps=2)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops)
    E = synth.random_csr_batch(3, Ug.shape[0], 2, synth.rng(1))
    with pytest.raises(Exception):
        g.project(0, to_dev(E))

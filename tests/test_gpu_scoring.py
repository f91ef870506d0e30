"""Pair scores U[i]^T Sigma V[j] (svlcov_score_pairs, the inference step of
the downstream tasks) against the oracle's scores: on an FP64 trajectory
against the oracle's own factors; on FP32 and BF16 storage against the
oracle's scoring of the library's materialised factors (the kernel's own
arithmetic); both directions for undirected graphs; out-of-range indices."""
import numpy as np
import pytest

import synth
from oracle import scoring

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import make_gpu, dev_batch, run_gpu, run_oracle  # noqa: E402
from tests.test_gpu_parity import _mixed_problem, _small_c2  # noqa: E402


def _pairs(m, n, cnt, seed):
    g = synth.rng(seed)
    return g.integers(0, m, cnt).astype(np.int32), g.integers(0, n, cnt).astype(np.int32)


@pytest.mark.parametrize("seed", [1, 2])
def test_scores_fp64_trajectory_match_oracle(seed):
    U, s, V, ops = _mixed_problem(seed)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp64", small="fp64")
    assert code == 0
    st = run_oracle(U, s, V, ops)
    Uo, so, Vo = st.factors()
    r, c = _pairs(Uo.shape[0], Vo.shape[0], 5000, seed)
    out = g.score_pairs(torch.as_tensor(r), torch.as_tensor(c)).cpu().numpy()
    ref = scoring.score_pairs(Uo, so, Vo, r, c)
    assert np.max(np.abs(out - ref)) < 1e-9 * so[0]
    assert g.status() == 0


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_scores_of_the_librarys_factors(storage):
    U, s, V, ops = _small_c2(n_batches=3)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage=storage, small="mixed", values_dtype=torch.float32,
                                  init_dtype=torch.float32)
    assert code == 0
    N = min(Ug.shape[0], Vg.shape[0])
    r, c = _pairs(N, N, 20000, 7)
    for sym in (False, True):
        out = g.score_pairs(torch.as_tensor(r), torch.as_tensor(c), symmetric=sym).cpu().numpy()
        ref = scoring.score_pairs(Ug, sg, Vg, r, c, symmetric=sym)
        # FP32 arithmetic on the stored rows: a few eps32 of |U'[i]| |M| |V'[j]|
        scale = sg[0] * np.abs(Ug).max() * np.abs(Vg).max() * Ug.shape[1]
        assert np.max(np.abs(out - ref)) < 3e-6 * scale, float(np.max(np.abs(out - ref)) / scale)


def test_scores_out_of_range_and_empty():
    from paper_2401_09703_gb300 import _abi
    U, s, V, ops = _mixed_problem(3, steps=2)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops)
    m, n = Ug.shape[0], Vg.shape[0]
    assert g.score_pairs(torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=torch.int32)).numel() == 0
    r = torch.tensor([0, m, 1, -1], dtype=torch.int32)
    c = torch.tensor([0, 0, n, 2], dtype=torch.int32)
    out = g.score_pairs(r, c).cpu().numpy()
    assert np.isfinite(out[0]) and np.all(np.isnan(out[1:]))
    assert g.status() & _abi.SVLCOV_DEV_BAD_CSR

"""The dense fold X' W on the tensor cores (BF16 pieces, FP32 accumulation):
the materialised factors U = U' U'' and the in-place reset X' <- X' W
against FP64 products of the library's own stored factors, and a forced
reset on every fold against the oracle, for k multiples of 16 (the tensor
path) and storage FP32 / BF16."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import compare, run_gpu, run_oracle  # noqa: E402
from tests.test_gpu_parity import _mixed_problem  # noqa: E402


@pytest.mark.parametrize("k", [16, 48, 64, 128])
@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_materialise_matches_fp64_product(k, storage):
    from paper_2401_09703_gb300 import SVLCOV
    g0 = synth.rng(300 + k)
    m, n = 1000 + 37, 700 + 5                      # ragged last tile
    U, _ = np.linalg.qr(g0.standard_normal((m, k)))
    V, _ = np.linalg.qr(g0.standard_normal((n, k)))
    s = np.sort(g0.uniform(1, 10, k))[::-1].copy()
    dev = torch.device("cuda")
    h = SVLCOV(torch.as_tensor(U, dtype=torch.float32, device=dev), torch.as_tensor(s, device=dev),
               torch.as_tensor(V, dtype=torch.float32, device=dev), max_m=m + 8, max_n=n + 32, max_s=8, max_nnz=64,
               storage=storage, small="mixed", reorth=-1)
    # a few column steps so that U'' is a general matrix
    for t in range(3):
        b = synth.random_csr_batch(8, m, 4, g0)
        from tests.gpu_util import to_dev
        h.add_cols(to_dev(b, torch.float32))
    assert h.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in h.get_factors(torch.float64))
    # the stored U' and U'' give the exact product in FP64
    Up = h.ubuf[: Ug.shape[0]].to(torch.float64).cpu().numpy()
    Wu = h.small_state()[0]
    ref = Up @ Wu
    err = np.max(np.abs(Ug - ref)) / (np.abs(Up).max() * np.abs(Wu).max() * k)
    assert err < 4 * 2.0 ** -24, err


# BF16: every reset rounds X' W to BF16 (relative 2^-9), so a reset on every
# fold sits at the BF16 tolerances of the fuzz suite
@pytest.mark.parametrize("storage,stol,vtol", [("fp32", 1e-5, 1e-4), ("bf16", 1e-2, 1e-1)])
def test_forced_reset_k16_matches_oracle(storage, stol, vtol):
    U, s, V, ops = _mixed_problem(7, m=80, n=60, k=16)
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage=storage, small="mixed", values_dtype=torch.float32,
                                  init_dtype=torch.float32, reset_threshold=1.0, reorth=-1)
    assert code == 0
    assert g.small_state()[3] >= len(ops)
    c = compare(Ug, sg, Vg, run_oracle(U, s, V, ops))
    assert c["sigma"] < stol and c["sin_u"] < vtol and c["sin_v"] < vtol, c

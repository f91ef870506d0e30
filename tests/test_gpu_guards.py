"""GPU parity of the conditioning guard and reset (the remedy for an
ill-conditioned small factor, Section 3.2), of the singular-factor case of
the fold (reading R17), and of a whole step at the headline configuration's
shape (k = 64, s = 256, K = 320^2), all against the FP64 oracle.

* The closed-form cases of the update definition (tests/golden/) run through
  the GPU: among them ``cols_replaces_direction``, where the new small factor
  U''(F[:k] - C_Q F[k:]) is exactly zero (the old direction leaves the top k),
  so the fold must take the reset form instead of inverting it.
* A reset threshold of 1 makes every fold reset (cond_1(W) >= 1 always): the
  factors stay those of the oracle (a reset leaves U' U'' unchanged), on FP64
  and FP32 storage.
* The C2 node-insertion step at k = 64, s = 256 (N = 20,000): the n = 320
  cluster Jacobi, the s = 256 panel Cholesky and the column-parallel inverse,
  as they run in the headline benchmark.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import checks, svlcov as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import compare, dev_batch, make_gpu, run_gpu, run_oracle  # noqa: E402
from tests.test_gpu_parity import _mixed_problem  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cases.json")


def _csr(d):
    return synth.CSR(np.array(d["indptr"], dtype=np.int32), np.array(d["indices"], dtype=np.int32),
                     np.array(d["values"], dtype=np.float64), d["rows"], d["cols"])


@pytest.mark.parametrize("small", ["fp64", "mixed"])
@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_closed_form_cases_on_gpu(case, small):
    U = np.array(case["U"]); s = np.array(case["sigma"]); V = np.array(case["V"])
    batch = (_csr(case["D"]), _csr(case["E"])) if case["op"] == "weights" else _csr(case["batch"])
    ops = [(case["op"], batch)]
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage="fp64", small=small)
    assert code == 0
    se = np.array(case["sigma_out"])
    assert np.max(np.abs(sg - se)) < 1e-12 * max(1.0, se[0]), (sg, se)
    assert checks.projector_err(Ug, np.array(case["U_out"])) < 1e-12
    assert checks.projector_err(Vg, np.array(case["V_out"])) < 1e-12
    if case["name"] == "cols_replaces_direction":
        assert g.small_state()[3] >= 1          # the fold went through the reset form (R17)


@pytest.mark.parametrize("storage,small,stol,vtol", [("fp64", "fp64", 1e-10, 1e-8),
                                                     ("fp32", "mixed", 1e-5, 1e-4)])
@pytest.mark.parametrize("seed", [1, 2])
def test_forced_reset_every_step_matches_oracle(seed, storage, small, stol, vtol):
    U, s, V, ops = _mixed_problem(seed)
    idt = torch.float64 if storage == "fp64" else torch.float32
    g, code, Ug, sg, Vg = run_gpu(U, s, V, ops, storage=storage, small=small, values_dtype=idt, init_dtype=idt,
                                  reset_threshold=1.0)
    assert code == 0
    resets = g.small_state()[3]
    assert resets >= len(ops), resets         # every fold reset (two per cols/rows step, two per weights step)
    c = compare(Ug, sg, Vg, run_oracle(U, s, V, ops))
    assert c["sigma"] < stol and c["sin_u"] < vtol and c["sin_v"] < vtol, c
    if storage == "fp64":
        assert checks.orth_err(Ug) < 1e-10 and checks.orth_err(Vg) < 1e-10
    # the small factors are the identity after a reset of both sides
    Wu, _, Wv, _ = g.small_state()
    if resets == 2 * len(ops):
        assert np.max(np.abs(Wu - np.eye(Wu.shape[0]))) == 0.0
        assert np.max(np.abs(Wv - np.eye(Wv.shape[0]))) == 0.0


def test_c2_step_at_headline_shape():
    """Four C2 node batches (add_rows then add_cols, s = 256) at k = 64 on a
    Chung-Lu graph of 20,000 nodes, FP32 factors with the mixed small steps
    (the headline path), against the oracle after every node batch."""
    p = synth.c2_problem(N=20_000, k=64, s=256, n_batches=4, power_iters=2)
    U, s, V, ops = p["U"], p["sigma"], p["V"], p["batches"]
    assert all(b.rows == 256 for _, b in ops)
    g = make_gpu(U, s, V, ops, storage="fp32", small="mixed", init_dtype=torch.float32)
    st = osv.State.init(U, s, V)
    for t, (kind, b) in enumerate(ops):
        g.apply(kind, dev_batch(kind, b, torch.float32))
        st.apply(kind, b)
        if kind == "cols":
            so = st.sigma
            assert checks.sigma_rel_err(g.sigma().cpu().numpy(), so) < 1e-5, t
    assert g.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    c = compare(Ug, sg, Vg, st)
    assert c["k_prime"] >= 8, c
    assert c["sigma"] < 1e-5, c
    assert c["sin_u"] < 1e-4 and c["sin_v"] < 1e-4, c

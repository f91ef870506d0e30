"""GPU parity of the -GKL and -RPI variants (approximate augmented space)
against the FP64 oracle (oracle.approx, pinned in test_oracle_approx.py),
with the same starting vectors on both sides.

Tolerances as for the exact steps (R15): FP64 factors and small steps 1e-10 on
singular values and 1e-8 on subspace sines; FP32 factors with mixed small
steps 1e-5 / 1e-4.  The approximate K is factored on the GPU through
K K^T = L L^T (a Gram of a (k + l) x (k + s) matrix), which keeps FP64
accuracy for the leading singular values when theta_1 / theta_k is moderate.
"""
import numpy as np
import pytest

import synth
from oracle import approx, checks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev_batch, make_gpu  # noqa: E402
from tests.test_oracle_pins import _mixed_problem  # noqa: E402


def _run(U, s, V, ops, method, lfun, storage, small, seed=5, t=3):
    g = make_gpu(U, s, V, ops, storage=storage, small=small,
                 init_dtype=torch.float64 if storage == "fp64" else torch.float32)
    st = approx.ApproxState.init(U, s, V)
    rng = synth.rng(seed)
    vdt = torch.float64 if storage == "fp64" else torch.float32
    for kind, b in ops:
        ss = b[0].rows if kind == "weights" else b.rows
        l = lfun(ss)
        start = rng.standard_normal(ss) if method == "gkl" else rng.standard_normal((ss, l))
        st.apply_approx(kind, b, method, l, start, t)
        g.apply_approx(kind, dev_batch(kind, b, vdt), method, l, torch.as_tensor(start), t)
    code = g.status()
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    Uo, so, Vo = st.factors()
    return code, checks.compare(Ug, sg, Vg, Uo, so, Vo)


@pytest.mark.parametrize("method", ["gkl", "rpi"])
@pytest.mark.parametrize("lmode", ["full", "partial"])
@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_trajectory_fp64(method, lmode, seed):
    U, s, V, ops = _mixed_problem(seed)
    lfun = (lambda ss: ss) if lmode == "full" else (lambda ss: max(1, ss - 1))
    code, c = _run(U, s, V, ops, method, lfun, "fp64", "fp64")
    assert code == 0
    assert c["sigma"] < 1e-10, c
    assert c["sin_u"] < 1e-8 and c["sin_v"] < 1e-8, c


@pytest.mark.parametrize("method", ["gkl", "rpi"])
@pytest.mark.parametrize("storage,small,tol", [("fp64", "fp64", 1e-10), ("fp64", "mixed", 1e-8),
                                               ("fp32", "mixed", 1e-5)])
def test_c3_like_wide_batches(method, storage, small, tol):
    """Ratings, users appended in batches of s = 512 with l = 10 (the setting
    the variants are for: the dense work drops from O(s^3) to O(s^2 l))."""
    p = synth.c3_problem(n_users=20000, n_items=5000, k=32, s=512, n_batches=2, power_iters=2)
    code, c = _run(p["U"], p["sigma"], p["V"], p["batches"], method, lambda ss: 10, storage, small)
    assert code == 0
    assert c["sigma"] < tol, c
    stol = 1e-8 if tol < 1e-9 else 10 * tol
    assert c["sin_u"] < stol and c["sin_v"] < stol, c


def test_bad_arguments_are_host_errors():
    from paper_2401_09703_gb300 import SvlcovError
    U, s, V, ops = _mixed_problem(3)
    g = make_gpu(U, s, V, ops)
    kind, b = ops[0]
    db = dev_batch(kind, b)
    with pytest.raises(SvlcovError):
        g.add_cols_approx(db, "gkl", b.rows + 1)           # l > s
    with pytest.raises(SvlcovError):
        g.add_cols_approx(db, "rpi", 1, start=None)        # RPI needs its start
    g.add_cols_approx(db, "gkl", 1)                        # p_1 = all ones
    assert g.status() == 0
    with pytest.raises(SvlcovError):
        g.intermediate(4)                                  # no exact-step intermediates

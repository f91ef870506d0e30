"""Randomised trajectories on the GPU against the FP64 oracle: small k and
s (including 1), empty update vectors, all three step kinds, every storage
and small-step precision, and the approximate-space variants.  Seeded;
sized so the oracle finishes each case in well under a second.  Singular
values are compared relative to sigma_1 (random spectra can hold values far
below it, whose own relative error only measures the precision mode)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import approx, checks, svlcov as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev_batch, make_gpu  # noqa: E402


def _case(seed):
    g = synth.rng(5000 + seed)
    m, n = int(g.integers(20, 70)), int(g.integers(15, 60))
    k = int(g.integers(1, min(m, n, 12)))
    A = sp.random(m, n, density=float(g.uniform(0.1, 0.4)), random_state=seed,
                  data_rvs=lambda x: g.standard_normal(x)).toarray()
    U, s, V = synth.init_factors(A, k, seed)
    ops, mm, nn = [], m, n
    for t in range(int(g.integers(3, 9))):
        kind = ("cols", "rows", "weights")[int(g.integers(0, 3))]
        ss = int(g.integers(1, 9))
        per = int(g.integers(1, 5))
        if kind == "cols":
            b = synth.random_csr_batch(ss, mm, per, g); nn += ss
        elif kind == "rows":
            b = synth.random_csr_batch(ss, nn, per, g); mm += ss
        else:
            b = (synth.random_csr_batch(ss, mm, per, g), synth.random_csr_batch(ss, nn, per, g))
        if kind != "weights" and g.uniform() < 0.3:   # an empty update vector
            r = int(g.integers(0, ss))
            keep = [j for j in range(ss) if j != r]
            rr, cc, vv = [], [], []
            for j in keep:
                a0, a1 = b.indptr[j], b.indptr[j + 1]
                rr += [j] * (a1 - a0); cc += list(b.indices[a0:a1]); vv += list(b.values[a0:a1])
            b = synth.csr_from_coo(np.array(rr, dtype=np.int64), np.array(cc, dtype=np.int64), np.array(vv), ss, b.cols)
        ops.append((kind, b))
    return U, s, V, ops


MODES = [("fp64", "fp64", 1e-9, 1e-6), ("fp64", "mixed", 1e-7, 1e-5), ("fp32", "mixed", 2e-5, 2e-3),
         ("fp32", "fp32", 2e-4, 2e-2), ("bf16", "mixed", 1e-2, 1e-1)]


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("storage,small,stol,vtol", MODES)
def test_random_trajectory(seed, storage, small, stol, vtol):
    U, s, V, ops = _case(seed)
    idt = torch.float64 if storage == "fp64" else torch.float32
    g = make_gpu(U, s, V, ops, storage=storage, small=small, init_dtype=idt)
    st = osv.State.init(U, s, V)
    for kind, b in ops:
        g.apply(kind, dev_batch(kind, b, idt))
        st.apply(kind, b)
    assert g.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    Uo, so, Vo = st.factors()
    c = checks.compare(Ug, sg, Vg, Uo, so, Vo, rel_gap=1e-2)
    c["sigma_vs_s1"] = float(np.max(np.abs(sg - so)) / so[0])
    assert c["sigma_vs_s1"] < stol, c
    assert c["sin_u"] < vtol and c["sin_v"] < vtol, c


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("method", ["gkl", "rpi"])
def test_random_trajectory_approximate(seed, method):
    U, s, V, ops = _case(seed)
    g = make_gpu(U, s, V, ops, storage="fp64", small="fp64")
    st = approx.ApproxState.init(U, s, V)
    rng = synth.rng(77 + seed)
    for kind, b in ops:
        ss = b[0].rows if kind == "weights" else b.rows
        l = int(rng.integers(1, ss + 1))
        start = rng.standard_normal(ss) if method == "gkl" else rng.standard_normal((ss, l))
        st.apply_approx(kind, b, method, l, start, 2)
        g.apply_approx(kind, dev_batch(kind, b), method, l, torch.as_tensor(start), 2)
    assert g.status() == 0
    Ug, sg, Vg = (x.cpu().numpy() for x in g.get_factors())
    Uo, so, Vo = st.factors()
    c = checks.compare(Ug, sg, Vg, Uo, so, Vo, rel_gap=1e-2)
    c["sigma_vs_s1"] = float(np.max(np.abs(sg - so)) / so[0])
    assert c["sigma_vs_s1"] < 1e-9 and c["sin_u"] < 1e-6 and c["sin_v"] < 1e-6, c

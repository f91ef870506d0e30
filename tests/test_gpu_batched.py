"""GPU tests of the batched path (svlcov_batch_run): many independent
handles updated concurrently give the same factors, bit for bit, as the
same updates run one handle at a time, and match the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import checks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev_batch, make_gpu, run_oracle  # noqa: E402


def _problem(seed=7):
    return synth.c4_problem(seed=seed, n_mats=5, m_lo=300, m_hi=900, density=0.02, ks=(6, 12), n_batches=4,
                            s_lo=3, s_hi=14, per_vec=4, power_iters=2)


@pytest.mark.parametrize("storage,small,tol,split", [("fp64", "fp64", 1e-10, 0), ("fp32", "mixed", 1e-5, 0),
                                                     ("fp32", "mixed", 1e-5, -1), ("fp64", "mixed", 1e-7, -1)])
def test_batched_equals_sequential_and_oracle(storage, small, tol, split):
    """Batched and sequential runs of the same handles are bit-identical, with
    the FP64 products split over clusters (default) or not (gemm_split < 0)."""
    from paper_2401_09703_gb300 import batch_run
    p = _problem()
    vd = torch.float64 if storage == "fp64" else torch.float32
    idt = torch.float64 if storage == "fp64" else torch.float32
    seq, bat, dev = [], [], []
    for mat in p["mats"]:
        ops = mat["batches"]
        kw = dict(storage=storage, small=small, init_dtype=idt, gemm_split=split)
        seq.append(make_gpu(mat["U"], mat["sigma"], mat["V"], ops, **kw))
        bat.append(make_gpu(mat["U"], mat["sigma"], mat["V"], ops, **kw))
        dev.append([dev_batch(kind, b, vd) for kind, b in ops])
    for r in range(len(p["mats"][0]["batches"])):
        for h, d in zip(seq, dev):
            h.update_weights(*d[r])
        batch_run([(h, "weights", d[r]) for h, d in zip(bat, dev)], concurrency=3)
    for i, mat in enumerate(p["mats"]):
        assert seq[i].status() == 0 and bat[i].status() == 0
        Us, ss, Vs = (x.cpu().numpy() for x in seq[i].get_factors())
        Ub, sb, Vb = (x.cpu().numpy() for x in bat[i].get_factors())
        assert np.array_equal(Us, Ub) and np.array_equal(ss, sb) and np.array_equal(Vs, Vb)
        st = run_oracle(mat["U"], mat["sigma"], mat["V"], mat["batches"])
        Uo, so, Vo = st.factors()
        c = checks.compare(Ub, sb, Vb, Uo, so, Vo)
        assert c["sigma"] < tol and c["sin_u"] < 10 * tol and c["sin_v"] < 10 * tol, (i, c)


def test_batched_run_captured_in_a_cuda_graph():
    """The batched run only enqueues work on streams forked from the caller's
    stream, so a whole round can be captured and replayed as one graph."""
    from paper_2401_09703_gb300 import batch_run
    p = _problem(seed=8)
    ref, gr, dev = [], [], []
    for mat in p["mats"]:
        ops = mat["batches"]
        ref.append(make_gpu(mat["U"], mat["sigma"], mat["V"], ops, storage="fp32", small="mixed",
                            init_dtype=torch.float32))
        gr.append(make_gpu(mat["U"], mat["sigma"], mat["V"], ops, storage="fp32", small="mixed",
                           init_dtype=torch.float32))
        dev.append([dev_batch(kind, b, torch.float32) for kind, b in ops])
    R = len(p["mats"][0]["batches"])
    for r in range(R):
        batch_run([(h, "weights", d[r]) for h, d in zip(ref, dev)], concurrency=4)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for r in range(R):
                batch_run([(h, "weights", d[r]) for h, d in zip(gr, dev)], concurrency=4, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, gr):
        assert b.status() == 0
        Ua, sa, Va = (x.cpu().numpy() for x in a.get_factors())
        Ub, sb, Vb = (x.cpu().numpy() for x in b.get_factors())
        assert np.array_equal(Ua, Ub) and np.array_equal(sa, sb) and np.array_equal(Va, Vb)


def test_steps_with_empty_batches_capture_in_a_cuda_graph():
    """Single-vector steps, some with no nonzeros (isolated nodes of a graph
    stream), captured in one CUDA graph: no zero-block launch may invalidate
    the capture, and the replay equals the same steps run without a graph."""
    p = synth.c2_problem(N=3000, k=8, s=1, n_batches=12, power_iters=2)
    ops = p["batches"]
    assert any(b.nnz == 0 for _, b in ops)
    outs = []
    for graph in (False, True):
        g = make_gpu(p["U"], p["sigma"], p["V"], ops, storage="fp32", small="mixed", init_dtype=torch.float32)
        bats = [(kind, dev_batch(kind, b, torch.float32)) for kind, b in ops]
        st = torch.cuda.Stream()
        if graph:
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.stream(st):
                with torch.cuda.graph(cg, stream=st):
                    for kind, b in bats:
                        g.apply(kind, b, stream=st)
            cg.replay()
        else:
            for kind, b in bats:
                g.apply(kind, b, stream=st)
        torch.cuda.synchronize()
        assert g.status() == 0
        outs.append([x.cpu().numpy() for x in g.get_factors()])
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)

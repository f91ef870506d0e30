"""Helpers for the GPU parity tests: run a synthetic trajectory through the
CUDA library (C ABI) and through the FP64 oracle."""
import numpy as np
import torch

from oracle import checks, svlcov as osv


def to_dev(b, dtype=torch.float64):
    from paper_2401_09703_gb300 import DeviceCSR
    return DeviceCSR.from_host(b.indptr, b.indices, b.values, b.rows, b.cols, values_dtype=dtype)


def dev_batch(kind, b, dtype=torch.float64):
    if kind == "weights":
        return (to_dev(b[0], dtype), to_dev(b[1], dtype))
    return to_dev(b, dtype)


def capacities(U, V, ops):
    m, n = U.shape[0], V.shape[0]
    max_s, max_nnz = 1, 1
    mm, nn = m, n
    for kind, b in ops:
        if kind == "cols":
            nn += b.rows; max_s = max(max_s, b.rows); max_nnz = max(max_nnz, b.nnz)
        elif kind == "rows":
            mm += b.rows; max_s = max(max_s, b.rows); max_nnz = max(max_nnz, b.nnz)
        else:
            max_s = max(max_s, b[0].rows); max_nnz = max(max_nnz, b[0].nnz, b[1].nnz)
    return mm, nn, max_s, max_nnz


def make_gpu(U, s, V, ops, storage="fp64", small="fp64", init_dtype=torch.float64, **kw):
    from paper_2401_09703_gb300 import SVLCOV
    mm, nn, max_s, max_nnz = capacities(U, V, ops)
    dev = torch.device("cuda")
    return SVLCOV(torch.as_tensor(U, dtype=init_dtype, device=dev), torch.as_tensor(s, device=dev),
                  torch.as_tensor(V, dtype=init_dtype, device=dev), max_m=mm + 8, max_n=nn + 8, max_s=max_s,
                  max_nnz=max_nnz, storage=storage, small=small, **kw)


def run_gpu(U, s, V, ops, storage="fp64", small="fp64", values_dtype=torch.float64, **kw):
    g = make_gpu(U, s, V, ops, storage=storage, small=small, **kw)
    for kind, b in ops:
        g.apply(kind, dev_batch(kind, b, values_dtype))
    code = g.status()
    Ug, sg, Vg = g.get_factors(torch.float64)
    torch.cuda.synchronize()
    return g, code, Ug.cpu().numpy(), sg.cpu().numpy(), Vg.cpu().numpy()


def run_oracle(U, s, V, ops):
    st = osv.State.init(U, s, V)
    for kind, b in ops:
        st.apply(kind, b)
    return st


def compare(Ug, sg, Vg, st):
    Uo, so, Vo = st.factors()
    return checks.compare(Ug, sg, Vg, Uo, so, Vo)

"""Torch-side convenience wrapper over the C ABI.

PyTorch provides device memory and streams only: buffers are allocated as
torch tensors and their pointers are handed to the library; every update
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np
import torch

from . import _abi
from ._abi import check, lib

_STORAGE = {"fp64": _abi.SVLCOV_FP64, "fp32": _abi.SVLCOV_FP32, "bf16": _abi.SVLCOV_BF16}
_SMALL = {"fp64": _abi.SVLCOV_SMALL_FP64, "fp32": _abi.SVLCOV_SMALL_FP32, "mixed": _abi.SVLCOV_SMALL_MIXED}
_TORCH_STORAGE = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class DeviceCSR:
    """A batch of update vectors on the device (row j = update vector j)."""
    indptr: torch.Tensor   # int32, rows + 1
    indices: torch.Tensor  # int32, nnz
    values: torch.Tensor   # float32 or float64, nnz
    rows: int
    cols: int

    @property
    def nnz(self) -> int:
        return int(self.indices.numel())

    def c(self) -> _abi.svlcov_csr:
        vd = _abi.SVLCOV_FP64 if self.values.dtype == torch.float64 else _abi.SVLCOV_FP32
        return _abi.svlcov_csr(self.rows, self.cols, self.nnz, self.indptr.data_ptr(),
                               self.indices.data_ptr() if self.nnz else None,
                               self.values.data_ptr() if self.nnz else None, vd)

    @staticmethod
    def from_host(indptr, indices, values, rows: int, cols: int, device="cuda",
                  values_dtype=torch.float32, non_blocking=False) -> "DeviceCSR":
        ip = torch.as_tensor(np.asarray(indptr, dtype=np.int32)).to(device, non_blocking=non_blocking)
        ix = torch.as_tensor(np.asarray(indices, dtype=np.int32)).to(device, non_blocking=non_blocking)
        vv = torch.as_tensor(np.asarray(values)).to(device=device, dtype=values_dtype, non_blocking=non_blocking)
        return DeviceCSR(ip, ix, vv, int(rows), int(cols))


class SVLCOV:
    """A rank-k truncated SVD maintained on one GPU (Section 3.2 extended
    decomposition); see include/svlcov.h for the semantics of each call."""

    def __init__(self, U0: torch.Tensor, sigma0: torch.Tensor, V0: torch.Tensor, *, max_m: int, max_n: int,
                 max_s: int, max_nnz: int, storage: str = "fp32", small: str = "mixed", tau: float = 0.0,
                 reset_threshold: float = 0.0, jacobi_block: int = 0, reorth: int = 0, gemm_split: int = 0,
                 tensor_gemm: int = 0, s1_secular: int = 0, literal_steps: int = 0, stream=None):
        assert U0.is_cuda and V0.is_cuda and sigma0.is_cuda
        m, k = U0.shape
        n = V0.shape[0]
        dev = U0.device
        self.k, self.storage, self.small = int(k), storage, small
        self.literal_steps = int(literal_steps)
        self.device = dev
        tdt = _TORCH_STORAGE[storage]
        self.ubuf = torch.empty((max_m, k), dtype=tdt, device=dev)
        self.vbuf = torch.empty((max_n, k), dtype=tdt, device=dev)
        self._U0 = U0.contiguous()
        self._V0 = V0.contiguous()
        self._s0 = sigma0.to(torch.float64).contiguous()
        init_dtype = _abi.SVLCOV_FP64 if U0.dtype == torch.float64 else _abi.SVLCOV_FP32
        d = _abi.svlcov_init_desc()
        d.m, d.n, d.k = m, n, k
        d.max_m, d.max_n, d.max_s, d.max_nnz = max_m, max_n, max_s, max_nnz
        d.storage, d.small = _STORAGE[storage], _SMALL[small]
        d.U0, d.sigma0, d.V0, d.init_dtype = self._U0.data_ptr(), self._s0.data_ptr(), self._V0.data_ptr(), init_dtype
        d.ubuf, d.vbuf = self.ubuf.data_ptr(), self.vbuf.data_ptr()
        d.tau, d.reset_threshold = tau, reset_threshold
        d.jacobi_block = jacobi_block
        d.reorth = reorth
        d.gemm_split = gemm_split
        d.tensor_gemm = tensor_gemm
        d.s1_secular = s1_secular
        d.literal_steps = literal_steps
        nbytes = lib().svlcov_workspace_bytes(C.byref(d))
        if nbytes == 0:
            raise _abi.SvlcovError(_abi.SVLCOV_ERR_INVALID_ARG, "svlcov_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        d.workspace, d.workspace_bytes = aligned, nbytes
        self._desc = d
        h = C.c_void_p()
        check(lib().svlcov_init(C.byref(h), C.byref(d), _stream(stream)), "svlcov_init")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().svlcov_destroy(h)
            self.h = None

    # ---- updates -------------------------------------------------------------
    def add_cols(self, batch: DeviceCSR, stream=None):
        check(lib().svlcov_add_cols(self.h, C.byref(batch.c()), _stream(stream)), "svlcov_add_cols")

    def add_rows(self, batch: DeviceCSR, stream=None):
        check(lib().svlcov_add_rows(self.h, C.byref(batch.c()), _stream(stream)), "svlcov_add_rows")

    def update_weights(self, D: DeviceCSR, E: DeviceCSR, stream=None):
        check(lib().svlcov_update_weights(self.h, C.byref(D.c()), C.byref(E.c()), _stream(stream)),
              "svlcov_update_weights")

    # ---- approximate augmented space (-GKL / -RPI) -------------------------------
    def _approx(self, method: str, l: int, start: Optional[torch.Tensor], t: int) -> _abi.svlcov_approx:
        nb = lib().svlcov_approx_work_bytes(self.h, int(l))
        if nb == 0:
            raise _abi.SvlcovError(_abi.SVLCOV_ERR_INVALID_ARG, "svlcov_approx_work_bytes")
        if getattr(self, "_ap_work", None) is None or self._ap_work.numel() < nb + 256:
            self._ap_work = torch.empty(nb + 256, dtype=torch.uint8, device=self.device)
        st = None
        if start is not None:   # column-major s x l (or s) FP64 on the device
            st = start.to(device=self.device, dtype=torch.float64)
            st = (st.t() if st.dim() == 2 else st).contiguous()
        self._ap_start = st
        m = {"gkl": _abi.SVLCOV_APPROX_GKL, "rpi": _abi.SVLCOV_APPROX_RPI}[method]
        return _abi.svlcov_approx(m, int(l), int(t), None if st is None else st.data_ptr(),
                                  (self._ap_work.data_ptr() + 255) & ~255)

    def add_cols_approx(self, batch: DeviceCSR, method: str, l: int, start: Optional[torch.Tensor] = None,
                        t: int = 3, stream=None):
        """Add columns with an approximate augmented space (start: GKL p_1 (s,)
        or RPI starting matrix (s, l), row-major)."""
        a = self._approx(method, l, start, t)
        check(lib().svlcov_add_cols_approx(self.h, C.byref(batch.c()), C.byref(a), _stream(stream)),
              "svlcov_add_cols_approx")

    def add_rows_approx(self, batch: DeviceCSR, method: str, l: int, start: Optional[torch.Tensor] = None,
                        t: int = 3, stream=None):
        a = self._approx(method, l, start, t)
        check(lib().svlcov_add_rows_approx(self.h, C.byref(batch.c()), C.byref(a), _stream(stream)),
              "svlcov_add_rows_approx")

    def update_weights_approx(self, D: DeviceCSR, E: DeviceCSR, method: str, l: int,
                              start: Optional[torch.Tensor] = None, t: int = 3, stream=None):
        a = self._approx(method, l, start, t)
        check(lib().svlcov_update_weights_approx(self.h, C.byref(D.c()), C.byref(E.c()), C.byref(a),
                                                 _stream(stream)), "svlcov_update_weights_approx")

    def apply_approx(self, op: str, batch, method: str, l: int, start=None, t: int = 3, stream=None):
        if op == "cols":
            self.add_cols_approx(batch, method, l, start, t, stream)
        elif op == "rows":
            self.add_rows_approx(batch, method, l, start, t, stream)
        else:
            self.update_weights_approx(batch[0], batch[1], method, l, start, t, stream)

    def apply(self, op: str, batch, stream=None):
        if op == "cols":
            self.add_cols(batch, stream)
        elif op == "rows":
            self.add_rows(batch, stream)
        else:
            self.update_weights(batch[0], batch[1], stream)

    # ---- read back -------------------------------------------------------------
    def shape(self) -> Tuple[int, int, int]:
        m, n, k = C.c_int64(), C.c_int64(), C.c_int32()
        check(lib().svlcov_get_shape(self.h, C.byref(m), C.byref(n), C.byref(k)), "svlcov_get_shape")
        return m.value, n.value, k.value

    def get_factors(self, dtype=torch.float64, stream=None):
        m, n, k = self.shape()
        U = torch.empty((m, k), dtype=dtype, device=self.device)
        V = torch.empty((n, k), dtype=dtype, device=self.device)
        s = torch.empty(k, dtype=torch.float64, device=self.device)
        od = _abi.SVLCOV_FP64 if dtype == torch.float64 else _abi.SVLCOV_FP32
        check(lib().svlcov_get_factors(self.h, _ptr(U), _ptr(s), _ptr(V), od, _stream(stream)), "svlcov_get_factors")
        return U, s, V

    def query_rows(self, side: int, idx: torch.Tensor, dtype=torch.float64, stream=None) -> torch.Tensor:
        idx = idx.to(device=self.device, dtype=torch.int32).contiguous()
        out = torch.empty((idx.numel(), self.k), dtype=dtype, device=self.device)
        od = _abi.SVLCOV_FP64 if dtype == torch.float64 else _abi.SVLCOV_FP32
        check(lib().svlcov_query_rows(self.h, side, _ptr(idx), idx.numel(), _ptr(out), od, _stream(stream)),
              "svlcov_query_rows")
        return out

    def sigma(self, stream=None) -> torch.Tensor:
        """The current singular values (device, FP64)."""
        s = torch.empty(self.k, dtype=torch.float64, device=self.device)
        check(lib().svlcov_get_factors(self.h, None, _ptr(s), None, _abi.SVLCOV_FP64, _stream(stream)),
              "svlcov_get_factors")
        return s

    def add_cols_backward(self, batch: DeviceCSR, rows_S: torch.Tensor, U_pre_S: torch.Tensor,
                          U_pre_nnz: torch.Tensor, dU_S: torch.Tensor, dtheta: Optional[torch.Tensor],
                          gap: float = 1e-6, stream=None) -> torch.Tensor:
        """dL/d(batch values) of the last add_cols step (svlcov_add_cols_backward)."""
        dev = self.device
        rows_S = rows_S.to(device=dev, dtype=torch.int32).contiguous()
        f64 = lambda t: t.to(device=dev, dtype=torch.float64).contiguous()
        U_pre_S, U_pre_nnz, dU_S = f64(U_pre_S), f64(U_pre_nnz), f64(dU_S)
        dtheta = None if dtheta is None else f64(dtheta)
        out = torch.empty(batch.nnz, dtype=torch.float64, device=dev)
        nb = lib().svlcov_add_cols_backward_work_bytes(self.h)
        if getattr(self, "_bw_work", None) is None or self._bw_work.numel() < nb + 256:
            self._bw_work = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        wp = (self._bw_work.data_ptr() + 255) & ~255
        check(lib().svlcov_add_cols_backward(self.h, C.byref(batch.c()), _ptr(rows_S), rows_S.numel(),
                                             _ptr(U_pre_S), _ptr(U_pre_nnz), _ptr(dU_S), _ptr(dtheta), _ptr(out),
                                             float(gap), C.c_void_p(wp), _stream(stream)),
              "svlcov_add_cols_backward")
        return out

    def status(self, stream=None) -> int:
        code = C.c_int32()
        check(lib().svlcov_status(self.h, C.byref(code), _stream(stream)), "svlcov_status")
        return code.value

    def small_state(self, stream=None):
        k = self.k
        Wu = np.zeros((k, k)); Wv = np.zeros((k, k)); s = np.zeros(k); r = C.c_int64()
        check(lib().svlcov_get_small_state(self.h, Wu.ctypes.data_as(C.c_void_p), Wv.ctypes.data_as(C.c_void_p),
                                           s.ctypes.data_as(C.c_void_p), C.byref(r), _stream(stream)),
              "svlcov_get_small_state")
        return Wu, s, Wv, r.value

    def get_state(self, stream=None):
        m, n, k = self.shape()
        tdt = {"fp64": np.float64, "fp32": np.float32, "bf16": np.uint16}[self.storage]
        Up = np.zeros((m, k), dtype=tdt); Vp = np.zeros((n, k), dtype=tdt)
        Wu = np.zeros((k, k)); Wv = np.zeros((k, k)); s = np.zeros(k)
        check(lib().svlcov_get_state(self.h, Up.ctypes.data_as(C.c_void_p), Vp.ctypes.data_as(C.c_void_p),
                                     Wu.ctypes.data_as(C.c_void_p), Wv.ctypes.data_as(C.c_void_p),
                                     s.ctypes.data_as(C.c_void_p), _stream(stream)), "svlcov_get_state")
        return dict(m=m, n=n, Up=Up, Vp=Vp, Wu=Wu, Wv=Wv, sigma=s)

    def set_state(self, st: dict, stream=None):
        arrs = [np.ascontiguousarray(st[x]) for x in ("Up", "Vp", "Wu", "Wv", "sigma")]
        check(lib().svlcov_set_state(self.h, st["m"], st["n"], *[a.ctypes.data_as(C.c_void_p) for a in arrs],
                                     _stream(stream)), "svlcov_set_state")

    PHASES = ("prep", "gather_gram", "cholqr2", "svd", "fold", "apply", "jacobi_kernel")

    def profile(self, enable: bool = True):
        check(lib().svlcov_profile_enable(self.h, 1 if enable else 0), "svlcov_profile_enable")

    def profile_read(self, reset: bool = True) -> dict:
        n = len(self.PHASES)
        ms = np.zeros(n); calls = np.zeros(n, dtype=np.int64); sw = C.c_int64()
        check(lib().svlcov_profile_read(self.h, ms.ctypes.data_as(C.c_void_p), calls.ctypes.data_as(C.c_void_p), n,
                                        1 if reset else 0, C.byref(sw)), "svlcov_profile_read")
        out = {p: (float(ms[i]), int(calls[i])) for i, p in enumerate(self.PHASES)}
        out["svd_sweeps"] = int(sw.value)
        return out

    def project(self, side: int, batch: "DeviceCSR", with_c0: bool = True, stream=None):
        """P = X'^T E^T (k x s) and C0 = X^T E^T of update vectors (side 0:
        columns over U's rows, side 1: rows over V's rows) without updating."""
        k, s = self.k, batch.rows
        P = torch.empty((s, k), dtype=torch.float64, device=self.device)     # column-major k x s
        C0 = torch.empty((s, k), dtype=torch.float64, device=self.device) if with_c0 else None
        check(lib().svlcov_project(self.h, side, C.byref(batch.c()), _ptr(P), _ptr(C0), _stream(stream)),
              "svlcov_project")
        return P.t(), (C0.t() if with_c0 else None)

    def score_pairs(self, rows: torch.Tensor, cols: torch.Tensor, symmetric: bool = False,
                    stream=None) -> torch.Tensor:
        """U[rows]^T Sigma V[cols] per pair (device FP64), the larger of both
        directions when `symmetric` (undirected graphs)."""
        r = rows.to(device=self.device, dtype=torch.int32).contiguous()
        c = cols.to(device=self.device, dtype=torch.int32).contiguous()
        out = torch.empty(r.numel(), dtype=torch.float64, device=self.device)
        check(lib().svlcov_score_pairs(self.h, _ptr(r), _ptr(c), r.numel(), 1 if symmetric else 0, _ptr(out),
                                       _stream(stream)), "svlcov_score_pairs")
        return out

    def intermediate(self, which: int, side: int = 0, stream=None) -> np.ndarray:
        r, c = C.c_int32(), C.c_int32()
        check(lib().svlcov_get_intermediate(self.h, which, side, None, 0, C.byref(r), C.byref(c), _stream(stream)),
              "svlcov_get_intermediate")
        out = np.zeros(r.value * c.value)
        check(lib().svlcov_get_intermediate(self.h, which, side, out.ctypes.data_as(C.c_void_p), out.size,
                                            C.byref(r), C.byref(c), _stream(stream)), "svlcov_get_intermediate")
        return out.reshape(c.value, r.value).T   # column-major on the device


class _AddColsGrad(torch.autograd.Function):
    """One add-columns step as a differentiable function of the batch's
    stored values: returns (U_new[rows_S], Theta).  The backward runs the
    library's adjoint kernels and must come before the next step on the
    same handle (its intermediates live in the handle's workspace)."""

    @staticmethod
    def forward(ctx, values, model, batch, rows_S, gap):
        b = DeviceCSR(batch.indptr, batch.indices, values.detach(), batch.rows, batch.cols)
        U_pre_S = model.query_rows(0, rows_S)
        U_pre_nnz = model.query_rows(0, batch.indices)
        model.add_cols(b)
        ctx.model, ctx.batch, ctx.gap, ctx.vdtype = model, b, gap, values.dtype
        ctx.save_for_backward(rows_S, U_pre_S, U_pre_nnz)
        return model.query_rows(0, rows_S), model.sigma()

    @staticmethod
    def backward(ctx, dU_S, dtheta):
        rows_S, U_pre_S, U_pre_nnz = ctx.saved_tensors
        g = ctx.model.add_cols_backward(ctx.batch, rows_S, U_pre_S, U_pre_nnz, dU_S, dtheta, ctx.gap)
        return g.to(ctx.vdtype), None, None, None, None


def add_cols_with_grad(model: SVLCOV, batch: DeviceCSR, rows_S: torch.Tensor, gap: float = 1e-6):
    """model.add_cols(batch), differentiable in batch.values: returns
    (U_new[rows_S] (FP64), Theta (FP64)).  rows_S: existing rows of U, strictly
    ascending.  Needs small mode "fp64" or "mixed" (created with
    literal_steps=1) and a batch without empty
    update vectors; after backward, model.status() reports SVLCOV_DEV_GAP_WARN
    if a singular-value pair fell under the gap guard."""
    if model.small == "mixed" and model.literal_steps <= 0:
        raise ValueError("add_cols_with_grad on a mixed handle needs literal_steps=1: the backward differentiates "
                         "through R, R^-1 and F, which the default R-free mixed step does not form")
    rows_S = rows_S.to(device=model.device, dtype=torch.int32).contiguous()
    return _AddColsGrad.apply(batch.values, model, batch, rows_S, gap)


_KIND = {"cols": 0, "rows": 1, "weights": 2}


def batch_run(items, concurrency: int = 16, stream=None):
    """Enqueue many (handle, op, batch) items: svlcov_batch_run.  `items` is
    a list of (SVLCOV, "cols"|"rows"|"weights", DeviceCSR or (D, E))."""
    n = len(items)
    hs = (C.c_void_p * n)()
    ops = (_abi.svlcov_op * n)()
    for i, (h, op, batch) in enumerate(items):
        hs[i] = h.h
        ops[i].kind = _KIND[op]
        if op == "weights":
            ops[i].a = batch[0].c()
            ops[i].b = batch[1].c()
        else:
            ops[i].a = batch.c()
    check(lib().svlcov_batch_run(hs, ops, n, int(concurrency), _stream(stream)), "svlcov_batch_run")
    # the host view of each handle's shape follows the enqueued appends


def kernel_launches() -> int:
    return int(lib().svlcov_kernel_launches())


def dgemm(A: torch.Tensor, B: torch.Tensor, *, ta: bool = False, tb: bool = False, alpha: float = 1.0,
          beta: float = 0.0, C: torch.Tensor = None, engine: str = "tensor", stream=None) -> torch.Tensor:
    """alpha op(A) op(B) + beta C in FP64 with the library's product kernels
    (engine "tensor": BF16 digit products on the tensor cores; "fp64": the
    FP64 pipe; "df32": double-float on the FP32 pipe, a few 2^-44 of
    sum_k |a_ik b_kj|).  Tensors are device FP64 matrices in the usual row-major
    torch layout; they are handed to the column-major C call as transposes."""
    A = A.to(torch.float64).contiguous()
    B = B.to(torch.float64).contiguous()
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    if C is None:
        C = torch.zeros((M, N), dtype=torch.float64, device=A.device)
    Ct = C.t().contiguous()                       # column-major M x N
    # row-major A (r x c) is column-major A^T: op(A) = A means the transpose flag set on the column-major view
    check(lib().svlcov_dgemm(0 if ta else 1, 0 if tb else 1, M, N, K, alpha, _ptr(A), A.shape[1], _ptr(B),
                             B.shape[1], beta, _ptr(Ct), M, {"fp64": 0, "tensor": 1, "df32": 2}[engine], _stream(stream)),
          "svlcov_dgemm")
    return Ct.t()


def small_svd_arrow(sigma: torch.Tensor, c: torch.Tensor, rho: float, stream=None):
    """SVD_k of K = [[diag(sigma), c], [0, rho]] with the library's
    secular-equation kernel (the one-vector step's SVD)."""
    dev = sigma.device
    k = sigma.numel()
    s = sigma.to(torch.float64).contiguous()
    cc = c.to(torch.float64).contiguous()
    r = torch.tensor([float(rho)], dtype=torch.float64, device=dev)
    F = torch.empty((k, k + 1), dtype=torch.float64, device=dev)
    G = torch.empty((k, k + 1), dtype=torch.float64, device=dev)
    th = torch.empty(k, dtype=torch.float64, device=dev)
    work = torch.empty(lib().svlcov_small_svd_arrow_work_bytes() + 256, dtype=torch.uint8, device=dev)
    wp = (work.data_ptr() + 255) & ~255
    check(lib().svlcov_small_svd_arrow(_ptr(s), _ptr(cc), _ptr(r), k, _ptr(F), _ptr(th), _ptr(G), C.c_void_p(wp),
                                       _stream(stream)), "svlcov_small_svd_arrow")
    return F.t(), th, G.t()


def small_svd(K: torch.Tensor, k: int, precision: str = "fp64", stream=None):
    """SVD_k of a small dense matrix with the library's Jacobi kernel."""
    n = K.shape[0]
    Kc = K.to(torch.float64).t().contiguous()      # column-major
    F = torch.empty((k, n), dtype=torch.float64, device=K.device)
    G = torch.empty((k, n), dtype=torch.float64, device=K.device)
    th = torch.empty(k, dtype=torch.float64, device=K.device)
    work = torch.empty(lib().svlcov_small_svd_work_bytes(n) + 256, dtype=torch.uint8, device=K.device)
    wp = (work.data_ptr() + 255) & ~255
    sweeps = C.c_int32()
    check(lib().svlcov_small_svd(_ptr(Kc), n, k, _ptr(F), _ptr(th), _ptr(G), _SMALL[precision], C.c_void_p(wp),
                                 C.byref(sweeps), _stream(stream)), "svlcov_small_svd")
    return F.t(), th, G.t(), sweeps.value

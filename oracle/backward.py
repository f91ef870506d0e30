"""Reference gradient of one add-columns step (TEST INFRASTRUCTURE ONLY).

Loss (the differentiation workload): for a set S of existing rows,
    L(e) = sum_{r in S} || U_new[r] Theta^{1/2} ||^2 = sum_{r,i} U_new[r,i]^2 theta_i,
where (U_new, Theta, V_new) is the rank-k truncated SVD of [A_k  E_c] (Section
3.3 definition; Algorithm 3) and e are the stored values of the batch E_c.

`grad_autograd` differentiates the dense Zha-Simon formulation (Section 2.1:
dense augmented matrix, Householder QR, SVD of K, U_new = [U Q] F_k) with
torch float64 autograd on the CPU -- a library adjoint, independent of any
hand-written backward.  `loss_oracle` evaluates L with the paper's sparse
method (oracle.svlcov) for finite differences.
"""
from __future__ import annotations

import numpy as np
import torch

from . import svlcov


def _dense_E(indptr, indices, values_t, s: int, m: int):
    E = torch.zeros((m, s), dtype=torch.float64)
    rows, cols = [], []
    for j in range(s):
        a, b = int(indptr[j]), int(indptr[j + 1])
        rows.extend(int(x) for x in indices[a:b])
        cols.extend([j] * (b - a))
    return E.index_put((torch.tensor(rows, dtype=torch.long), torch.tensor(cols, dtype=torch.long)), values_t,
                       accumulate=False)


def loss_dense_torch(U, sigma, indptr, indices, values_t, s: int, S_rows):
    """L through the dense Zha-Simon update, differentiable in values_t."""
    U = torch.as_tensor(U, dtype=torch.float64)
    sg = torch.as_tensor(sigma, dtype=torch.float64)
    m, k = U.shape
    E = _dense_E(indptr, indices, values_t, s, m)
    C = U.T @ E
    Z = E - U @ C
    Q, R = torch.linalg.qr(Z, mode="reduced")
    K = torch.zeros((k + s, k + s), dtype=torch.float64)
    K = K.index_put((torch.arange(k), torch.arange(k)), sg)
    top = torch.cat([torch.diag(sg), C], dim=1)
    bot = torch.cat([torch.zeros((s, k), dtype=torch.float64), R], dim=1)
    K = torch.cat([top, bot], dim=0)
    F, th, Gt = torch.linalg.svd(K)
    Fk, thk = F[:, :k], th[:k]
    Un = torch.cat([U, Q], dim=1) @ Fk
    Us = Un[torch.as_tensor(S_rows, dtype=torch.long)]
    return (Us * Us * thk).sum()


def grad_autograd(U, sigma, indptr, indices, values, s: int, S_rows) -> np.ndarray:
    v = torch.tensor(np.asarray(values, dtype=np.float64), requires_grad=True)
    L = loss_dense_torch(U, sigma, indptr, indices, v, s, S_rows)
    (g,) = torch.autograd.grad(L, v)
    return g.numpy()


def loss_oracle(U, sigma, V, indptr, indices, values, s: int, S_rows) -> float:
    """L evaluated with the sparse SV-LCOV oracle (Algorithm 3)."""
    st = svlcov.State.init(U, sigma, V)
    st.add_cols(indptr, indices, values, s)
    Un = st.query_u(np.asarray(S_rows))
    return float(np.sum(Un * Un * st.sigma))


def grad_fd(U, sigma, V, indptr, indices, values, s: int, S_rows, which, h: float = 1e-3) -> np.ndarray:
    """Central finite differences of loss_oracle for the nonzeros `which`."""
    values = np.asarray(values, dtype=np.float64)
    out = np.zeros(len(which))
    for t, e in enumerate(which):
        vp = values.copy(); vp[e] += h
        vm = values.copy(); vm[e] -= h
        out[t] = (loss_oracle(U, sigma, V, indptr, indices, vp, s, S_rows) -
                  loss_oracle(U, sigma, V, indptr, indices, vm, s, S_rows)) / (2 * h)
    return out

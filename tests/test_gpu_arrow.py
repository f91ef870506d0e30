"""The one-vector SVD_k (svlcov_small_svd_arrow: secular equation of the
rank-one change K K^T = diag(sigma^2, 0) + z z^T) against LAPACK's SVD of the
same K, through the C ABI, on generic and degenerate inputs: ties in sigma,
zero components of c, rho = 0, zero sigmas, an empty update, clustered
spectra, and k = 1 closed forms."""
import numpy as np
import pytest

import synth
from oracle import checks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(name, k, g):
    sig = np.sort(g.uniform(1, 30, k))[::-1].copy()
    c = g.standard_normal(k)
    rho = 2.0
    if name == "small_update":
        c, rho = c * 1e-9, 1e-9
    elif name == "tie" and k > 1:
        sig[k // 3] = sig[k // 3 + 1]
    elif name == "zero_c":
        c[k // 5] = 0.0
    elif name == "rho0":
        rho = 0.0
    elif name == "zero_sigmas":
        sig[-3:] = 0.0
    elif name == "zero_sigmas_rho0":
        sig[-3:] = 0.0
        rho = 0.0
    elif name == "empty":
        c, rho = np.zeros(k), 0.0
    elif name == "clustered":
        sig = 30 * 0.999 ** np.arange(k)
        c = 0.1 * c
        rho = 0.5
    elif name == "huge_update":
        c, rho = 1e4 * c, 3e4
    return sig, c, rho


NAMES = ["random", "small_update", "tie", "zero_c", "rho0", "zero_sigmas", "zero_sigmas_rho0", "empty",
         "clustered", "huge_update"]


@pytest.mark.parametrize("k", [1, 2, 7, 64, 128])
@pytest.mark.parametrize("name", NAMES)
def test_arrow_svd_matches_lapack(name, k):
    from paper_2401_09703_gb300 import small_svd_arrow
    g = synth.rng(100 * k + NAMES.index(name))
    sig, c, rho = _case(name, k, g)
    K = np.zeros((k + 1, k + 1))
    K[:k, :k] = np.diag(sig)
    K[:k, k] = c
    K[k, k] = rho
    F, th, G = (x.cpu().numpy() for x in small_svd_arrow(torch.as_tensor(sig, device="cuda"),
                                                           torch.as_tensor(c, device="cuda"), rho))
    U, s, Vt = np.linalg.svd(K)
    s1 = max(s[0], 1e-300)
    assert np.max(np.abs(th - s[:k])) <= 1e-14 * s1 * np.sqrt(k + 1), (th[:4], s[:4])
    assert np.all(np.diff(th) <= 0)
    assert np.max(np.abs(F.T @ F - np.eye(k))) < 1e-13
    assert np.max(np.abs(G.T @ G - np.eye(k))) < 1e-13
    assert np.max(np.abs(K @ G - F * th)) < 1e-14 * s1 * np.sqrt(k + 1)
    assert np.max(np.abs(K.T @ F - G * th)) < 1e-14 * s1 * np.sqrt(k + 1)
    kp = checks.gapped_prefix(s[:k], 1e-6)
    if kp:
        assert checks.max_sin_angle(F[:, :kp], U[:, :kp]) < 1e-9
        assert checks.max_sin_angle(G[:, :kp], Vt.T[:, :kp]) < 1e-9

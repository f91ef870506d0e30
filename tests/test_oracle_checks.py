"""Pins of the oracle's rulers (oracle/checks.py) against answers fixed by
the mathematics alone.

Every GPU parity assertion goes through ``sigma_rel_err``,
``gapped_prefix`` and ``max_sin_angle``; a mistake in one of them would let
a wrong result pass.  Each is checked here on inputs whose answer is known in
closed form, and each plausible mistake (2-norm taken as the Frobenius norm,
the orthonormalisation left out, an off-by-one in the gap scan, an absolute
instead of a relative error, the floor ignored) is planted in a copy of the
function and shown to fail at least one of these cases.
"""
import numpy as np
import pytest

from oracle import checks


def _rot_pair(n, angles, seed=0):
    """Two orthonormal n x k blocks whose principal angles are exactly
    ``angles``: Xref = [e_0, e_2, e_4, ...], X rotates e_{2i} towards
    e_{2i+1} by angles[i]; then both go through the same random orthogonal
    map (principal angles are invariant under it)."""
    k = len(angles)
    Xref = np.zeros((n, k))
    X = np.zeros((n, k))
    for i, t in enumerate(angles):
        Xref[2 * i, i] = 1.0
        X[2 * i, i] = np.cos(t)
        X[2 * i + 1, i] = np.sin(t)
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return Q @ X, Q @ Xref


# ---------------------------------------------------------------- max_sin_angle
def test_sin_angle_single_plane():
    for t in (1e-9, 1e-4, 0.3, 1.2):
        X, Xr = _rot_pair(12, [t, 0.0, 0.0])
        assert abs(checks.max_sin_angle(X, Xr) - np.sin(t)) < 1e-15 + 1e-12 * np.sin(t)


def test_sin_angle_is_the_largest_of_several():
    # angles 0.3 and 0.2 in two planes: the largest sine is sin 0.3 (a
    # Frobenius norm would give sqrt(sin^2 0.3 + sin^2 0.2))
    X, Xr = _rot_pair(10, [0.2, 0.3, 0.0])
    assert abs(checks.max_sin_angle(X, Xr) - np.sin(0.3)) < 1e-14


def test_sin_angle_ignores_the_basis_within_the_subspace():
    # any invertible recombination of the columns spans the same subspace
    X, Xr = _rot_pair(9, [0.05, 0.0, 0.01])
    M = np.array([[2.0, 0.3, -1.0], [0.0, 0.5, 0.7], [1.0, 1.0, 3.0]])
    assert abs(checks.max_sin_angle(X @ M, Xr) - np.sin(0.05)) < 1e-13
    assert abs(checks.max_sin_angle(X, Xr @ M.T) - np.sin(0.05)) < 1e-13
    # a column sign flip is no angle at all
    assert checks.max_sin_angle(X * np.array([1, -1, 1]), X) < 1e-15


def test_sin_angle_orthogonal_and_identical():
    Xr = np.eye(6)[:, :2]
    assert abs(checks.max_sin_angle(np.eye(6)[:, 2:4], Xr) - 1.0) < 1e-15
    assert checks.max_sin_angle(Xr, Xr) == 0.0


def test_sin_angle_rank_deficient_block_fails():
    X, Xr = _rot_pair(8, [0.0, 0.0, 0.0])
    Xz = X.copy()
    Xz[:, 2] = 0.0                     # a lost direction
    assert checks.max_sin_angle(Xz, Xr) == 1.0
    Xd = X.copy()
    Xd[:, 2] = X[:, 0] + X[:, 1]       # dependent columns
    assert checks.max_sin_angle(Xd, Xr) == 1.0


def test_sin_angle_empty_block_and_width_mismatch():
    assert checks.max_sin_angle(np.zeros((5, 0)), np.zeros((5, 0))) == 0.0
    with pytest.raises(ValueError):
        checks.max_sin_angle(np.eye(5)[:, :2], np.eye(5)[:, :3])


# ---------------------------------------------------------------- gapped_prefix
GAP_CASES = [
    # (spectrum, rel_gap, k')
    ([3.0, 2.0, 1.0], 1e-3, 3),                            # gap at the end (last value against zero)
    ([5.0, 4.0, 4.0, 1e-9, 1e-9], 1e-3, 3),                # tie in the middle of the block, tail below the gap
    ([5.0, 3.0, 3.0, 3.0 - 1e-4, 1e-6], 1e-3, 4),          # the block ends before a value below the gap
    ([1.0, 1.0 - 4e-4, 1.0 - 8e-4, 1.0 - 1.2e-3], 1e-3, 4),  # no internal gap; the last value clears zero
    (list(1.0 - 5e-4 * np.arange(2000)), 1e-3, 0),         # values 5e-4 apart down to 5e-4: no gap at all
    ([1.0, 0.75, 0.5], 0.5, 3),                            # a gap exactly at the threshold counts (>=)
    ([1.0, 0.5, 0.25], 0.5, 1),                            # only the first gap reaches 0.5 (exactly)
    ([1.0, 0.9999, 0.5, 0.4999], 1e-3, 4),
    ([1.0, 0.9999, 0.5, 0.4999, 0.0], 1e-3, 4),            # a trailing zero is below every gap
]


@pytest.mark.parametrize("s,gap,kp", GAP_CASES)
def test_gapped_prefix_known_answers(s, gap, kp):
    assert checks.gapped_prefix(np.array(s), gap) == kp


def test_gapped_prefix_brute_force():
    # brute force from the definition: the largest k' with s_k' - s_k'+1 >= gap * s_1
    rng = np.random.default_rng(3)
    for _ in range(200):
        k = int(rng.integers(1, 12))
        s = np.sort(rng.choice([1.0, 0.9995, 0.5, 0.4996, 0.1, 1e-4, 0.0], size=k))[::-1]
        if s[0] == 0:
            continue
        ext = list(s) + [0.0]
        best = 0
        for kp in range(1, k + 1):
            if ext[kp - 1] - ext[kp] >= 1e-3 * s[0]:
                best = kp
        assert checks.gapped_prefix(s, 1e-3) == best


# ---------------------------------------------------------------- sigma_rel_err
def test_sigma_rel_err_relative_and_max():
    ref = np.array([100.0, 10.0, 1.0])
    s = ref * np.array([1 + 1e-7, 1 - 3e-6, 1 + 2e-6])
    assert abs(checks.sigma_rel_err(s, ref) - 3e-6) < 1e-15


def test_sigma_rel_err_floor():
    ref = np.array([1.0, 0.5, 1e-13])          # the last value lies below 1e-12 * s_1: ignored
    s = np.array([1.0, 0.5, 5e-13])
    assert checks.sigma_rel_err(s, ref) == 0.0
    ref2 = np.array([1.0, 0.5, 1e-11])         # above the floor: counted (relative error 1)
    s2 = np.array([1.0, 0.5, 2e-11])
    assert abs(checks.sigma_rel_err(s2, ref2) - 1.0) < 1e-12


def test_sigma_rel_err_small_values_weigh_relatively():
    # an absolute error of 1e-6 on a value of 1e-3 is a relative error of 1e-3
    ref = np.array([1.0, 1e-3])
    s = np.array([1.0, 1e-3 + 1e-6])
    assert abs(checks.sigma_rel_err(s, ref) - 1e-3) < 1e-12


# ---------------------------------------------------------------- planted mistakes
def _sin_frobenius(X, Xr):
    Q, _ = np.linalg.qr(X)
    Qr, _ = np.linalg.qr(Xr)
    return float(np.linalg.norm(Q - Qr @ (Qr.T @ Q)))


def _sin_no_qr(X, Xr):
    return float(np.linalg.norm(X - Xr @ (Xr.T @ X), 2))


def _sin_no_rank_check(X, Xr):
    Q, _ = np.linalg.qr(X)
    Qr, _ = np.linalg.qr(Xr)
    return float(np.linalg.norm(Q - Qr @ (Qr.T @ Q), 2))


def _gap_off_by_one_low(s, rel_gap=1e-3):
    return max(checks.gapped_prefix(s, rel_gap) - 1, 0)


def _gap_no_trailing_zero(s, rel_gap=1e-3):
    s = np.asarray(s, dtype=np.float64)
    for kp in range(s.shape[0] - 1, 0, -1):
        if s[kp - 1] - s[kp] >= rel_gap * s[0]:
            return kp
    return 0


def _gap_strict(s, rel_gap=1e-3):
    ext = np.append(np.asarray(s, dtype=np.float64), 0.0)
    for kp in range(len(s), 0, -1):
        if ext[kp - 1] - ext[kp] > rel_gap * s[0]:
            return kp
    return 0


def _sig_absolute(s, r, floor=1e-12):
    keep = r > floor * r[0]
    return float(np.max(np.abs(s[keep] - r[keep])))


def _sig_no_floor(s, r, floor=1e-12):
    return float(np.max(np.abs(s - r) / r))


def _sin_cases():
    X, Xr = _rot_pair(10, [0.2, 0.3, 0.0])
    X2, Xr2 = _rot_pair(9, [0.05, 0.0, 0.01])
    M = np.array([[2.0, 0.3, -1.0], [0.0, 0.5, 0.7], [1.0, 1.0, 3.0]])
    Xz = X.copy()
    Xz[:, 2] = 0.0
    return [(X, Xr, np.sin(0.3)), (X2 @ M, Xr2, np.sin(0.05)), (Xz, Xr, 1.0)]


@pytest.mark.parametrize("wrong", [_sin_frobenius, _sin_no_qr, _sin_no_rank_check])
def test_planted_sin_angle_mistake_fails_a_pin(wrong):
    cases = _sin_cases()
    assert all(abs(checks.max_sin_angle(X, Xr) - t) < 1e-13 for X, Xr, t in cases)
    assert any(abs(wrong(X, Xr) - t) > 1e-6 for X, Xr, t in cases)


@pytest.mark.parametrize("wrong", [_gap_off_by_one_low, _gap_no_trailing_zero, _gap_strict])
def test_planted_gap_mistake_fails_a_pin(wrong):
    assert any(wrong(np.array(s), g) != kp for s, g, kp in GAP_CASES)


@pytest.mark.parametrize("wrong", [_sig_absolute, _sig_no_floor])
def test_planted_sigma_mistake_fails_a_pin(wrong):
    cases = [(np.array([1.0, 1e-3 + 1e-6]), np.array([1.0, 1e-3]), 1e-3),
             (np.array([1.0, 0.5, 5e-13]), np.array([1.0, 0.5, 1e-13]), 0.0)]
    assert all(abs(checks.sigma_rel_err(s, r) - e) < 1e-12 for s, r, e in cases)
    assert any(abs(wrong(s, r) - e) > 1e-6 for s, r, e in cases)


def test_planted_mistakes_change_a_parity_decision():
    """The rulers as a parity test uses them: a result whose leading block is
    rotated by 1e-3 out of the reference subspace must fail a 1e-4 subspace
    tolerance, and an exact result must pass; each planted ruler gets one of
    the two decisions wrong."""
    rng = np.random.default_rng(11)
    n, k = 40, 6
    Ur, _ = np.linalg.qr(rng.standard_normal((n, k + 1)))
    U_good = Ur[:, :k] @ np.diag([1, -1, 1, 1, -1, 1])                     # signs only
    U_bad = Ur[:, :k].copy()
    U_bad[:, 3] = np.cos(1e-3) * Ur[:, 3] + np.sin(1e-3) * Ur[:, k]        # out of the subspace by 1e-3
    U_scaled = U_good @ np.diag([3.0, 1.0, 0.5, 2.0, 1.0, 7.0])            # unnormalised columns
    assert checks.max_sin_angle(U_good, Ur[:, :k]) < 1e-4
    assert checks.max_sin_angle(U_scaled, Ur[:, :k]) < 1e-4
    assert checks.max_sin_angle(U_bad, Ur[:, :k]) > 1e-4
    U_lost = U_good.copy()
    U_lost[:, 5] = 0.0
    assert checks.max_sin_angle(U_lost, Ur[:, :k]) > 1e-4
    # no orthonormalisation: the rotated block with short columns is wrongly accepted
    assert checks.max_sin_angle(0.01 * U_bad, Ur[:, :k]) > 1e-4
    assert _sin_no_qr(0.01 * U_bad, Ur[:, :k]) < 1e-4
    # no rank check: the QR of a block with a zero column completes it with an arbitrary
    # unit vector, here (coordinate blocks) one inside the reference subspace, and a
    # block that lost a column is wrongly accepted
    E = np.eye(n)[:, :k]
    E_lost = E.copy()
    E_lost[:, 5] = 0.0
    assert checks.max_sin_angle(E_lost, E) == 1.0
    assert _sin_no_rank_check(E_lost, E) < 1e-4
    # gap scan one short: a spectrum with its only gap at the end gives k' = k - 1 and
    # leaves the rotated direction (index k - 1) out of the comparison
    s = np.array([6.0, 5.0, 4.0, 3.0, 2.0, 1.0])
    U_bad_last = Ur[:, :k].copy()
    U_bad_last[:, k - 1] = np.cos(1e-3) * Ur[:, k - 1] + np.sin(1e-3) * Ur[:, k]
    kp = checks.gapped_prefix(s)
    assert kp == k and checks.max_sin_angle(U_bad_last[:, :kp], Ur[:, :kp]) > 1e-4
    kw = _gap_off_by_one_low(s)
    assert checks.max_sin_angle(U_bad_last[:, :kw], Ur[:, :kw]) < 1e-4

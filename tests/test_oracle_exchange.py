"""Pins of the oracle's Adaptive Type Exchange (Sec. 3.2, Eqs. 3-5; App. D,
Eqs. 17-19) against what the paper states.  CPU only."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import native as O

# the permutation matrices as printed in Eq. 5 / App. D
P_X = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], np.float64)
P_Y = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], np.float64)


def rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_erank_values_stated_in_paper():
    # isotropic -> 3 and flattened -> 2 (Sec. 3.2)
    assert abs(O.erank(0.3, 0.3, 0.3) - 3.0) < 1e-12
    assert abs(O.erank(0.0, 0.0, -30.0) - 2.0) < 1e-12
    assert abs(O.erank(0.0, -30.0, -30.0) - 1.0) < 1e-12
    # (1, 1, s_z): rises, then back to 2 near s_z ~ 2.6 (App. D)
    f = lambda s: O.erank(0.0, 0.0, math.log(s)) - 2.0
    root = brentq(f, 1.5, 5.0, xtol=1e-12)
    assert abs(root - 2.6) < 0.05
    vals = [O.erank(0.0, 0.0, math.log(s)) for s in (0.01, 0.3, 1.0)]
    assert vals[0] < vals[1] < vals[2]
    # definition (Eq. 3) written out directly
    rng = np.random.default_rng(0)
    for ls in rng.normal(-3, 1, size=(100, 3)):
        q = np.exp(2 * ls)
        p = q / q.sum()
        assert abs(O.erank(*ls) - math.exp(-(p * np.log(p)).sum())) < 1e-12


def _cov(ls, q):
    R = rot(q)
    return R @ np.diag(np.exp(2 * np.asarray(ls, np.float64))) @ R.T


def test_3d_to_2d_reparameterisation_preserves_covariance():
    rng = np.random.default_rng(1)
    n = 400
    ls = rng.normal(-3, 1, size=(n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    t = np.ones(n, np.uint8)
    ls_o, q_o, t_o, nf = O.exchange(ls, q, t, mode="mask", mask=np.ones(n, np.uint8))
    assert nf == n and np.all(t_o == 0)
    for i in range(n):
        S0 = _cov(ls[i], q[i])
        S1 = _cov(ls_o[i], q_o[i])
        np.testing.assert_allclose(S1, S0, rtol=1e-9, atol=1e-12 * np.abs(S0).max())
        # least significant scale now on z
        assert ls_o[i, 2] <= ls_o[i, 0] and ls_o[i, 2] <= ls_o[i, 1]
        R0, R1 = rot(q[i]), rot(q_o[i])
        assert np.linalg.det(R1) > 0
        # R* = R P^T with P the printed matrix selected by the smallest axis
        if ls[i, 2] <= ls[i, 0] and ls[i, 2] <= ls[i, 1]:
            np.testing.assert_allclose(R1, R0, atol=1e-12)
        elif ls[i, 0] <= ls[i, 1]:
            np.testing.assert_allclose(R1, R0 @ P_X.T, atol=1e-12)
            np.testing.assert_allclose(np.diag(np.exp(ls_o[i])),
                                       P_X @ np.diag(np.exp(ls[i].astype(np.float64))) @ P_X.T, rtol=1e-12)
        else:
            np.testing.assert_allclose(R1, R0 @ P_Y.T, atol=1e-12)
            np.testing.assert_allclose(np.diag(np.exp(ls_o[i])),
                                       P_Y @ np.diag(np.exp(ls[i].astype(np.float64))) @ P_Y.T, rtol=1e-12)
        # quaternion norm preserved (unit p)
        assert abs(np.linalg.norm(q_o[i]) - np.linalg.norm(q[i].astype(np.float64))) < 1e-6


def test_permutations_are_rotations():
    for P in (P_X, P_Y):
        np.testing.assert_allclose(P @ P.T, np.eye(3))
        assert abs(np.linalg.det(P) - 1.0) < 1e-12


def test_2d_to_3d_is_a_flag_flip():
    rng = np.random.default_rng(2)
    n = 50
    ls = rng.normal(-3, 1, size=(n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    t = np.zeros(n, np.uint8)
    ls_o, q_o, t_o, nf = O.exchange(ls, q, t, mode="mask", mask=np.ones(n, np.uint8))
    assert nf == n and np.all(t_o == 1)
    np.testing.assert_array_equal(ls_o, ls.astype(np.float64))
    np.testing.assert_array_equal(q_o, q.astype(np.float64))


@pytest.mark.parametrize("theta", [2.05, 1.9, 2.15])
def test_erank_rule(theta):
    rng = np.random.default_rng(3)
    n = 2000
    ls = rng.normal(-3, 1.0, size=(n, 3)).astype(np.float32)
    t = (rng.random(n) < 0.5).astype(np.uint8)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    ls_o, q_o, t_o, nf = O.exchange(ls, q, t, mode="erank", theta=theta)
    qq = np.exp(2 * ls.astype(np.float64))
    p = qq / qq.sum(1, keepdims=True)
    er = np.exp(-(p * np.log(p)).sum(1))
    want = np.where(t == 1, er < theta, er > theta)
    np.testing.assert_array_equal(t_o != t, want)
    assert nf == want.sum() and 0 < nf < n

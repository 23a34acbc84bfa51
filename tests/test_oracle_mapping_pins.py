"""Pins of the mapping oracle (oracle/mapping.py) to things other than itself.

  * isotropy term: zero for an isotropic Gaussian; sqrt(6) s^2 for scales (s, s, 2s) by hand;
    equal to the Frobenius norm of the deviatoric part of R diag(s^2) R^T built with the
    rasterizer oracle's rotation, for random rotations (the rotation invariance it relies on);
  * psi: 2 log 2 at alpha = 1/2, symmetric in the logit, its derivative 2 alpha - 1;
  * gradients of R against central finite differences (log-scales, logits, means);
  * EMA, counters and the pruning bounds on planted values.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mapping


def test_isotropy_term_closed_forms_and_rotation_invariance():
    s = 0.3
    val, *_ = mapping.regularizer(np.log([[s, s, s]]), [0.0], np.zeros((1, 3)), None, 1.0, 0.0, 0.0)
    assert val == pytest.approx(0.0, abs=1e-15)
    val, *_ = mapping.regularizer(np.log([[s, s, 2 * s]]), [0.0], np.zeros((1, 3)), None, 1.0, 0.0,
                                  0.0)
    assert val == pytest.approx(math.sqrt(6.0) * s * s, rel=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(10):
        ls = rng.normal(-2, 0.5, size=3)
        q = rng.normal(size=4)
        R = oracle.quat_to_rotmat(q[None] / np.linalg.norm(q))[0]
        Sig = R @ np.diag(np.exp(2 * ls)) @ R.T
        ref = np.linalg.norm(Sig - np.trace(Sig) / 3 * np.eye(3), "fro")
        val, *_ = mapping.regularizer(ls[None], [0.0], np.zeros((1, 3)), None, 1.0, 0.0, 0.0)
        assert val == pytest.approx(ref, rel=1e-10)


def test_psi_values_and_derivative():
    val, _, d, _ = mapping.regularizer(np.zeros((1, 3)), [0.0], np.zeros((1, 3)), None, 0.0, 1.0, 0.0)
    assert val == pytest.approx(2 * math.log(2.0)) and d[0] == pytest.approx(0.0)
    a, _, da, _ = mapping.regularizer(np.zeros((2, 3)), [1.7, -1.7], np.zeros((2, 3)), None, 0.0,
                                      1.0, 0.0)
    alpha = 1 / (1 + math.exp(-1.7))
    assert da[0] == pytest.approx(2 * alpha - 1) and da[1] == pytest.approx(-(2 * alpha - 1))
    assert a == pytest.approx(2 * (-math.log(alpha) - math.log(1 - alpha)))


def test_regularizer_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    n = 6
    ls = rng.normal(-2, 0.4, size=(n, 3))
    lg = rng.normal(0, 1.5, size=n)
    mu = rng.normal(size=(n, 3))
    ema = mu + rng.normal(0, 0.1, size=(n, 3))
    lam = (0.7, 0.3, 2.0)
    _, d_ls, d_lg, d_mu = mapping.regularizer(ls, lg, mu, ema, *lam)
    h = 1e-6

    def f(a, b, c):
        return mapping.regularizer(a, b, c, ema, *lam)[0]

    for i in range(n):
        for k in range(3):
            for arr, grad in ((ls, d_ls), (mu, d_mu)):
                p, m = arr.copy(), arr.copy()
                p[i, k] += h
                m[i, k] -= h
                args_p = (p, lg, mu) if arr is ls else (ls, lg, p)
                args_m = (m, lg, mu) if arr is ls else (ls, lg, m)
                assert grad[i, k] == pytest.approx((f(*args_p) - f(*args_m)) / (2 * h), rel=1e-6,
                                                   abs=1e-8)
        p, m = lg.copy(), lg.copy()
        p[i] += h
        m[i] -= h
        assert d_lg[i] == pytest.approx((f(ls, p, mu) - f(ls, m, mu)) / (2 * h), rel=1e-6, abs=1e-8)


def test_ema_counters_and_prune_on_planted_values():
    np.testing.assert_allclose(mapping.ema([[1.0, 2.0, 3.0]], [[0.0, 0.0, 0.0]], 0.25),
                               [[0.25, 0.5, 0.75]])
    obs, vis = mapping.counters([3, 0], [1.0, 0.0], [2, 0], [0.0, 10.0])
    assert list(obs) == [5, 0]
    assert vis[0] == pytest.approx(2.0) and vis[1] == 0.0
    ls = np.log([[0.1, 0.1, 0.1], [0.9, 0.9, 0.9], [0.1, 0.1, 0.1], [0.1, 0.1, 0.1],
                 [0.1, 0.1, 0.1]])
    lg = np.array([0.0, 0.0, -8.0, 0.0, 0.0])
    keep = mapping.prune_mask(ls, lg, [10, 10, 10, 10, 2], [5.0, 5.0, 5.0, 0.5, 0.5])
    # 1: tr = 3 * 0.81 > 1; 2: alpha = 3.4e-4 < 0.005; 3: observed 10 times, score 0.5 < 1;
    # 4: the same score but only 2 observations.
    assert list(keep) == [True, False, False, False, True]

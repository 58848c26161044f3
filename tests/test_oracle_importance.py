"""Pins of oracle.importance: closed forms, special cases and brute force."""
import math

import numpy as np
import pytest

from oracle import importance


def test_equal_likelihoods_give_uniform_weights():
    offs = np.array([0, 5, 5, 17])
    w, ess, eff, lnz = importance.importance_weights(np.full(17, -3.25), offs)
    np.testing.assert_allclose(w[:5], 0.2, rtol=1e-15)
    np.testing.assert_allclose(w[5:], 1.0 / 12.0, rtol=1e-15)
    np.testing.assert_allclose(ess, [5.0, 0.0, 12.0], rtol=1e-15)
    np.testing.assert_allclose(eff, [1.0, 0.0, 1.0], rtol=1e-15)
    assert lnz[1] == -np.inf
    np.testing.assert_allclose(lnz[[0, 2]], -3.25, rtol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 1000])
def test_linear_weights_closed_form(n):
    """w_i = i (i = 1..n): ESS = (n(n+1)/2)^2 / (n(n+1)(2n+1)/6) = 3n(n+1) / (2(2n+1)),
    evidence (1/n) sum i = (n+1)/2, weight_i = 2i / (n(n+1))."""
    i = np.arange(1, n + 1, dtype=np.float64)
    w, ess, eff, lnz = importance.importance_weights(np.log(i), [0, n])
    np.testing.assert_allclose(w, 2.0 * i / (n * (n + 1)), rtol=1e-13)
    np.testing.assert_allclose(ess[0], 3.0 * n * (n + 1) / (2.0 * (2 * n + 1)), rtol=1e-13)
    np.testing.assert_allclose(eff[0], 3.0 * (n + 1) / (2.0 * (2 * n + 1)), rtol=1e-13)
    np.testing.assert_allclose(lnz[0], math.log((n + 1) / 2.0), rtol=1e-13, atol=1e-15)


def test_shift_invariance_and_log_ratio():
    rng = np.random.default_rng(3)
    lnl = rng.normal(-50.0, 4.0, 300)
    offs = [0, 100, 300]
    w0, e0, f0, z0 = importance.importance_weights(lnl, offs)
    w1, e1, f1, z1 = importance.importance_weights(lnl + 1234.5, offs)
    np.testing.assert_allclose(w1, w0, rtol=1e-12)
    np.testing.assert_allclose(e1, e0, rtol=1e-12)
    np.testing.assert_allclose(z1, z0 + 1234.5, rtol=1e-14)
    r = rng.normal(0.0, 1.0, 300)
    w2, _, _, _ = importance.importance_weights(lnl, offs, log_ratio=r)
    w3, _, _, _ = importance.importance_weights(lnl + r, offs)
    np.testing.assert_array_equal(w2, w3)


def test_one_dominant_sample():
    lnl = np.array([0.0, -800.0, -900.0, -1000.0])
    w, ess, eff, lnz = importance.importance_weights(lnl, [0, 4])
    np.testing.assert_allclose(w, [1.0, 0.0, 0.0, 0.0], atol=1e-300)
    assert ess[0] == 1.0 and eff[0] == 0.25
    np.testing.assert_allclose(lnz[0], -math.log(4.0), rtol=1e-15)


def test_minus_infinity_samples():
    lnl = np.array([-np.inf, -2.0, -np.inf, -np.inf, -np.inf])
    w, ess, eff, lnz = importance.importance_weights(lnl, [0, 3, 5])
    np.testing.assert_array_equal(w, [0.0, 1.0, 0.0, 0.0, 0.0])
    np.testing.assert_array_equal(ess, [1.0, 0.0])
    np.testing.assert_allclose(lnz[0], -2.0 - math.log(3.0), rtol=1e-15)
    assert lnz[1] == -np.inf


def test_brute_force_small():
    """Direct sums of exp(ln w) with Python floats (no factoring) on moderate values."""
    rng = np.random.default_rng(11)
    counts = [3, 1, 0, 9, 4]
    offs = np.concatenate([[0], np.cumsum(counts)])
    lnl = rng.uniform(-20.0, 5.0, offs[-1])
    lr = rng.uniform(-1.0, 1.0, offs[-1])
    w, ess, eff, lnz = importance.importance_weights(lnl, offs, log_ratio=lr)
    for e, n in enumerate(counts):
        ws = [math.exp(lnl[s] + lr[s]) for s in range(offs[e], offs[e + 1])]
        if n == 0:
            assert ess[e] == 0.0 and lnz[e] == -np.inf
            continue
        tot = math.fsum(ws)
        np.testing.assert_allclose(w[offs[e]:offs[e + 1]], [x / tot for x in ws], rtol=1e-13)
        np.testing.assert_allclose(ess[e], tot * tot / math.fsum(x * x for x in ws), rtol=1e-13)
        np.testing.assert_allclose(eff[e], ess[e] / n, rtol=1e-15)
        np.testing.assert_allclose(lnz[e], math.log(tot / n), rtol=1e-13)

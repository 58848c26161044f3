"""The Stockham pass plans of the fused simulation pass, in exact FP64 arithmetic (CPU).

A pass of radix R and stride Ns on n points gives butterfly j (j < n/R) the inputs
x[j + r n/R], r < R, multiplies input r by e^{-+2 pi i jm r/(R Ns)} with jm = j mod Ns,
takes their R-point transform and writes output r to x[(j - jm) R + jm + r Ns].  The
forward transform runs the radices of the plan in order with Ns = 1, R_0, R_0 R_1, ...;
the inverse runs them in reverse order.  Plans: radix-16 passes and a short last radix
2^(log2 n mod 4) when log2 n is not a multiple of 4 (16 16 16 2 for n = 2^13), radix-8
passes otherwise (8 8 8 8 for 2^12).  This test runs those plans as stated against
numpy's transforms for every size the kernel is built for, so a wrong slot, stride or
twiddle exponent fails here before any GPU run."""
import numpy as np
import pytest


def _plan(logn):
    if logn % 4:
        return [16] * (logn // 4) + [1 << (logn % 4)]
    rl = {0: 8, 1: 2, 2: 4}[logn % 3]          # n = 8^P rl
    return [8] * ((logn - (rl.bit_length() - 1)) // 3) + [rl]


def _pass(x, R, Ns, sign):
    n = x.size
    nR = n // R
    F = np.exp(sign * 2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    y = np.empty_like(x)
    for j in range(nR):
        jm = j % Ns
        v = x[j + nR * np.arange(R)] * np.exp(sign * 2j * np.pi * jm * np.arange(R) / (R * Ns))
        y[(j - jm) * R + jm + Ns * np.arange(R)] = F @ v
    return y


def _run(x, radices, sign):
    Ns = 1
    for R in radices:
        x = _pass(x, R, Ns, sign)
        Ns *= R
    assert Ns == x.size
    return x


@pytest.mark.parametrize("logn", [9, 10, 11, 12, 13])
def test_plans_compute_the_dft(logn):
    n = 1 << logn
    plan = _plan(logn)
    assert int(np.prod(plan)) == n
    rng = np.random.default_rng(logn)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    fwd = _run(x, plan, -1.0)
    assert np.abs(fwd - np.fft.fft(x)).max() <= 1e-9 * np.sqrt(n)
    inv = _run(fwd, plan[::-1], +1.0)
    assert np.abs(inv / n - x).max() <= 1e-12 * np.sqrt(n)


def test_the_headline_plan_is_16_16_16_2():
    assert _plan(13) == [16, 16, 16, 2]
    assert _plan(12) == [8, 8, 8, 8]
    assert _plan(10) == [16, 16, 4]


def test_a_wrong_twiddle_stride_fails():
    """Planted slip: the twiddle exponent over R Ns replaced by one over Ns alone."""
    n = 1 << 10
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Ns, y = 1, x
    for R in _plan(10):
        nR = n // R
        F = np.exp(-2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
        z = np.empty_like(y)
        for j in range(nR):
            jm = j % Ns
            v = y[j + nR * np.arange(R)] * np.exp(-2j * np.pi * jm * np.arange(R) / Ns)
            z[(j - jm) * R + jm + Ns * np.arange(R)] = F @ v
        y, Ns = z, Ns * R
    assert np.abs(y - np.fft.fft(x)).max() > 1.0

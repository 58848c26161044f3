"""The algebra of the merger-time marginal's transforms, in exact FP64 arithmetic (CPU).

The GPU kernel evaluates, for each sub-grid offset r < u, the grid values
    x(u m + r) = Re sum_{k <= n} c_k e^{2 pi i k (u m + r)/(N u)},   m < n_tc,  N = 2n,
as a complex inverse transform of n points of Z_j = a^j (P_j + e^{-i pi r/u} Q_j) with
r-independent tables P_j = c_j (1 + i conj w^j)/2, Q_j = conj(c_{n-j}) (1 - i conj w^j)/2
(w = e^{-2 pi i/N}, a = e^{2 pi i r/(N u)}), the ramp a^j folded into the twiddle base of
each Stockham pass as a^{n/(R Ns)}, radix-16 passes and a last pass of radix
RS = 2^(log2 n mod 4) (16 when that is 0) evaluated, when only its output 0 is needed, by
Horner's rule.  This test restates that decomposition step by step in numpy and checks it
against the direct sum for every transform size the kernel supports up to 2^12 and both
last-pass forms, so a wrong digit weight, sign or pairing in the reasoning fails here
before any GPU run."""
import numpy as np
import pytest


def _direct(c, u, n_tc, r):
    n = c.size - 1
    N = 2 * n
    m = np.arange(n_tc)
    k = np.arange(n + 1)
    return np.real(np.exp(2j * np.pi * np.outer(u * m + r, k) / (N * u)) @ c)


def _kernel_plan(c, u, n_tc, r, horner):
    n = c.size - 1
    N, logn = 2 * n, int(np.log2(c.size - 1))
    Nu = N * u
    j = np.arange(n)
    w = np.exp(-2j * np.pi * j / N)
    c_nj = np.concatenate([[c[n]], c[n - 1:0:-1]])          # c_{n-j}
    P = c[:n] * (1 + 1j * np.conj(w)) / 2
    Q = np.conj(c_nj) * (1 - 1j * np.conj(w)) / 2
    a = np.exp(2j * np.pi * r / Nu)
    Z = P + np.exp(-1j * np.pi * r / u) * Q                  # without the ramp a^j
    T = n // 16
    RS = 16 if logn % 4 == 0 else 1 << (logn % 4)
    F16 = np.exp(2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)   # inverse DFT, 16 points
    # first pass: radix 16, stride 1, inputs times (a^{n/16})^q; output q of butterfly t at 16 t + q
    x = np.empty(n, complex)
    tw = a ** ((n // 16) * np.arange(16))
    for t in range(T):
        x[16 * t + np.arange(16)] = F16 @ (Z[t + T * np.arange(16)] * tw)
    Ns = 16
    while Ns * RS < n:                                        # middle radix-16 passes
        y = np.empty(n, complex)
        W = n // (16 * Ns)
        for t in range(T):
            jm = t % Ns
            base = np.exp(2j * np.pi * jm / (16 * Ns)) * a ** W
            y[(t - jm) * 16 + jm + Ns * np.arange(16)] = F16 @ (x[t + T * np.arange(16)] * base ** np.arange(16))
        x = y
        Ns *= 16
    assert Ns * RS == n
    NB = n // RS
    out = np.full(n, np.nan + 0j)
    FR = np.exp(2j * np.pi * np.outer(np.arange(RS), np.arange(RS)) / RS)
    for jj in range(NB):
        b = np.exp(2j * np.pi * jj / n) * a                    # weight 1: e^{2 pi i (jj + r/(2u))/n}
        v = x[jj + NB * np.arange(RS)]
        if horner:                                             # output 0 alone
            acc = v[RS - 1]
            for l in range(RS - 2, -1, -1):
                acc = acc * b + v[l]
            out[jj] = acc
        else:
            out[jj + NB * np.arange(RS)] = FR @ (v * b ** np.arange(RS))
    got = np.empty(n_tc)
    got[0::2] = out[:(n_tc + 1) // 2].real
    got[1::2] = out[:n_tc // 2].imag
    return got


@pytest.mark.parametrize("logn,u,n_tc,horner", [
    (7, 4, 64, False),      # last radix 8
    (8, 2, 100, False),     # last radix 16
    (9, 2, 129, False),     # last radix 2
    (10, 4, 512, True),     # last radix 4, output 0 alone (the two-detector workload's window)
    (10, 1, 2048, False),   # the whole window
    (11, 2, 999, False),    # last radix 8 after a middle pass
    (12, 1, 300, False),    # last radix 16 after a middle pass
])
def test_folded_ramp_radix16_plan_equals_the_direct_sum(logn, u, n_tc, horner):
    n = 1 << logn
    rng = np.random.default_rng(logn + 10 * u)
    c = np.zeros(n + 1, complex)
    lo, hi = 3, n - 5                                          # zero at k = 0 and near k = n, as band bins are
    c[lo:hi] = rng.standard_normal(hi - lo) + 1j * rng.standard_normal(hi - lo)
    for r in sorted({0, u // 2, u - 1}):
        ref = _direct(c, u, n_tc, r)
        got = _kernel_plan(c, u, n_tc, r, horner)
        assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref)), (r, np.max(np.abs(got - ref)))


def test_a_wrong_digit_weight_fails():
    """The check is sharp: folding the ramp into the middle pass with the first pass's
    weight instead of its own changes the values."""
    logn, u, n_tc, r = 10, 4, 512, 3
    n = 1 << logn
    rng = np.random.default_rng(5)
    c = np.zeros(n + 1, complex)
    c[3:n - 5] = rng.standard_normal(n - 8) + 1j * rng.standard_normal(n - 8)
    ref = _direct(c, u, n_tc, r)
    # the same plan with a^{n/16} on the middle pass's base (its own weight is n/256)
    N, Nu = 2 * n, 2 * n * u
    a = np.exp(2j * np.pi * r / Nu)
    good = _kernel_plan(c, u, n_tc, r, True)
    assert np.max(np.abs(good - ref)) <= 1e-11 * np.max(np.abs(ref))
    j = np.arange(n)
    w = np.exp(-2j * np.pi * j / N)
    c_nj = np.concatenate([[c[n]], c[n - 1:0:-1]])
    Z = c[:n] * (1 + 1j * np.conj(w)) / 2 + np.exp(-1j * np.pi * r / u) * np.conj(c_nj) * (1 - 1j * np.conj(w)) / 2
    T = n // 16
    F16 = np.exp(2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
    x = np.empty(n, complex)
    for t in range(T):
        x[16 * t + np.arange(16)] = F16 @ (Z[t + T * np.arange(16)] * a ** ((n // 16) * np.arange(16)))
    y = np.empty(n, complex)
    for t in range(T):
        jm = t % 16
        base = np.exp(2j * np.pi * jm / 256) * a ** (n // 16)          # wrong weight
        y[(t - jm) * 16 + jm + 16 * np.arange(16)] = F16 @ (x[t + T * np.arange(16)] * base ** np.arange(16))
    out = np.empty(n // 4, complex)
    for jj in range(n // 4):
        b = np.exp(2j * np.pi * jj / n) * a
        v = y[jj + (n // 4) * np.arange(4)]
        out[jj] = ((v[3] * b + v[2]) * b + v[1]) * b + v[0]
    wrong = np.empty(n_tc)
    wrong[0::2] = out[:n_tc // 2].real
    wrong[1::2] = out[:n_tc // 2].imag
    assert np.max(np.abs(wrong - ref)) > 1e-3 * np.max(np.abs(ref))

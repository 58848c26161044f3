"""The background generator's transform algebra, in exact FP64 arithmetic (CPU).

The coloured background of L samples is made in the frequency domain and brought to the
time domain by one complex inverse transform of n = L/2 points: its spectrum X_k
(k = 0 .. n) is packed as Z_k = E_k + i O_k, E_k = (X_k + conj X_{n-k})/2,
O_k = (X_k - conj X_{n-k}) w^{-k}/2, w = e^{-2 pi i/L} (with X_0 = 0, Z_0 = X_n (1 - i)/2),
so that the inverse transform of Z, divided by n, is x_2m + i x_2m+1 for x = irfft(X).
The inverse transform runs in four steps (Bailey 1990) with n = n1 n2, k = k1 + n1 k2
and m = n2 m1 + m2: pass A forms G[k1][m2] = e^{2 pi i k1 m2/n} sum_k2 e^{2 pi i k2 m2/n2}
Z_k, pass B z_m = sum_k1 e^{2 pi i k1 m1/n1} G[k1][m2].  This test restates both steps
and checks them against numpy, so a wrong index split, twiddle or packing sign fails here
before any GPU run.  The forward counterpart (the likelihood's data rows) unpacks
Z = FFT_n(x_2m + i x_2m+1) into X_k = E + w^k O and X_{n-k} = conj(E - w^k O) with
E = (Z_k + conj Z_{n-k})/2, O = -i (Z_k - conj Z_{n-k})/2."""
import numpy as np
import pytest


def _pack(X):
    n = X.size - 1
    L = 2 * n
    k = np.arange(n)
    Xnk = np.concatenate([[X[n]], X[n - 1:0:-1]])
    w = np.exp(-2j * np.pi / L)
    return (X[:n] + np.conj(Xnk)) / 2 + 1j * (X[:n] - np.conj(Xnk)) * w ** (-k) / 2


def _fourstep_inverse(Z, n1, n2, twiddle_sign=1.0):
    n = n1 * n2
    k1 = np.arange(n1)[:, None]
    k2 = np.arange(n2)[None, :]
    Zk = Z[k1 + n1 * k2]                                    # [k1][k2]
    m2 = np.arange(n2)
    A = np.exp(2j * np.pi * np.outer(np.arange(n2), m2) / n2)   # [k2][m2]
    G = (Zk @ A) * np.exp(twiddle_sign * 2j * np.pi * k1 * m2[None, :] / n)
    m1 = np.arange(n1)
    Bm = np.exp(2j * np.pi * np.outer(m1, np.arange(n1)) / n1)  # [m1][k1]
    zm = Bm @ G                                             # [m1][m2]
    z = np.empty(n, complex)
    z[(n2 * m1[:, None] + m2[None, :]).ravel()] = zm.ravel()
    return z


def _spectrum(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(n + 1) + 1j * rng.standard_normal(n + 1)
    X[0] = 0.0
    X[n] = X[n].real                                        # the Nyquist bin is real
    return X


@pytest.mark.parametrize("n", [16, 256, 4096])
def test_packing_gives_the_real_inverse(n):
    X = _spectrum(n, n)
    x = np.fft.irfft(X, 2 * n)
    z = np.fft.ifft(_pack(X))
    assert np.abs(z.real - x[0::2]).max() < 1e-13 and np.abs(z.imag - x[1::2]).max() < 1e-13


def test_the_first_packed_element():
    X = _spectrum(64, 1)
    Z = _pack(X)
    assert abs(Z[0] - X[64].real * (0.5 - 0.5j)) < 1e-15


@pytest.mark.parametrize("n1,n2", [(4, 8), (32, 16), (512, 256)])
def test_four_steps_are_the_unnormalised_inverse(n1, n2):
    n = n1 * n2
    rng = np.random.default_rng(n)
    Z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = n * np.fft.ifft(Z)
    assert np.abs(_fourstep_inverse(Z, n1, n2) - ref).max() <= 1e-10 * np.sqrt(n) * np.abs(Z).max()


def test_a_wrong_twiddle_sign_fails():
    n1, n2 = 32, 16
    rng = np.random.default_rng(2)
    Z = rng.standard_normal(n1 * n2) + 1j * rng.standard_normal(n1 * n2)
    ref = n1 * n2 * np.fft.ifft(Z)
    assert np.abs(_fourstep_inverse(Z, n1, n2, twiddle_sign=-1.0) - ref).max() > 1.0


@pytest.mark.parametrize("n", [16, 1024])
def test_unpacking_gives_the_real_spectrum(n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(2 * n)
    Z = np.fft.fft(x[0::2] + 1j * x[1::2])
    X = np.fft.rfft(x)
    w = np.exp(-2j * np.pi / (2 * n))
    for k in range(1, n // 2 + 1):
        Znk = Z[(n - k) % n]
        E = (Z[k] + np.conj(Znk)) / 2
        O = -1j * (Z[k] - np.conj(Znk)) / 2
        assert abs(E + w ** k * O - X[k]) < 1e-11 * np.sqrt(n)
        assert abs(np.conj(E - w ** k * O) - X[n - k]) < 1e-11 * np.sqrt(n)

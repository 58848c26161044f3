"""The fused simulation pass's frequency-domain step, in exact FP64 arithmetic (CPU).

The kernel never forms the real spectrum X_k of a window x of N = 2n samples: it
transforms the packed points z_m = x_{2m} + i x_{2m+1} (n-point complex transform Z),
whitens and injects on bin pairs (k, n - k) of Z directly, and inverts with an
unnormalised n-point transform.  With s_k = W_k / n, theta = 2 pi k / N and
(cs, sn) = (cos, sin) theta it sets, for 0 < k < n/2,
  Z'_k  = alpha_k Z_k + i beta conj(Z_nk) + p s_k H_k + q s_nk conj(H_nk),
  Z'_nk = alpha_nk Z_nk + i beta conj(Z_k) + p' s_nk H_nk + q' s_k conj(H_k),
  alpha_k = A - sn Dl, alpha_nk = A + sn Dl, beta = cs Dl, A = (s_k + s_nk)/2,
  Dl = (s_k - s_nk)/2, p = (1 - sn)/2 + i cs/2, q = (1 + sn)/2 - i cs/2, p' = conj(p),
  q' = conj(q);
the bin n/2 becomes s Z + conj(s H), and the DC / Nyquist pair carried in Z_0 becomes
(a x + b y) + i (b x + a y) with a, b = (s_0 +- s_n)/2.  This test restates those
formulas and checks them against numpy's irfft(W (X + H)) for several transform sizes,
so a sign or pairing slip in the derivation fails before any GPU run."""
import numpy as np
import pytest


def _step(x, h_spec, W, beta_sign=1.0, with_q=True):
    N = x.size
    n = N // 2
    z = x[0::2] + 1j * x[1::2]
    Z = np.fft.fft(z)
    s = W / n
    Zp = Z.copy()
    a, b = 0.5 * (s[0] + s[n]), 0.5 * (s[0] - s[n])
    Zp[0] = (a * Z[0].real + b * Z[0].imag) + 1j * (b * Z[0].real + a * Z[0].imag)
    for k in range(1, n // 2):
        nk = n - k
        th = 2 * np.pi * k / N
        cs, sn = np.cos(th), np.sin(th)
        A, Dl = 0.5 * (s[k] + s[nk]), 0.5 * (s[k] - s[nk])
        alk, alnk, be = A - sn * Dl, A + sn * Dl, beta_sign * cs * Dl
        p = 0.5 * (1 - sn) + 0.5j * cs
        q = (0.5 * (1 + sn) - 0.5j * cs) if with_q else 0.0
        hk, hnk = s[k] * h_spec[k], s[nk] * h_spec[nk]
        Zp[k] = alk * Z[k] + 1j * be * np.conj(Z[nk]) + p * hk + q * np.conj(hnk)
        Zp[nk] = alnk * Z[nk] + 1j * be * np.conj(Z[k]) + np.conj(p) * hnk + np.conj(q) * np.conj(hk)
    h2 = n // 2
    Zp[h2] = s[h2] * Z[h2] + np.conj(s[h2] * h_spec[h2])
    y = n * np.fft.ifft(Zp)                     # unnormalised inverse
    out = np.empty(N)
    out[0::2], out[1::2] = y.real, y.imag
    return out


def _case(n, seed):
    rng = np.random.default_rng(seed)
    N = 2 * n
    x = rng.standard_normal(N)
    H = np.fft.rfft(rng.standard_normal(N))
    H[0] = H[n] = 0.0                           # the waveform is zero at DC and Nyquist
    W = rng.uniform(0.2, 3.0, n + 1)
    return x, H, W, np.fft.irfft(W * (np.fft.rfft(x) + H), N)


@pytest.mark.parametrize("n", [8, 64, 1024, 8192])
def test_packed_step_equals_whitening_the_real_spectrum(n):
    x, H, W, ref = _case(n, n)
    got = _step(x, H, W)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("slip", ["beta_sign", "no_q"])
def test_a_slip_in_the_derivation_fails(slip):
    x, H, W, ref = _case(64, 3)
    got = _step(x, H, W, beta_sign=-1.0) if slip == "beta_sign" else _step(x, H, W, with_q=False)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()

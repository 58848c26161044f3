"""Pins for the oracle's noise, Welch, whitening and injection (CPU only)."""
import math

import numpy as np
import pytest
from scipy import signal, stats

from oracle import noise, spectral, taylorf2, detector
from oracle import constants as C
import workloads


def dft(x):
    n = len(x)
    k = np.arange(n)
    return np.exp(-2j * math.pi * np.outer(k, k) / n) @ x


@pytest.mark.parametrize("n", [8, 16, 64, 256])
def test_numpy_fft_matches_brute_force_dft(n):
    x = workloads.random_strain(n, n, 1.0)
    X = dft(x)
    np.testing.assert_allclose(np.fft.rfft(x), X[: n // 2 + 1], atol=1e-11)
    np.testing.assert_allclose(np.fft.irfft(X[: n // 2 + 1], n=n), x, atol=1e-12)
    assert abs(X[0].imag) < 1e-12 and abs(X[n // 2].imag) < 1e-11


def test_aligo_psd_special_values():
    # x = 1: 1e-49 (1 - 5 + 111 * 0.5 / 1.5) = 3.3e-48 ; x = 2: 2^-4.14 - 5/4 + 111 * 5 / 3
    assert abs(noise.aligo_psd(215.0) / 3.3e-48 - 1) < 1e-14
    assert abs(noise.aligo_psd(430.0) / (1e-49 * (2 ** -4.14 - 1.25 + 185.0)) - 1) < 1e-14
    f = np.linspace(5, 4096, 100000)
    assert noise.aligo_psd(f).min() > 0
    np.testing.assert_allclose(noise.noise_psd([3.0, 10.0, 20.0, 50.0], 20.0)[:3], noise.aligo_psd(20.0))


def test_box_muller_normals():
    g_re, g_im = noise.standard_normals(3, 0, 2, 100001)
    for g in (g_re.ravel(), g_im.ravel()):
        assert stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(g_re.ravel(), g_im.ravel())[0, 1]) < 0.01
    assert abs(np.corrcoef(g_re[0], g_re[1])[0, 1]) < 0.01


def test_welch_matches_scipy():
    x = workloads.random_strain(1, (3, 16384), 1e-21)
    for M, stride in ((1024, 512), (4096, 2048), (256, 128), (1000, 500)):
        P = spectral.welch_psd(x, 1024.0, M, stride)
        f, Q = signal.welch(x, fs=1024.0, window="hann", nperseg=M, noverlap=M - stride,
                            detrend=False, scaling="density", average="mean", axis=-1)
        np.testing.assert_allclose(P, Q, rtol=1e-12)


@pytest.mark.parametrize("name,K,spread", [("small", 31, 0.184), ("hl3", 63, 0.129)])
def test_welch_recovers_the_noise_psd(name, K, spread):
    """Welch on the generated background recovers S within the chi-square spread
    of K half-overlapped Hann periodograms (relative std sqrt((1 + 2 rho^2) / K),
    rho = 1/6 for 50 % overlap)."""
    wl = workloads.workload(name)
    n = noise.colored_noise(wl["noise_seed"], 0, len(wl["dets"]), wl["L"], wl["fs"], wl["f_lo"])
    P = spectral.welch_psd(n, wl["fs"], wl["seg_len"], wl["seg_stride"])
    assert (wl["L"] - wl["seg_len"]) // wl["seg_stride"] + 1 == K
    assert abs(math.sqrt((1 + 2 / 36) / K) - spread) < 0.003
    f = np.arange(wl["seg_len"] // 2 + 1) * wl["fs"] / wl["seg_len"]
    band = (f >= 30) & (f < 0.9 * wl["fs"] / 2)
    r = (P / noise.noise_psd(f, wl["f_lo"]))[:, band]
    assert abs(r.mean() - 1) < 5 * spread / math.sqrt(r.size)
    assert abs(r.std() / spread - 1) < 0.1


def test_noise_variance_matches_psd_integral():
    wl = workloads.workload("small")
    L, fs = 1 << 18, wl["fs"]
    n = noise.colored_noise(9, 0, 2, L, fs, wl["f_lo"])
    f = np.arange(L // 2 + 1) * fs / L
    expect = np.sum(noise.noise_psd(f[1:], wl["f_lo"])) * fs / L
    assert abs(n.var() / expect - 1) < 0.05


def test_interp_psd():
    psd = np.array([[1.0, 3.0, 7.0, 15.0, 31.0]])          # seg_len 8 -> 5 bins
    S = spectral.interp_psd(psd, 8, 16)                      # to N = 16 -> 9 bins
    np.testing.assert_allclose(S[0, ::2], psd[0])
    np.testing.assert_allclose(S[0, 1::2], 0.5 * (psd[0, :-1] + psd[0, 1:]))
    lin = np.arange(5.0)[None] * 2 + 1                       # linear PSD: interpolation is exact
    np.testing.assert_allclose(spectral.interp_psd(lin, 8, 32)[0], np.arange(17) * 0.5 + 1)


@pytest.fixture(scope="module")
def whitened_noise():
    wl = workloads.workload("small")
    n = noise.colored_noise(wl["noise_seed"], 5, 2, 64 * wl["N"], wl["fs"], wl["f_lo"])
    d = n.reshape(2, 64, wl["N"]).transpose(1, 0, 2)
    f = np.arange(wl["seg_len"] // 2 + 1) * wl["fs"] / wl["seg_len"]
    true_psd = np.tile(noise.noise_psd(f, wl["f_lo"]), (2, 1))
    return wl, d, true_psd


def test_whitened_noise_has_unit_variance_per_bin(whitened_noise):
    wl, d, S = whitened_noise
    N = wl["N"]
    y = spectral.whiten(d, S, wl["seg_len"], wl["fs"], wl["f_lo"])
    k_lo = math.ceil(wl["f_lo"] * N / wl["fs"])
    K_ret = N // 2 - k_lo
    assert abs(y.var() / (2 * K_ret / N) - 1) < 0.02
    assert abs(2 * K_ret / N - 0.9609375) < 1e-12
    Y = np.fft.rfft(y, axis=-1)
    per_bin = (np.abs(Y[..., k_lo + 100: N // 2]) ** 2 / N).mean()
    assert abs(per_bin - 1) < 0.02


def test_whitening_parseval_linearity_and_inverse(whitened_noise):
    wl, d, S = whitened_noise
    N = wl["N"]
    args = (S, wl["seg_len"], wl["fs"], wl["f_lo"])
    y = spectral.whiten(d, *args)
    Y = np.fft.fft(y, axis=-1)
    np.testing.assert_allclose(np.sum(y ** 2, axis=-1), np.sum(np.abs(Y) ** 2, axis=-1) / N, rtol=1e-12)
    a, b = d[:8], d[8:16] * 0.3
    np.testing.assert_allclose(spectral.whiten(a + b, *args), spectral.whiten(a, *args) + spectral.whiten(b, *args),
                               atol=1e-12 * np.abs(y).max())
    band = spectral.band_mask(N, wl["fs"], wl["f_lo"])
    x_band = np.fft.irfft(np.fft.rfft(d, axis=-1) * band, n=N, axis=-1)
    np.testing.assert_allclose(spectral.unwhiten(y, *args), x_band, atol=1e-12 * np.abs(x_band).max())


def test_injection_energy_parseval():
    """sum s_n^2 / fs equals the continuous Parseval integral 2 sum |h~_k|^2 df."""
    wl = workloads.workload("small")
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    th = workloads.random_theta(2, 4, wl["prior"])
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, N // 2 + 1)
    h = detector.project(hp, hc, th, ["H1", "L1"], 0.0, df)
    zero_bg = np.zeros((2, 3 * N))
    d = spectral.inject(zero_bg, np.array([0, N, 2 * N, 5]), h, N, fs)
    np.testing.assert_allclose(np.sum(d ** 2, axis=-1) / fs, 2 * df * np.sum(np.abs(h) ** 2, axis=-1), rtol=1e-10)
    bg = workloads.random_strain(4, (2, 3 * N))
    d2 = spectral.inject(bg, np.array([0, N, 2 * N, 5]), h, N, fs)
    np.testing.assert_allclose(d2[3] - d[3], bg[:, 5:5 + N], atol=1e-30)

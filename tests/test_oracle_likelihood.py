"""Pins for the oracle's inner product, log-likelihood and mismatch (CPU only)."""
import math

import numpy as np
from scipy import integrate

from oracle import likelihood, noise, spectral, taylorf2, detector
from oracle import constants as C
import workloads


def test_optimal_snr_matches_quadrature():
    """<h,h> on the grid against 4 int A(f)^2 / S(f) df by adaptive quadrature."""
    m1 = m2 = 12.0
    th = np.zeros((C.P, 1))
    th[C.M1], th[C.M2], th[C.DIST] = m1, m2, 400.0
    df, F, f_lo = 1.0 / 64.0, 64 * 1024 + 1, 20.0
    hp, _ = taylorf2.generate_waveforms(th, f_lo, df, F)
    f = np.arange(F) * df
    S = noise.aligo_psd(np.maximum(f, 1.0))
    on = np.nonzero(hp[0])[0]
    snr2 = likelihood.inner_product(hp, hp, S, df, on[0], on[-1] + 1)[0]
    Mc = (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2 * C.MTSUN_S
    D = 400.0 * C.MPC_M / C.C_MS
    amp2 = lambda x: (5 / 24) * math.pi ** (-4 / 3) * Mc ** (5 / 3) * x ** (-7 / 3) / D ** 2
    ref, _ = integrate.quad(lambda x: 4 * amp2(x) / noise.aligo_psd(x), on[0] * df, (on[-1] + 1) * df, limit=200)
    assert abs(snr2 / ref - 1) < 2e-3


def test_mismatch_closed_form():
    wl = workloads.workload("small")
    df = wl["fs"] / wl["N"]
    F = wl["N"] // 2 + 1
    th = workloads.random_theta(8, 2, wl["prior"])
    hp, _ = taylorf2.generate_waveforms(th, wl["f_lo"], df, F)
    S = noise.aligo_psd(np.maximum(np.arange(F) * df, 1.0))
    assert abs(likelihood.mismatch(hp, hp, S, df, 40, F - 1)).max() < 1e-14
    for delta in (1e-3, 0.2, 1.0):
        mm = likelihood.mismatch(hp, hp * np.exp(1j * delta), S, df, 40, F - 1)
        np.testing.assert_allclose(mm, 1 - math.cos(delta), rtol=1e-10, atol=1e-16)


def _events(wl, E, seed, with_noise=True):
    """E events; each background window is its own periodic N-sample stretch, so its
    DFT bins are exactly independent Gaussians of variance N fs S / 2."""
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    dets = wl["dets"]
    th = workloads.random_theta(seed, E, wl["prior"])
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, N // 2 + 1)
    h = detector.project(hp, hc, th, dets, 0.0, df)
    if with_noise:
        bg = np.concatenate([noise.colored_noise(seed, e, len(dets), N, fs, wl["f_lo"]) for e in range(E)], axis=1)
    else:
        bg = np.zeros((len(dets), E * N))
    d = spectral.inject(bg, np.arange(E) * N, h, N, fs)
    f = np.arange(wl["seg_len"] // 2 + 1) * fs / wl["seg_len"]
    psd = np.tile(noise.noise_psd(f, wl["f_lo"]), (len(dets), 1))
    return th, h, d, psd


def test_log_likelihood_at_truth_noise_free_is_zero():
    wl = workloads.workload("small")
    th, h, d, psd = _events(wl, 4, 11, with_noise=False)
    y = spectral.whiten(d, psd, wl["seg_len"], wl["fs"], wl["f_lo"])
    lnl = likelihood.log_likelihood(y, psd, wl["seg_len"], wl["fs"], wl["f_lo"], th, np.arange(5), wl["dets"])
    th_other = th[:, ::-1].copy()
    lnl_wrong = likelihood.log_likelihood(y, psd, wl["seg_len"], wl["fs"], wl["f_lo"], th_other, np.arange(5),
                                          wl["dets"])
    assert np.abs(lnl).max() < 1e-9 * np.abs(lnl_wrong).max()
    assert np.all(lnl_wrong < -1.0)


def test_log_likelihood_equals_standard_inner_product():
    wl = workloads.workload("small")
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    th, h, d, psd = _events(wl, 3, 12)
    y = spectral.whiten(d, psd, wl["seg_len"], fs, wl["f_lo"])
    th2 = workloads.random_theta(99, 3, wl["prior"])
    lnl = likelihood.log_likelihood(y, psd, wl["seg_len"], fs, wl["f_lo"], th2, np.arange(4), wl["dets"])
    hp, hc = taylorf2.generate_waveforms(th2, wl["f_lo"], df, N // 2 + 1)
    h2 = detector.project(hp, hc, th2, wl["dets"], 0.0, df)
    S = spectral.interp_psd(psd, wl["seg_len"], N)
    k_lo = math.ceil(wl["f_lo"] / df)
    for e in range(3):
        r = np.fft.rfft(d[e], axis=-1) / fs - h2[e]
        ref = -0.5 * np.sum(likelihood.inner_product(r, r, S, df, k_lo, N // 2))
        assert abs(lnl[e] - ref) < 1e-9 * abs(ref)


def test_log_likelihood_at_truth_is_chi_square():
    """-2 ln L(theta_true) on noisy data ~ chi^2 with 2 K_ret D degrees of freedom."""
    wl = workloads.workload("small")
    E = 48
    th, h, d, psd = _events(wl, E, 13)
    y = spectral.whiten(d, psd, wl["seg_len"], wl["fs"], wl["f_lo"])
    lnl = likelihood.log_likelihood(y, psd, wl["seg_len"], wl["fs"], wl["f_lo"], th, np.arange(E + 1), wl["dets"])
    k_lo = math.ceil(wl["f_lo"] * wl["N"] / wl["fs"])
    dof = 2 * (wl["N"] // 2 - k_lo) * len(wl["dets"])
    x = -2 * lnl
    assert abs(x.mean() - dof) < 5 * math.sqrt(2 * dof / E)
    assert abs(x.var() / (2 * dof) - 1) < 5 * math.sqrt(2 / (E - 1))


def test_ragged_events_and_empty_events():
    wl = workloads.workload("small")
    th, h, d, psd = _events(wl, 3, 14)
    y = spectral.whiten(d, psd, wl["seg_len"], wl["fs"], wl["f_lo"])
    samples = workloads.random_theta(5, 7, wl["prior"])
    offs = np.array([0, 0, 4, 7])
    lnl = likelihood.log_likelihood(y, psd, wl["seg_len"], wl["fs"], wl["f_lo"], samples, offs, wl["dets"])
    one = likelihood.log_likelihood(y[1:2], psd, wl["seg_len"], wl["fs"], wl["f_lo"], samples[:, :4],
                                    np.array([0, 4]), wl["dets"])
    np.testing.assert_allclose(lnl[:4], one, rtol=1e-14)

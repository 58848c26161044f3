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


# ---------------------------------------------------------------- merger-time marginal
def _noisy_case(E=2, S_per=3, seed=21):
    wl = workloads.workload("small")
    th, h, d, psd = _events(wl, E, seed)
    y = spectral.whiten(d, psd, wl["seg_len"], wl["fs"], wl["f_lo"])
    samples = workloads.random_theta(seed + 1, E * S_per, wl["prior"])
    # half of the samples near their event's source, so that the grid sum has a sharp peak
    for e in range(E):
        samples[:, e * S_per] = th[:, e]
        samples[C.DIST, e * S_per] *= 1.1
    offs = np.arange(E + 1) * S_per
    return wl, th, y, psd, samples, offs


def test_tmarg_is_the_log_mean_exp_of_the_likelihood_on_the_grid():
    """Brute force: ln L at every grid time from log_likelihood (tc in the parameter
    vector), then ln of their mean -- no phase-rotation identity involved."""
    wl, th, y, psd, samples, offs = _noisy_case()
    fs = wl["fs"]
    tc_lo, n_tc, u = 1.1, 6, 2
    got = likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], samples, offs, wl["dets"],
                                          tc_lo, n_tc, u)
    grid = []
    for j in range(u * n_tc):
        s = samples.copy()
        s[C.TC] = tc_lo + j / (u * fs)
        grid.append(likelihood.log_likelihood(y, psd, wl["seg_len"], fs, wl["f_lo"], s, offs, wl["dets"]))
    grid = np.array(grid)
    mx = grid.max(axis=0)
    ref = mx + np.log(np.mean(np.exp(grid - mx), axis=0))
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-9)
    # the tc row of theta is not used
    s2 = samples.copy()
    s2[C.TC] = 123.0
    np.testing.assert_array_equal(
        likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], s2, offs, wl["dets"], tc_lo, n_tc, u),
        got)


def test_tmarg_single_grid_point_and_silent_template():
    wl, th, y, psd, samples, offs = _noisy_case(seed=31)
    fs = wl["fs"]
    one = likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], samples, offs, wl["dets"],
                                          1.3, 1, 1)
    s = samples.copy()
    s[C.TC] = 1.3
    ref = likelihood.log_likelihood(y, psd, wl["seg_len"], fs, wl["f_lo"], s, offs, wl["dets"])
    np.testing.assert_allclose(one, ref, rtol=1e-12)
    # a template of vanishing amplitude: every grid point gives -|Y|^2 / N
    far = samples.copy()
    far[C.DIST] = 1e30
    got = likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], far, offs, wl["dets"], 1.0, 512, 16)
    k_lo = math.ceil(wl["f_lo"] * wl["N"] / fs)
    Y = np.fft.rfft(y, axis=-1)[..., k_lo:wl["N"] // 2]
    yy = np.sum(np.abs(Y) ** 2, axis=(1, 2)) / wl["N"]
    np.testing.assert_allclose(got, -np.repeat(yy, 3), rtol=1e-12)


def test_tmarg_invariant_under_a_circular_shift_of_data_and_window():
    """Shifting the data by s samples (circularly) and the window by s / fs leaves the
    marginal unchanged: fixes the sign and scale of the time in the phase rotation."""
    wl, th, y, psd, samples, offs = _noisy_case(seed=41)
    fs = wl["fs"]
    a = likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], samples, offs, wl["dets"],
                                        1.0, 64, 4)
    for sh in (37, -200):
        b = likelihood.log_likelihood_tmarg(np.roll(y, sh, axis=-1), psd, wl["seg_len"], fs, wl["f_lo"], samples,
                                            offs, wl["dets"], 1.0 + sh / fs, 64, 4)
        np.testing.assert_allclose(b, a, rtol=1e-11, atol=1e-8)


def test_tmarg_laplace_limit_of_a_loud_noise_free_signal():
    """Noise-free data, template at the truth, merger well inside the window: for a loud
    signal the grid sum tends to the Gaussian integral of the merger-time peak,
    ln L_m -> ln( sqrt(2 pi) sigma / (n_tc / fs) ), 1 / sigma^2 = (2 pi)^2 <f h, f h>
    (second-order expansion of <h(t) - h(t*), h(t) - h(t*)> about the truth)."""
    wl = workloads.workload("small")
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    dets = wl["dets"]
    th = np.zeros((C.P, 1))
    th[C.M1], th[C.M2], th[C.DIST], th[C.TC] = 14.0, 11.0, 100.0, 1.2468
    th[C.THETAJN], th[C.PSI], th[C.RA], th[C.DEC], th[C.PHIC] = 0.4, 0.3, 1.1, 0.2, 0.7
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, N // 2 + 1)
    h = detector.project(hp, hc, th, dets, 0.0, df)
    d = spectral.inject(np.zeros((len(dets), N)), np.array([0]), h, N, fs)
    f = np.arange(wl["seg_len"] // 2 + 1) * fs / wl["seg_len"]
    psd = np.tile(noise.noise_psd(f, wl["f_lo"]), (len(dets), 1))
    y = spectral.whiten(d, psd, wl["seg_len"], fs, wl["f_lo"])
    S = spectral.interp_psd(psd, wl["seg_len"], N)
    k_lo = math.ceil(wl["f_lo"] / df)
    fk = np.arange(N // 2 + 1) * df
    rho2 = np.sum(likelihood.inner_product(h[0], h[0], S, df, k_lo, N // 2))
    ff = np.sum(likelihood.inner_product(fk * h[0], fk * h[0], S, df, k_lo, N // 2))
    assert rho2 > 150.0 ** 2                       # loud: the expansion's error is O(1 / rho^2)
    sigma = 1.0 / (2.0 * math.pi * math.sqrt(ff))
    n_tc, u = 64, 128                              # window [1.22, 1.2825) s, grid 7.6 us < sigma
    ref = math.log(math.sqrt(2.0 * math.pi) * sigma / (n_tc / fs))
    got = likelihood.log_likelihood_tmarg(y, psd, wl["seg_len"], fs, wl["f_lo"], th, np.array([0, 1]), dets,
                                          1.22, n_tc, u)[0]
    assert abs(got - ref) < 1e-4, (got, ref)

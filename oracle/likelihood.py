"""Noise-weighted inner product, log-likelihood and mismatch (oracle; test infrastructure).

Sec. 6 (Fig. 5 caption) compares with nested sampling under the usual GW
likelihood: Gaussian stationary noise with one-sided PSD S gives

    <a, b> = 4 df Re sum_k a~_k conj(b~_k) / S_k,     ln L = -1/2 <d - h, d - h>

over the analysis band (k_lo <= k < N/2) and without the normalisation constant
(reading).  a~ is the continuous Fourier transform, a~_k = rfft(a)_k / fs.

For whitened data Y_k = rfft(d)_k M_k / sqrt(S~_k fs/2) the same inner product
is (2/N) Re sum Y_a conj(Y_b), so the log-likelihood of a whitened window y
against a template h_det (continuous FT per detector) is

    ln L = -(1/N) sum_d sum_{band} |rfft(y_d)_k - fs h_det,d(f_k) W_d,k|^2,

W = M / sqrt(S~ fs / 2) the whitening filter.  Readings: tc and spins are taken
from the sample's parameter vector; one PSD (the whitening PSD) for all events.

Sec. 5 leaves the coalescence time out of the estimated parameters: it is
marginalised over.  ``log_likelihood_tmarg`` states that marginal for the judge of
the flow's samples: with tc uniform over the window [tc_lo, tc_lo + n_tc / fs) of
the prior,

    ln L_m(theta) = ln( (1/J) sum_{j<J} exp ln L(theta, tc = tc_lo + j delta) ),
    delta = 1 / (u fs),  J = u n_tc,

the rectangle rule for (1/(n_tc/fs)) int exp ln L dtc on a grid u times finer than
the sampling interval (reading: the paper does not say how tc is integrated out;
the grid spacing u is an argument).  A time shift only rotates the template's
phase, H(tc) = H(0) e^{-2 pi i f tc}, so with c_k = sum_d Y_d,k conj(fs h_d,k W_d,k)
(template at tc = 0)

    ln L(theta, tc) = -(1/N) [ sum |Y|^2 + sum |fs h W|^2 ] + (2/N) Re sum_k c_k e^{2 pi i k tc / T}.
"""
import math
import numpy as np

from . import constants as C
from . import spectral
from . import taylorf2
from . import detector


def inner_product(a_fd, b_fd, S, df, k_lo, k_hi):
    """<a, b> for continuous-FT arrays over bins k_lo <= k < k_hi (last axis)."""
    sl = slice(k_lo, k_hi)
    return 4.0 * df * np.real(np.sum(a_fd[..., sl] * np.conj(b_fd[..., sl]) / S[..., sl], axis=-1))


def mismatch(h1, h2, S, df, k_lo, k_hi):
    """1 - <h1,h2> / sqrt(<h1,h1><h2,h2>), not maximised over time or phase."""
    o12 = inner_product(h1, h2, S, df, k_lo, k_hi)
    o11 = inner_product(h1, h1, S, df, k_lo, k_hi)
    o22 = inner_product(h2, h2, S, df, k_lo, k_hi)
    return 1.0 - o12 / np.sqrt(o11 * o22)


def log_likelihood(y_data, psd, seg_len, fs, f_lo, theta, event_offsets, dets, gmst=0.0, pn_order=7):
    """ln L [S] for samples theta [P][S], sample s belonging to event e when
    event_offsets[e] <= s < event_offsets[e+1]; y_data [E][D][N] whitened windows."""
    y_data = np.asarray(y_data, dtype=np.float64)
    E, D, N = y_data.shape
    F = N // 2 + 1
    df = fs / N
    W = spectral.whitening_filter(psd, seg_len, fs, f_lo, N)
    band = spectral.band_mask(N, fs, f_lo) > 0
    S_total = int(event_offsets[-1])
    out = np.zeros(S_total)
    for e in range(E):
        s0, s1 = int(event_offsets[e]), int(event_offsets[e + 1])
        if s1 == s0:
            continue
        th = np.asarray(theta)[:, s0:s1]
        Y = np.fft.rfft(y_data[e], axis=-1)                      # [D][F]
        hp, hc = taylorf2.generate_waveforms(th, f_lo, df, F, pn_order)
        h = detector.project(hp, hc, th, dets, gmst, df)         # [S][D][F]
        R = Y[None] - fs * h * W[None]
        out[s0:s1] = -np.sum(np.abs(R[..., band]) ** 2, axis=(1, 2)) / N
    return out


def log_likelihood_tmarg(y_data, psd, seg_len, fs, f_lo, theta, event_offsets, dets, tc_lo, n_tc, oversample,
                         gmst=0.0, pn_order=7):
    """Marginal of ln L over a uniform merger time (module docstring), [S]; the tc row of
    theta is not used.  Grid t_j = tc_lo + j / (oversample fs), j < oversample n_tc."""
    y_data = np.asarray(y_data, dtype=np.float64)
    E, D, N = y_data.shape
    F = N // 2 + 1
    df = fs / N
    T = N / fs
    W = spectral.whitening_filter(psd, seg_len, fs, f_lo, N)
    band = spectral.band_mask(N, fs, f_lo) > 0
    kb = np.nonzero(band)[0]
    J = int(oversample) * int(n_tc)
    t = tc_lo + np.arange(J) / (oversample * fs)
    phase = np.exp(2j * np.pi * np.outer(t, kb) / T)              # [J][band]: e^{2 pi i k t_j / T}
    S_total = int(event_offsets[-1])
    out = np.zeros(S_total)
    for e in range(E):
        s0, s1 = int(event_offsets[e]), int(event_offsets[e + 1])
        if s1 == s0:
            continue
        th = np.array(np.asarray(theta)[:, s0:s1], dtype=np.float64)
        th[C.TC] = 0.0                                             # template at tc = 0
        Y = np.fft.rfft(y_data[e], axis=-1)                        # [D][F]
        hp, hc = taylorf2.generate_waveforms(th, f_lo, df, F, pn_order)
        G = fs * detector.project(hp, hc, th, dets, gmst, df) * W[None]   # [S][D][F]
        c = np.sum(Y[None][..., kb] * np.conj(G[..., kb]), axis=1)       # [S][band]
        base = -(np.sum(np.abs(Y[:, kb]) ** 2) + np.sum(np.abs(G[..., kb]) ** 2, axis=(1, 2))) / N
        lnl_t = base[:, None] + (2.0 / N) * np.real(c @ phase.T)        # [S][J]: ln L at each grid time
        mx = lnl_t.max(axis=1)
        out[s0:s1] = mx + np.log(np.mean(np.exp(lnl_t - mx[:, None]), axis=1))
    return out

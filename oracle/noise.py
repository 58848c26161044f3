"""Analytic aLIGO PSD and coloured Gaussian background (oracle; test infrastructure).

Sec. 3.2 trains on a real two-detector background chunk held in GPU memory.
That data is not available here, so seeded coloured Gaussian noise stands in
for it, drawn from the analytic aLIGO design fit

    S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)],  x = f / 215 Hz.

Definition of one background stretch of L samples at rate fs per detector d
(one-sided PSD S_g(f) = S(max(f, f_lo)), flattened below f_lo so that Hann
leakage from the steep low-frequency wall stays out of the analysis band):

    X_0 = 0
    X_k = sqrt(L fs S_g(f_k) / 4) (g_re + i g_im),   0 < k < L/2
    X_{L/2} = sqrt(L fs S_g(f_{L/2}) / 2) g_re
    n = irfft(X)                                       (numpy normalisation, 1/L)

so that E|X_k|^2 = L fs S_g / 2, the DFT of a stationary process with one-sided
density S_g.  The standard normals come from the Box-Muller transform of
Philox words: bins 2j and 2j+1 of detector d use counter (j, d, TAG_NOISE, step);
bin 2j takes words (0, 1), bin 2j+1 words (2, 3), each pair mapped to
uniforms u1, u2 on the 2^-24 grid, g_re = r cos(2 pi u2), g_im = r sin(2 pi u2),
r = sqrt(-2 ln u1).
"""
import math
import numpy as np

from .philox import TAG_NOISE, key_of, philox4x32_10, uniform24


def aligo_psd(f):
    """Analytic aLIGO design one-sided PSD [1/Hz]."""
    x = np.asarray(f, dtype=np.float64) / 215.0
    return 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))


def noise_psd(f, f_lo):
    """The PSD the background is drawn from: S(max(f, f_lo))."""
    return aligo_psd(np.maximum(np.asarray(f, dtype=np.float64), f_lo))


def standard_normals(seed, step, D, K):
    """(g_re, g_im) [D][K] for bins 0..K-1 of each detector (Box-Muller on Philox words)."""
    k0, k1 = key_of(seed)
    J = (K + 1) // 2
    j = np.arange(J, dtype=np.uint64).astype(np.uint32)
    g_re = np.empty((D, 2 * J))
    g_im = np.empty((D, 2 * J))
    for d in range(D):
        w = philox4x32_10(j, np.uint32(d), np.uint32(TAG_NOISE), np.uint32(step & 0xFFFFFFFF), k0, k1)
        for half, (a, b) in enumerate(((w[0], w[1]), (w[2], w[3]))):
            u1 = uniform24(a)
            u2 = uniform24(b)
            r = np.sqrt(-2.0 * np.log(u1))
            g_re[d, half::2] = r * np.cos(2.0 * math.pi * u2)
            g_im[d, half::2] = r * np.sin(2.0 * math.pi * u2)
    return g_re[:, :K], g_im[:, :K]


def colored_noise(seed, step, D, L, fs, f_lo):
    """Background stretch n [D][L] float64 (definition in the module docstring). L even."""
    assert L % 2 == 0
    K = L // 2 + 1
    g_re, g_im = standard_normals(seed, step, D, K)
    f = np.arange(K, dtype=np.float64) * fs / L
    S = noise_psd(f, f_lo)
    sigma = np.sqrt(L * fs * S / 4.0)
    X = sigma[None, :] * (g_re + 1j * g_im)
    X[:, 0] = 0.0
    X[:, -1] = math.sqrt(2.0) * sigma[-1] * g_re[:, -1]
    return np.fft.irfft(X, n=L, axis=-1)

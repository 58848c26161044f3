"""Welch PSD, PSD interpolation, injection and whitening (oracle; test infrastructure).

Sec. 3.2: the PSD is estimated from a background chunk, N crops of the window
length are taken from that chunk, the signals are injected into them and the batch
is whitened with the estimated spectrum, with the transforms, the spectral estimate
and the whitening all run on the accelerator.  The paper gives no formulas; these
are the textbook definitions, with the readings listed per function.

Welch (P. D. Welch 1967), one-sided density, mean of K periodograms:
    P_k = c_k / (fs sum_n w_n^2) (1/K) sum_s |sum_n w_n x_{s*stride+n} e^{-2 pi i k n/M}|^2
with w the periodic Hann window, c_k = 1 at DC and at Nyquist and 2 elsewhere.
Readings: no detrending, mean (not median) average.

Whitening of a window d of N samples, Delta f = fs/N, k_lo = ceil(f_lo/Delta f):
    Y_k = rfft(d)_k M_k / sqrt(S~_k fs / 2),   y = irfft(Y)
with M_k = 1 for k_lo <= k < N/2, else 0, and S~ the Welch estimate linearly
interpolated from its grid (fs/M) to f_k.  Readings: no taper, no
inverse-spectrum truncation.

Injection (circular window, "Definition A"): the frequency-domain detector
strain h_det(f) is a continuous Fourier transform, so its DFT on the window is
fs * h_det(f_k) and
    d = n[off : off + N] + irfft(fs h_det)
with one crop offset per draw shared by all detectors.
"""
import math
import numpy as np


def hann_periodic(M):
    n = np.arange(M, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * n / M)


def welch_psd(x, fs, seg_len, stride):
    """P [D][seg_len/2+1] float64 from x [D][L] (definition in the module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    D, L = x.shape
    M = seg_len
    K = (L - M) // stride + 1
    w = hann_periodic(M)
    acc = np.zeros((D, M // 2 + 1))
    for s in range(K):
        seg = x[:, s * stride: s * stride + M] * w[None, :]
        acc += np.abs(np.fft.rfft(seg, axis=-1)) ** 2
    P = acc / K / (fs * np.sum(w ** 2))
    P[:, 1:] *= 2.0
    if M % 2 == 0:
        P[:, -1] /= 2.0
    return P


def interp_psd(psd, seg_len, N):
    """S~ [D][N/2+1]: psd on the grid fs/seg_len, linearly interpolated to fs/N.

    Bin k sits at position k * seg_len / N on the Welch grid; the fractional part
    is the exact rational (k * seg_len mod N) / N.
    """
    psd = np.asarray(psd, dtype=np.float64)
    k = np.arange(N // 2 + 1, dtype=np.int64)
    num = k * seg_len
    j0 = num // N
    frac = (num % N).astype(np.float64) / N
    j1 = np.minimum(j0 + 1, psd.shape[-1] - 1)
    return psd[:, j0] + (psd[:, j1] - psd[:, j0]) * frac[None, :]


def band_mask(N, fs, f_lo):
    """M_k [N/2+1]: 1 for ceil(f_lo / (fs/N)) <= k < N/2, else 0."""
    k_lo = math.ceil(f_lo / (fs / N))
    k = np.arange(N // 2 + 1)
    return ((k >= k_lo) & (k < N // 2)).astype(np.float64)


def whitening_filter(psd, seg_len, fs, f_lo, N):
    """W [D][N/2+1] = M_k / sqrt(S~_k fs / 2)."""
    S = interp_psd(psd, seg_len, N)
    M = band_mask(N, fs, f_lo)
    W = np.zeros_like(S)
    on = M > 0
    W[:, on] = 1.0 / np.sqrt(S[:, on] * fs / 2.0)
    return W


def whiten(d, psd, seg_len, fs, f_lo):
    """y [B][D][N] from d [B][D][N] (definition in the module docstring)."""
    d = np.asarray(d, dtype=np.float64)
    N = d.shape[-1]
    W = whitening_filter(psd, seg_len, fs, f_lo, N)
    return np.fft.irfft(np.fft.rfft(d, axis=-1) * W, n=N, axis=-1)


def unwhiten(y, psd, seg_len, fs, f_lo):
    """Inverse of whiten on the band: irfft(rfft(y) M_k sqrt(S~_k fs / 2))."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[-1]
    S = interp_psd(psd, seg_len, N)
    M = band_mask(N, fs, f_lo)
    return np.fft.irfft(np.fft.rfft(y, axis=-1) * M * np.sqrt(S * fs / 2.0), n=N, axis=-1)


def crop(noise, offsets, N):
    """n_crop [B][D][N]: noise[:, off_b : off_b + N] for each draw b."""
    noise = np.asarray(noise, dtype=np.float64)
    return np.stack([noise[:, o:o + N] for o in np.asarray(offsets)]) if len(offsets) else \
        np.zeros((0, noise.shape[0], N))


def inject(noise, offsets, h_det, N, fs):
    """d [B][D][N] = crop + irfft(fs h_det) (definition in the module docstring)."""
    sig = np.fft.irfft(fs * np.asarray(h_det), n=N, axis=-1)
    return crop(noise, offsets, N) + sig

"""One whole per-batch pass, step by step and unfused (oracle; test infrastructure).

Sec. 3.2 lists the on-the-fly workflow: a background chunk resident on the
device with its power spectrum fitted once, then per batch: draw N prior
points, generate their waveforms, inject them into N lazily cropped background
windows and whiten the batch with the estimated spectrum.  Here the background
is the seeded coloured-noise stand-in (``noise.colored_noise``), and every
batch gets a fresh background (noise counter = step).

Steps, in the paper's order:
    A4 background    n     = colored_noise(noise_seed, step)       [D][L]
    A5 Welch         S     = welch_psd(n)                          [D][M/2+1]
    A1 prior         theta, offsets = sample_prior(param_seed, step)
    A2 waveform      h+, hx = generate_waveforms(theta)            (tc = 0)
    A3 projection    h_det = project(h+, hx, theta)                (tc + delay)
    A6 injection     d     = crop(n, offsets) + irfft(fs h_det)
    A7 whitening     y     = whiten(d, S)
"""
import numpy as np

from . import constants as C
from .prior import sample_prior
from .taylorf2 import generate_waveforms
from .detector import project
from .noise import colored_noise
from .spectral import crop, welch_psd, inject, whiten


def background(wl, step):
    """(noise [D][L], psd [D][M/2+1]) of one step's background."""
    n = colored_noise(wl["noise_seed"], step, len(wl["dets"]), wl["L"], wl["fs"], wl["f_lo"])
    S = welch_psd(n, wl["fs"], wl["seg_len"], wl["seg_stride"])
    return n, S


def simulate_batch(wl, step, draws=None, bg=None):
    """Whitened batch for workload ``wl`` at ``step``.

    Returns dict with y [b][D][N] (for the selected draws), theta [P][B],
    offsets [B], noise, psd.  ``draws`` selects a subset of draw indices (all by
    default); theta and offsets are always returned for the whole batch.
    """
    N = wl["N"]
    fs = wl["fs"]
    df = fs / N
    F = N // 2 + 1
    noise, psd = bg if bg is not None else background(wl, step)
    theta, offsets = sample_prior(wl["prior"], wl["param_seed"], step, wl["B"], wl["L"], N)
    sel = np.arange(wl["B"]) if draws is None else np.asarray(draws, dtype=np.int64)
    th = theta[:, sel]
    hp, hc = generate_waveforms(th, wl["f_lo"], df, F)
    h = project(hp, hc, th, wl["dets"], wl.get("gmst", 0.0), df)
    d = inject(noise, offsets[sel], h, N, fs)
    y = whiten(d, psd, wl["seg_len"], fs, wl["f_lo"])
    return {"y": y, "theta": theta, "offsets": offsets, "noise": noise, "psd": psd, "draws": sel}


def simulate_batch_padded(wl, step, N_pad, draws=None, bg=None):
    """Definition B (padded grid): the waveform is evaluated on the grid of a padded
    segment of N_pad >= N samples, f_k = k fs / N_pad, projected with the draw's own tc and
    delays, inverse-transformed over the whole padded segment, and its first N samples
    are injected:  d = crop(n, offsets) + irfft_{N_pad}(fs h_det)[:N],  y = whiten(d, S).
    On the circular padded segment the part of the inspiral before the window start wraps
    to the segment's far end, outside the window, whenever N_pad / fs >= T + tau - tc
    (tau the signal's duration from f_lo); N_pad = N is Definition A.  Returns the same
    dict as simulate_batch."""
    N = wl["N"]
    fs = wl["fs"]
    df = fs / N_pad
    F = N_pad // 2 + 1
    noise, psd = bg if bg is not None else background(wl, step)
    theta, offsets = sample_prior(wl["prior"], wl["param_seed"], step, wl["B"], wl["L"], N)
    sel = np.arange(wl["B"]) if draws is None else np.asarray(draws, dtype=np.int64)
    th = theta[:, sel]
    hp, hc = generate_waveforms(th, wl["f_lo"], df, F)
    h = project(hp, hc, th, wl["dets"], wl.get("gmst", 0.0), df)
    sig = np.fft.irfft(fs * h, n=N_pad, axis=-1)[..., :N]
    d = crop(noise, offsets[sel], N) + sig
    y = whiten(d, psd, wl["seg_len"], fs, wl["f_lo"])
    return {"y": y, "theta": theta, "offsets": offsets, "noise": noise, "psd": psd, "draws": sel}


__all__ = ["background", "simulate_batch", "simulate_batch_padded", "C"]

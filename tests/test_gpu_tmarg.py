"""Parity of gwx_log_likelihood_tmarg (ln L with the merger time integrated out) with
the FP64 oracle (needs a GPU).

Tolerance: |Delta ln L| <= 1e-3, the likelihood target of the method.  The marginal's
own arithmetic: the grid values come from FP32 transforms of the band products, whose
rounding is a few ulp of the largest overlap (~rho^2 / 2), i.e. ~1e-4 at SNR 30 and
~1e-3 at SNR 130; the data and template norms and the final sums are FP64."""
import numpy as np
import pytest

import workloads
from oracle import detector, likelihood, noise, spectral, taylorf2
from oracle import constants as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _events(wl, E, seed):
    """E whitened events with non-spinning sources in the prior's merger-time window."""
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    D = len(wl["dets"])
    prior = dict(wl["prior"], chi_lo=0.0, chi_hi=0.0)
    th = workloads.random_theta(seed, E, prior)
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, N // 2 + 1)
    h = detector.project(hp, hc, th, wl["dets"], 0.0, df)
    bg = noise.colored_noise(seed, 0, D, wl["L"], fs, wl["f_lo"])
    psd = spectral.welch_psd(bg, fs, wl["seg_len"], wl["seg_stride"])
    off = workloads.random_offsets(seed, E, wl["L"], N)
    d = spectral.inject(bg, off, h, N, fs)
    y = spectral.whiten(d, psd, wl["seg_len"], fs, wl["f_lo"]).astype(np.float32)
    return th, y, psd, prior


def _samples(th_true, counts, prior, seed):
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    s = workloads.random_theta(seed, S, prior)
    rng = np.random.default_rng(seed + 1)
    for e in range(len(counts)):
        if counts[e] == 0:
            continue
        # the first samples of an event near its source (a sharp peak over the grid), the
        # merger time of the samples anywhere (it is integrated out)
        k = min(3, counts[e])
        s[:, offs[e]:offs[e] + k] = th_true[:, e:e + 1]
        s[C.DIST, offs[e]:offs[e] + k] *= 1.0 + 0.05 * rng.standard_normal(k)
        s[C.M1, offs[e] + 1:offs[e] + k] *= 1.0 + 0.002 * rng.standard_normal(k - 1)
    return s, offs


# The transforms have n = N/2 points: radix-16 passes and a last pass of radix 2^(log2 n
# mod 4) (16 when that is 0), whose needed outputs (2 q n/RS < n_tc) are evaluated one by
# one (few) or by the full butterfly; the cases cover every n from 2^7 to 2^13 and both.
CASES = [
    ("small", 16, 512, 1.0),     # the two-detector workload's prior window [1, 1.5) s, grid 61 us
    ("small", 1, 37, 0.93),      # odd window length, no sub-grid
    ("small", 4, 2048, 0.0),     # the whole circular window (full last butterflies)
    ("hl3", 4, 256, 2.2),        # three detectors, N = 8192 (last radix 16, one output each)
    ("hl3", 2, 6000, 0.4),       # N = 8192, twelve of sixteen outputs (full last butterflies)
    ("sweep", 2, 64, 4.5),       # N = 16384 (one transform per block, in place)
    ("sweep", 64, 40, 4.5),      # N = 16384 at the largest oversampling (the most shared memory)
    (("small", 128, 2.0), 8, 64, 1.0),     # N = 256 (last radix 8, two outputs each)
    (("small", 256, 2.0), 4, 100, 0.97),   # N = 512 (last radix 16, four outputs each)
    (("small", 512, 2.0), 2, 129, 1.0),    # N = 1024 (last radix 2)
    (("small", 2048, 2.0), 4, 700, 1.0),   # N = 4096 (last radix 8, full)
    (("small", 2048, 2.0), 64, 200, 1.1),  # N = 4096, one output each, the largest oversampling
]


@pytest.mark.parametrize("name,u,n_tc,tc_lo", CASES)
def test_tmarg_matches_oracle(gwx, name, u, n_tc, tc_lo):
    wl = workloads.resampled(*name) if isinstance(name, tuple) else workloads.workload(name)
    E = 5
    th_true, y, psd, prior = _events(wl, E, 51)
    counts = workloads.ragged_counts(52, E, 3, 37, zeros=1)
    samples, offs = _samples(th_true, counts, prior, 53)
    ref = likelihood.log_likelihood_tmarg(y.astype(np.float64), psd, wl["seg_len"], wl["fs"], wl["f_lo"], samples,
                                          offs, wl["dets"], tc_lo, n_tc, u)
    got = host(gwx.log_likelihood_tmarg(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                        tc_lo, n_tc, u, cuda(samples), cuda(offs)))
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert err.max() <= 1e-3, (err.max(), ref[np.argmax(err)])


def test_tmarg_importance_weighting_scale_sampled(gwx):
    """64 events with 2k..50k samples each (~1.7 million samples) on the two-detector
    workload with its merger-time window: the oracle recomputes a sample of them,
    including every event's first and last sample (the ragged boundaries)."""
    wl = workloads.workload("small")
    E = 64
    th_true, y, psd, prior = _events(wl, E, 61)
    counts = workloads.ragged_counts(62, E, 2000, 50000)
    samples, offs = _samples(th_true, counts, prior, 63)
    S = int(offs[-1])
    got = host(gwx.log_likelihood_tmarg(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                        1.0, 512, 16, cuda(samples), cuda(offs)))
    assert got.shape == (S,) and np.all(np.isfinite(got))
    rng = np.random.default_rng(64)
    evs = rng.choice(E, 6, replace=False)
    for e in evs:
        pick = np.unique(np.concatenate([[offs[e], offs[e] + 1, offs[e + 1] - 1],
                                         rng.integers(offs[e], offs[e + 1], 3)]))
        ref = likelihood.log_likelihood_tmarg(y[e:e + 1].astype(np.float64), psd, wl["seg_len"], wl["fs"], wl["f_lo"],
                                              samples[:, pick], np.array([0, len(pick)]), wl["dets"], 1.0, 512, 16)
        assert np.abs(got[pick] - ref).max() <= 1e-3, (e, np.abs(got[pick] - ref).max())


def test_tmarg_one_grid_point_is_the_plain_likelihood(gwx):
    wl = workloads.workload("hl3")
    th_true, y, psd, prior = _events(wl, 3, 71)
    samples, offs = _samples(th_true, np.array([9, 0, 17]), prior, 72)
    got = host(gwx.log_likelihood_tmarg(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                        2.41, 1, 1, cuda(samples), cuda(offs)))
    s2 = samples.copy()
    s2[C.TC] = 2.41
    plain = host(gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                    cuda(s2), cuda(offs)))
    assert np.abs(got - plain).max() <= 1e-3


def test_tmarg_empty_and_errors(gwx):
    wl = workloads.workload("small")
    th_true, y, psd, prior = _events(wl, 2, 81)
    args = (cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0)
    out = gwx.log_likelihood_tmarg(*args, 1.0, 512, 16, cuda(np.zeros((11, 0))), cuda(np.array([0, 0, 0])))
    assert out.shape == (0,)
    th = cuda(th_true)
    offs = cuda(np.array([0, 1, 2]))
    for tc_lo, n_tc, u in ((1.0, 512, 3), (1.0, 0, 16), (1.0, 4096, 1), (float("inf"), 512, 16), (1.0, 512, 128)):
        with pytest.raises(gwx.GwxError):
            gwx.log_likelihood_tmarg(*args, tc_lo, n_tc, u, th, offs)

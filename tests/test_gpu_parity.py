"""Parity of every libgwx entry point with the FP64 oracle (needs a GPU).

Each test feeds the same seeded inputs to the CUDA path (through the C ABI via
the Python binding) and to the oracle, and compares element by element.
Tolerances (from the precision targets of the method):
  * waveforms: mismatch <= 1e-6 (analytic PSD, not maximised) and per-bin error
    <= 2e-5 of the draw's peak amplitude;
  * whitened strain: max-abs error <= 1e-4 of the oracle RMS;
  * log-likelihood: |Delta ln L| <= 1e-3;
  * Welch: relative error <= 1e-4 per bin; projection and injection: <= 2e-5
    of the peak; prior draws: offsets bit-exact, doubles within 4 ulp.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import detector, likelihood, noise, pipeline, prior, spectral, taylorf2
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


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rms(x):
    return float(np.sqrt(np.mean(np.abs(x) ** 2)))


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("N,R", [(256, 3), (2048, 5), (8192, 3), (16384, 2)])
def test_rfft_irfft_match_numpy(gwx, N, R):
    x = workloads.random_strain(N + R, (R, N), 1.0)
    X = host(gwx.rfft(cuda(x, torch.float32)))
    ref = np.fft.rfft(x.astype(np.float32).astype(np.float64), axis=-1)
    assert np.abs(X - ref).max() <= 2e-6 * rms(ref) * math.log2(N)
    back = host(gwx.irfft(cuda(ref.astype(np.complex64)), N))
    ref_back = np.fft.irfft(ref.astype(np.complex64).astype(np.complex128), n=N, axis=-1)
    assert np.abs(back - ref_back).max() <= 2e-6 * rms(ref_back) * math.log2(N)


def test_rfft_matches_brute_force_dft(gwx):
    N = 256
    x = workloads.random_strain(3, N, 1.0).astype(np.float32)
    k = np.arange(N)
    X_brute = (np.exp(-2j * math.pi * np.outer(k, k) / N) @ x.astype(np.float64))[: N // 2 + 1]
    X = host(gwx.rfft(cuda(x[None])))[0]
    assert np.abs(X - X_brute).max() < 1e-5 * rms(X_brute)


# ------------------------------------------------------------------ A1 prior
@pytest.mark.parametrize("name,step", [("small", 0), ("hl3", 7)])
def test_sample_prior_matches_oracle(gwx, name, step):
    wl = workloads.workload(name)
    th_ref, off_ref = prior.sample_prior(wl["prior"], wl["param_seed"], step, wl["B"], wl["L"], wl["N"])
    th, off = gwx.sample_prior(wl["prior"], wl["param_seed"], step, wl["B"], wl["L"], wl["N"])
    np.testing.assert_array_equal(host(off), off_ref)
    np.testing.assert_allclose(host(th), th_ref, rtol=4 * 2.0 ** -52, atol=4 * 2.0 ** -52)


def test_sample_prior_edge_sizes(gwx):
    wl = workloads.workload("small")
    th, off = gwx.sample_prior(wl["prior"], 3, 1, 0, wl["L"], wl["N"])
    assert th.shape == (11, 0) and off.shape == (0,)
    th, off = gwx.sample_prior(wl["prior"], 3, 1, 1, wl["N"], wl["N"])     # L == N: offset 0
    assert int(host(off)[0]) == 0


# ------------------------------------------------------------------ A2 waveforms
def _mismatch_per_draw(h_gpu, h_ref, df, k_lo):
    h_gpu = h_gpu.astype(np.complex128)      # |h|^2 ~ 1e-46 would underflow in float32
    F = h_ref.shape[-1]
    S = noise.aligo_psd(np.maximum(np.arange(F) * df, 1.0))
    out = []
    for b in range(h_ref.shape[0]):
        if np.abs(h_ref[b]).max() == 0:
            assert np.abs(h_gpu[b]).max() == 0
            out.append(0.0)
            continue
        out.append(float(likelihood.mismatch(h_gpu[b], h_ref[b], S, df, k_lo, F)))
    return np.array(out)


@pytest.mark.parametrize("name", ["small", "hl3"])
def test_generate_waveforms_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    N, fs = wl["N"], wl["fs"]
    df, F = fs / N, N // 2 + 1
    th = workloads.random_theta(21, wl["B"], wl["prior"])
    hp_ref, hc_ref = taylorf2.generate_waveforms(th, wl["f_lo"], df, F)
    hp, hc = gwx.generate_waveforms(cuda(th), wl["f_lo"], df, F)
    hp, hc = host(hp), host(hc)
    k_lo = math.ceil(wl["f_lo"] / df)
    for got, ref in ((hp, hp_ref), (hc, hc_ref)):
        peak = np.abs(ref).max(axis=1, keepdims=True)
        np.testing.assert_array_equal(got == 0, ref == 0)
        assert np.max(np.abs(got - ref) / np.where(peak > 0, peak, 1)) <= 2e-5
    mm = _mismatch_per_draw(hp, hp_ref, df, k_lo)
    assert mm.max() <= 1e-6, mm.max()


def test_generate_waveforms_lightest_system_phase(gwx):
    """5+5 Msun from 20 Hz on 0.25 Hz bins: ~1400 rad of PN phase at the band edge."""
    th = np.zeros((11, 2))
    th[C.M1], th[C.M2], th[C.DIST] = 5.0, 5.0, 100.0
    th[C.CHI1], th[C.CHI2] = 0.99, -0.99
    th[:, 1] = th[:, 0]
    th[C.CHI1, 1], th[C.CHI2, 1] = 0.99, 0.99
    hp_ref, _ = taylorf2.generate_waveforms(th, 20.0, 0.25, 4097)
    hp, _ = gwx.generate_waveforms(cuda(th), 20.0, 0.25, 4097)
    hp = host(hp)
    on = hp_ref != 0
    dphi = np.angle(hp[on] / hp_ref[on])
    assert np.abs(dphi).max() < 2e-5
    assert _mismatch_per_draw(hp, hp_ref, 0.25, 80).max() <= 1e-6


def test_generate_waveforms_rejects_phenomd_and_bad_sizes(gwx):
    th = cuda(np.ones((11, 2)))
    with pytest.raises(gwx.GwxError) as e:
        gwx.generate_waveforms(th, 20.0, 0.25, 4097, approximant=gwx.IMRPHENOMD)
    assert e.value.status == -6
    with pytest.raises(gwx.GwxError):
        gwx.generate_waveforms(th, 20.0, 0.25, 40000)
    with pytest.raises(gwx.GwxError):
        gwx.generate_waveforms(th, -1.0, 0.25, 4097)


# ------------------------------------------------------------------ A3 projection
@pytest.mark.parametrize("name", ["small", "hl3"])
def test_project_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    N, fs = wl["N"], wl["fs"]
    df, F = fs / N, N // 2 + 1
    B = min(wl["B"], 256)
    th = workloads.random_theta(22, B, wl["prior"])
    hp_ref, hc_ref = taylorf2.generate_waveforms(th, wl["f_lo"], df, F)
    hp32, hc32 = hp_ref.astype(np.complex64), hc_ref.astype(np.complex64)
    ref = detector.project(hp32.astype(np.complex128), hc32.astype(np.complex128), th, wl["dets"], 0.3, df)
    got = host(gwx.project(cuda(hp32), cuda(hc32), cuda(th), wl["dets"], 0.3, df))
    peak = np.abs(ref).max(axis=-1, keepdims=True)
    assert np.max(np.abs(got - ref) / np.where(peak > 0, peak, 1)) <= 2e-5


# ------------------------------------------------------------------ A4 noise
@pytest.mark.parametrize("name", ["small", "hl3"])
def test_colored_noise_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    D = len(wl["dets"])
    ref = noise.colored_noise(wl["noise_seed"], 3, D, wl["L"], wl["fs"], wl["f_lo"])
    got = host(gwx.colored_noise(wl["noise_seed"], 3, D, wl["L"], wl["fs"], wl["f_lo"]))
    r = rms(ref)
    assert np.abs(got - ref).max() <= 1e-4 * r
    assert rms(got - ref) <= 1e-5 * r


def test_colored_noise_longest_background(gwx):
    """The largest background the call accepts, L = 2^24 samples (2.3 h at 2048 Hz), one
    detector: the four-step transform's largest factorisation and 64-bit indexing."""
    L = 1 << 24
    ref = noise.colored_noise(2, 9, 1, L, 2048.0, 20.0)
    got = host(gwx.colored_noise(2, 9, 1, L, 2048.0, 20.0))
    r = rms(ref)
    assert np.abs(got - ref).max() <= 1e-4 * r
    assert rms(got - ref) <= 1e-5 * r


# ------------------------------------------------------------------ A5 Welch
@pytest.mark.parametrize("name", ["small", "hl3"])
def test_welch_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    D = len(wl["dets"])
    x = noise.colored_noise(wl["noise_seed"], 4, D, wl["L"], wl["fs"], wl["f_lo"]).astype(np.float32)
    ref = spectral.welch_psd(x.astype(np.float64), wl["fs"], wl["seg_len"], wl["seg_stride"])
    got = host(gwx.welch_psd(cuda(x), wl["fs"], wl["seg_len"], wl["seg_stride"]))
    assert np.max(np.abs(got / ref - 1)) <= 1e-4


def test_welch_ragged_segments(gwx):
    x = workloads.random_strain(5, (2, 5000), 1e-21).astype(np.float32)
    ref = spectral.welch_psd(x.astype(np.float64), 1024.0, 512, 300)
    got = host(gwx.welch_psd(cuda(x), 1024.0, 512, 300))
    assert np.max(np.abs(got / ref - 1)) <= 1e-4


# ------------------------------------------------------------------ A6 injection
@pytest.mark.parametrize("name", ["small", "hl3"])
def test_inject_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    N, fs, L = wl["N"], wl["fs"], wl["L"]
    df, F = fs / N, N // 2 + 1
    B = 37
    th = workloads.random_theta(23, B, wl["prior"])
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, F)
    h = detector.project(hp, hc, th, wl["dets"], 0.0, df).astype(np.complex64)
    bg = noise.colored_noise(wl["noise_seed"], 0, len(wl["dets"]), L, fs, wl["f_lo"]).astype(np.float32)
    off = workloads.random_offsets(24, B, L, N)
    off[0], off[-1] = 0, L - N
    ref = spectral.inject(bg.astype(np.float64), off, h.astype(np.complex128), N, fs)
    got = host(gwx.inject(cuda(bg), cuda(off), cuda(h), N, fs))
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


# ------------------------------------------------------------------ A7 whitening
@pytest.mark.parametrize("name", ["small", "hl3"])
def test_whiten_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    N, fs, L = wl["N"], wl["fs"], wl["L"]
    D = len(wl["dets"])
    bg = noise.colored_noise(wl["noise_seed"], 0, D, L, fs, wl["f_lo"])
    psd = spectral.welch_psd(bg, fs, wl["seg_len"], wl["seg_stride"])
    B = 29
    off = workloads.random_offsets(25, B, L, N)
    d = spectral.crop(bg, off, N).astype(np.float32)
    ref = spectral.whiten(d.astype(np.float64), psd, wl["seg_len"], fs, wl["f_lo"])
    got = host(gwx.whiten(cuda(d), cuda(psd), wl["seg_len"], fs, wl["f_lo"]))
    assert np.abs(got - ref).max() <= 1e-4 * rms(ref)


@pytest.mark.parametrize("name", ["small", "hl3"])
def test_unwhiten_matches_oracle_and_inverts_whiten(gwx, name):
    """unwhiten against the oracle (max-abs 1e-4 of the RMS), and unwhiten(whiten(x)) =
    x restricted to the band within 1e-5 of its RMS in FP32."""
    wl = workloads.workload(name)
    D, N = len(wl["dets"]), wl["N"]
    bg = noise.colored_noise(3, 0, D, wl["L"], wl["fs"], wl["f_lo"])
    psd = spectral.welch_psd(bg, wl["fs"], wl["seg_len"], wl["seg_stride"])
    y = workloads.random_strain(41, (5, D, N), 1.0)
    ref = spectral.unwhiten(y, psd, wl["seg_len"], wl["fs"], wl["f_lo"])
    got = host(gwx.unwhiten(cuda(y, torch.float32), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"]))
    assert np.abs(got - ref).max() <= 1e-4 * rms(ref)
    x = workloads.random_strain(42, (5, D, N), 1e-21)
    band = spectral.band_mask(N, wl["fs"], wl["f_lo"])
    x_band = np.fft.irfft(np.fft.rfft(x.astype(np.float32).astype(np.float64), axis=-1) * band, n=N, axis=-1)
    xc = cuda(x, torch.float32)
    back = host(gwx.unwhiten(gwx.whiten(xc, cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"]), cuda(psd),
                             wl["seg_len"], wl["fs"], wl["f_lo"]))
    assert np.abs(back - x_band).max() <= 1e-5 * rms(x_band)


def test_whiten_in_place(gwx):
    wl = workloads.workload("small")
    d = workloads.random_strain(26, (3, 2, wl["N"]), 1e-21).astype(np.float32)
    psd = np.full((2, wl["seg_len"] // 2 + 1), 1e-42)
    t = cuda(d)
    ref = host(gwx.whiten(t, cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"]))
    got = host(gwx.whiten(t, cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], out=t))
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------ fused pass
def _gpu_background(gwx, wl, step):
    D = len(wl["dets"])
    n = gwx.colored_noise(wl["noise_seed"], step, D, wl["L"], wl["fs"], wl["f_lo"])
    S = gwx.welch_psd(n, wl["fs"], wl["seg_len"], wl["seg_stride"])
    return n, S


def test_simulate_batch_small_matches_oracle(gwx):
    wl = workloads.workload("small")
    step = 0
    n, S = _gpu_background(gwx, wl, step)
    y, th, off = gwx.simulate_batch(wl["prior"], wl["param_seed"], step, n, S, wl["seg_len"], wl["fs"], wl["f_lo"],
                                    wl["dets"], 0.0, wl["B"], wl["N"])
    ref = pipeline.simulate_batch(wl, step)
    np.testing.assert_array_equal(host(off), ref["offsets"])
    np.testing.assert_allclose(host(th), ref["theta"], rtol=4 * 2.0 ** -52, atol=4 * 2.0 ** -52)
    yr = ref["y"]
    assert np.abs(host(y) - yr).max() <= 1e-4 * rms(yr)


@pytest.mark.parametrize("N_pad", [2048, 8192, 16384])
def test_definition_b_matches_oracle(gwx, N_pad):
    """Padded-grid waveforms (Definition B): waveforms and projection on the N_pad-point
    grid, padded inverse transforms, injection of their first N samples, whitening."""
    wl = workloads.workload("small")
    step = 0
    n, S = _gpu_background(gwx, wl, step)
    y, th, off = gwx.simulate_batch_padded(wl["prior"], wl["param_seed"], step, n, S, wl["seg_len"], wl["fs"],
                                           wl["f_lo"], wl["dets"], 0.0, wl["B"], wl["N"], N_pad)
    ref = pipeline.simulate_batch_padded(wl, step, N_pad)
    np.testing.assert_array_equal(host(off), ref["offsets"])
    yr = ref["y"]
    assert np.abs(host(y) - yr).max() <= 1e-4 * rms(yr)
    if N_pad == wl["N"]:                     # no padding: the fused Definition A pass, to rounding
        ya, _, _ = gwx.simulate_batch(wl["prior"], wl["param_seed"], step, n, S, wl["seg_len"], wl["fs"], wl["f_lo"],
                                      wl["dets"], 0.0, wl["B"], wl["N"])
        assert np.abs(host(ya) - host(y)).max() <= 1e-4 * rms(yr)


def test_simulate_batch_unaligned_background(gwx):
    """A background that starts at an odd float (not 8-byte aligned) takes the scalar
    crop-load path; same results."""
    wl = workloads.workload("small")
    step = 0
    n, S = _gpu_background(gwx, wl, step)
    D, L = n.shape
    buf = torch.empty(D * L + 1, dtype=torch.float32, device=n.device)
    buf[1:].copy_(n.reshape(-1))
    n_mis = buf[1:].view(D, L)
    assert n_mis.data_ptr() % 16 != 0
    y, th, off = gwx.simulate_batch(wl["prior"], wl["param_seed"], step, n_mis, S, wl["seg_len"], wl["fs"],
                                    wl["f_lo"], wl["dets"], 0.0, wl["B"], wl["N"])
    ref = pipeline.simulate_batch(wl, step)
    np.testing.assert_array_equal(host(off), ref["offsets"])
    yr = ref["y"]
    assert np.abs(host(y) - yr).max() <= 1e-4 * rms(yr)


def test_simulate_batch_full_size_sampled(gwx):
    """Three-detector 4 s windows, 2048 draws, in the launch configuration the
    benchmark times; the oracle checks a sample of draws including the first
    and the last."""
    wl = workloads.workload("hl3")
    step = 5
    n, S = _gpu_background(gwx, wl, step)
    y, th, off = gwx.simulate_batch(wl["prior"], wl["param_seed"], step, n, S, wl["seg_len"], wl["fs"], wl["f_lo"],
                                    wl["dets"], 0.0, wl["B"], wl["N"])
    draws = np.unique(np.concatenate([[0, wl["B"] - 1], np.random.default_rng(27).integers(0, wl["B"], 14)]))
    ref = pipeline.simulate_batch(wl, step, draws=draws)
    np.testing.assert_array_equal(host(off), ref["offsets"])
    yr = ref["y"]
    assert np.abs(host(y)[draws] - yr).max() <= 1e-4 * rms(yr)


def test_simulate_equals_whiten_of_inject(gwx):
    """The fused pass equals the unfused inject -> whiten chain on the same inputs."""
    wl = workloads.workload("small")
    n, S = _gpu_background(gwx, wl, 2)
    y, th, off = gwx.simulate_batch(wl["prior"], 9, 2, n, S, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                    wl["B"], wl["N"])
    df, F = wl["fs"] / wl["N"], wl["N"] // 2 + 1
    hp, hc = gwx.generate_waveforms(th, wl["f_lo"], df, F)
    h = gwx.project(hp, hc, th, wl["dets"], 0.0, df)
    d = gwx.inject(n, off, h, wl["N"], wl["fs"])
    y2 = gwx.whiten(d, S, wl["seg_len"], wl["fs"], wl["f_lo"])
    a, b = host(y), host(y2)
    assert np.abs(a - b).max() <= 1e-4 * rms(b)


def test_split_prepare_and_simulate_on_two_streams(gwx):
    """prepare_batch on a side stream + simulate_prepared (the Simulator's step) gives
    the same batch as the single simulate_batch call."""
    import paper_2407_19048_gb300.simulator as S
    wl = workloads.workload("small", B=96)
    sim = S.Simulator(wl)
    y1, th1, off1 = [t.clone() for t in sim.step(11)]
    sim2 = S.Simulator(wl)
    sim2.background(11)
    sim2.simulate(11)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(off1), host(sim2.offsets))
    np.testing.assert_array_equal(host(th1), host(sim2.theta))
    np.testing.assert_array_equal(host(y1), host(sim2.y))


def test_pipelined_simulator_matches_single_calls(gwx):
    """The pipelined Simulator (next batch prepared on the side stream, two buffer sets,
    background every 2 steps) gives the same batches as single simulate_batch calls."""
    import paper_2407_19048_gb300.simulator as S
    wl = workloads.workload("small", B=96)
    sim = S.Simulator(wl, pipeline=True, background_every=2)
    got = [[t.clone() for t in sim.step(st)] for st in (11, 12, 13)]
    again = [t.clone() for t in sim.step(20)]          # a jump in the counter re-prepares
    ref = S.Simulator(wl)
    for st, g in zip((11, 12, 13, 20), got + [again]):
        if st in (11, 13):                              # every second step: 11, 13
            ref.background(st)
        ref.simulate(st)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(g[2]), host(ref.offsets))
        np.testing.assert_array_equal(host(g[1]), host(ref.theta))
        np.testing.assert_array_equal(host(g[0]), host(ref.y))


@pytest.mark.parametrize("B", [0, 1, 3, 1000])
def test_simulate_batch_ragged_sizes(gwx, B):
    wl = workloads.workload("small")
    n, S = _gpu_background(gwx, wl, 1)
    y, th, off = gwx.simulate_batch(wl["prior"], 4, 1, n, S, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                    B, wl["N"])
    if B == 0:
        return
    draws = np.unique([0, B - 1, B // 2])
    ref = pipeline.simulate_batch(dict(wl, B=B, param_seed=4), 1, draws=draws)
    assert np.abs(host(y)[draws] - ref["y"]).max() <= 1e-4 * rms(ref["y"])


def test_simulate_batch_sweep_full_size_sampled(gwx):
    """Three detectors, 8 s windows at 2048 Hz (N = 16384), 8192 draws: the full
    throughput-sweep batch (1.6 GB of output) through the Simulator's two-stream step,
    with the oracle checking a sample of draws."""
    import paper_2407_19048_gb300.simulator as S
    wl = workloads.workload("sweep")
    sim = S.Simulator(wl)
    step = 3
    y, th, off = sim.step(step)
    draws = np.unique(np.concatenate([[0, wl["B"] - 1], np.random.default_rng(28).integers(0, wl["B"], 6)]))
    ref = pipeline.simulate_batch(wl, step, draws=draws)
    np.testing.assert_array_equal(host(off), ref["offsets"])
    got = host(y[torch.from_numpy(draws).cuda()])
    assert np.abs(got - ref["y"]).max() <= 1e-4 * rms(ref["y"])
    del sim, y
    torch.cuda.empty_cache()


def test_simulate_batch_longest_window(gwx):
    """8 s windows at 2048 Hz (N = 16384, the largest supported) with three detectors."""
    wl = workloads.workload("sweep", B=24)
    n, S = _gpu_background(gwx, wl, 0)
    y, th, off = gwx.simulate_batch(wl["prior"], wl["param_seed"], 0, n, S, wl["seg_len"], wl["fs"], wl["f_lo"],
                                    wl["dets"], 0.0, wl["B"], wl["N"])
    draws = np.array([0, 11, 23])
    ref = pipeline.simulate_batch(wl, 0, draws=draws)
    assert np.abs(host(y)[draws] - ref["y"]).max() <= 1e-4 * rms(ref["y"])


# ------------------------------------------------------------------ A8 log-likelihood
def _events(wl, E, seed):
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    D = len(wl["dets"])
    th = workloads.random_theta(seed, E, wl["prior"])
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, N // 2 + 1)
    h = detector.project(hp, hc, th, wl["dets"], 0.0, df)
    bg = noise.colored_noise(seed, 0, D, wl["L"], fs, wl["f_lo"])
    psd = spectral.welch_psd(bg, fs, wl["seg_len"], wl["seg_stride"])
    off = workloads.random_offsets(seed, E, wl["L"], N)
    d = spectral.inject(bg, off, h, N, fs)
    y = spectral.whiten(d, psd, wl["seg_len"], fs, wl["f_lo"]).astype(np.float32)
    return th, y, psd


@pytest.mark.parametrize("name", ["small", "hl3", "sweep"])
def test_log_likelihood_matches_oracle(gwx, name):
    wl = workloads.workload(name)
    E = 6
    th_true, y, psd = _events(wl, E, 31)
    counts = workloads.ragged_counts(32, E, 3, 40, zeros=1)
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    samples = workloads.random_theta(33, S, wl["prior"])
    for e in range(1, E):            # the first sample of every non-empty event is the truth
        samples[:, offs[e]] = th_true[:, e]
    ref = likelihood.log_likelihood(y.astype(np.float64), psd, wl["seg_len"], wl["fs"], wl["f_lo"], samples, offs,
                                    wl["dets"])
    got = host(gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                  cuda(samples), cuda(offs)))
    assert np.abs(got - ref).max() <= 1e-3, np.abs(got - ref).max()


def test_log_likelihood_importance_weighting_scale_sampled(gwx):
    """64 events with 2k..50k samples each (about 1.7 million samples, three
    detectors, 4 s windows): the scale of importance-weighting a flow's samples.  The oracle
    recomputes a sample of 40 samples spread over the events."""
    wl = workloads.workload("hl3")
    E = 64
    th_true, y, psd = _events(wl, E, 35)
    counts = workloads.ragged_counts(36, E, 2000, 50000)
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    samples = workloads.random_theta(37, S, wl["prior"])
    pick = np.unique(np.concatenate([offs[:-1], offs[1:] - 1, np.random.default_rng(38).integers(0, S, 12)]))[:40]
    samples[:, offs[:-1]] = th_true                  # each event's first sample is its truth
    got = host(gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                                  cuda(samples), cuda(offs)))
    ev = np.searchsorted(offs, pick, side="right") - 1
    ref = np.empty(len(pick))
    for i, (s_, e) in enumerate(zip(pick, ev)):
        ref[i] = likelihood.log_likelihood(y[e:e + 1].astype(np.float64), psd, wl["seg_len"], wl["fs"], wl["f_lo"],
                                           samples[:, s_:s_ + 1], np.array([0, 1]), wl["dets"])[0]
    assert np.abs(got[pick] - ref).max() <= 1e-3


def test_log_likelihood_empty_and_errors(gwx):
    wl = workloads.workload("small")
    th_true, y, psd = _events(wl, 2, 34)
    out = gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                             cuda(np.zeros((11, 0))), cuda(np.array([0, 0, 0])))
    assert out.shape == (0,)
    with pytest.raises(gwx.GwxError):
        gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                           cuda(th_true), cuda(np.array([0, 1, 2])), approximant=gwx.IMRPHENOMD)


def test_simulator_step_captures_in_a_cuda_graph(gwx):
    """The hot calls allocate nothing and never synchronise the host, so one simulator
    step (side-stream preparation, background, fused pass) can be captured in a CUDA graph;
    replaying it gives the eager batch bit for bit."""
    import paper_2407_19048_gb300.simulator as S
    wl = workloads.workload("small", B=96)
    eager = S.Simulator(wl)
    y0, th0, off0 = [t.clone() for t in eager.step(21)]
    sim = S.Simulator(wl)
    sim.step(20)                       # warm-up outside the capture (tables, first-call set-up)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            y, th, off = sim.step(21)
    sim.y.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(off), host(off0))
    np.testing.assert_array_equal(host(th), host(th0))
    np.testing.assert_array_equal(host(y), host(y0))


@pytest.mark.parametrize("name", ["small", "hl3", "sweep"])
def test_simulate_launch_shapes_are_bit_identical_and_autotuned(gwx, name):
    """Every launch shape of the fused pass (two-buffer or in-place passes, all or one
    resident block per SM, crop and filter staged in shared memory by bulk copies or read
    from global memory) gives the same batch bit for bit; the autotuner picks one of them
    for the workload's (N, D) and the simulator then uses it; no staged copy timed out."""
    import paper_2407_19048_gb300.simulator as S
    wl = workloads.workload(name, B=min(workloads.workload(name)["B"], 1024))
    D, N = len(wl["dets"]), wl["N"]
    default = gwx.simulate_shape(N, D, -1)
    assert default == (8 if N >= 8192 else 0)
    sim = S.Simulator(wl)
    outs = []
    for shape in (0, 1, 2, 3, 8, 10):
        assert gwx.simulate_shape(N, D, shape) == shape
        y, th, off = sim.step(5)
        outs.append(y.clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    gwx.simulate_shape(N, D, -1)
    picked = sim.autotune(step=5)
    assert picked in (0, 1, 2, 3, 8, 10) and gwx.simulate_shape(N, D) == picked
    y, _, _ = sim.step(5)
    assert torch.equal(y, outs[0])
    gwx.simulate_shape(N, D, -1)
    assert gwx._lib.load().gwx_device_status() == 0

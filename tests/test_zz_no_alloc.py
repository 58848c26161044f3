"""gwx_whiten_static: whitening for callers that cannot allocate device memory.

Such callers (a plug-in whose host owns every device allocation, a serving loop
under a fixed pre-reserved memory budget, a binding that can pass only data
pointers) cannot hand gwx_whiten a workspace.  gwx_whiten_static keeps the
whitening filter in a fixed device array inside the library instead.  These
tests call it through the C ABI and compare it bit for bit with gwx_whiten on two
calls in a row with different shapes and spectra, so that a stale filter left in
the shared array by the first call would show up in the second.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import noise, spectral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2407_19048_gb300 import build, _lib
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return _lib.load()


def _case(name, B, seed):
    wl = workloads.workload(name)
    D = len(wl["dets"])
    bg = noise.colored_noise(wl["noise_seed"], seed, D, wl["L"], wl["fs"], wl["f_lo"])
    psd = spectral.welch_psd(bg, wl["fs"], wl["seg_len"], wl["seg_stride"])
    off = workloads.random_offsets(seed, B, wl["L"], wl["N"])
    d = spectral.crop(bg, off, wl["N"]).astype(np.float32)
    return wl, torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _whiten_with_workspace(lib, wl, d, psd, stream):
    B, D, N = d.shape
    y = torch.empty_like(d)
    nb = lib.gwx_whiten_workspace(D, N)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    st = lib.gwx_whiten(_p(d), _p(psd), wl["seg_len"], wl["fs"], wl["f_lo"], B, D, N, _p(y),
                        ctypes.c_void_p(ws.data_ptr() + off), nb, stream)
    assert st == 0, lib.gwx_last_error()
    return y


def _whiten_static(lib, wl, d, psd, stream):
    B, D, N = d.shape
    y = torch.empty_like(d)
    st = lib.gwx_whiten_static(_p(d), _p(psd), wl["seg_len"], wl["fs"], wl["f_lo"], B, D, N, _p(y), stream)
    assert st == 0, lib.gwx_last_error()
    return y


def test_static_whiten_matches_workspace_whiten_twice(lib):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for name, B, seed in (("hl3", 17, 3), ("small", 9, 4)):      # two calls in a row, different filters
        wl, d, psd = _case(name, B, seed)
        got = _whiten_static(lib, wl, d, psd, stream)
        ref = _whiten_with_workspace(lib, wl, d, psd, stream)
        torch.cuda.synchronize()
        # the same two kernels on the same inputs: the outputs agree bit for bit, so a
        # filter entry left over from the first call would show up here
        assert torch.equal(got, ref)
        assert bool(torch.isfinite(got).all())


def test_static_whiten_rejects_windows_longer_than_its_scratch(lib):
    """N = 32768 would need a filter larger than the static array; the window check
    (a power of two in [256, 16384], shared with gwx_whiten) refuses it first."""
    st = lib.gwx_whiten_static(None, None, 4096, 2048.0, 20.0, 1, 4, 32768, None, None)
    assert st == -2
    assert b"power of two in [256, 16384]" in lib.gwx_last_error()
    st = lib.gwx_whiten_static(None, None, 4096, 2048.0, 20.0, 1, 5, 16384, None, None)   # D > GWX_MAX_DET
    assert st == -2

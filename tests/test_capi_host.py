"""Host-side checks of the C ABI (CPU only): the library builds, loads, exports
every entry point the header declares, and its pure-host functions agree with
the oracle.  No call here launches device work."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gwx.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2407_19048_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gwx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gwx_generate_waveforms", "gwx_project", "gwx_inject", "gwx_welch_psd", "gwx_whiten",
                     "gwx_log_likelihood", "gwx_sample_prior", "gwx_colored_noise", "gwx_simulate_batch"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2407_19048_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gwx_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(_lib.SIGNATURES) <= exported


def test_version_and_status_strings(lib):
    assert lib.gwx_version() == 100
    assert lib.gwx_status_string(0) == b"ok"
    assert lib.gwx_status_string(-6) == b"unsupported"


def test_detector_geometry_matches_oracle(lib):
    import paper_2407_19048_gb300 as gwx
    from oracle import detector
    for name in ("H1", "L1", "V1"):
        T, r = gwx.detector_geometry(name)
        D_ref, r_ref = detector.geometry(name)
        np.testing.assert_allclose(np.array(T), D_ref, atol=1e-15)
        np.testing.assert_allclose(np.array(r), r_ref, rtol=1e-15)


def test_workspace_sizes(lib):
    import paper_2407_19048_gb300 as gwx
    assert gwx.workspace_bytes("whiten", 3, 8192) == ((3 * 4097 * 4 + 255) // 256) * 256
    K = (131072 - 4096) // 2048 + 1
    assert gwx.workspace_bytes("welch_psd", 3, 131072, 4096, 2048) >= 3 * K * 2049 * 8
    assert gwx.workspace_bytes("colored_noise", 3, 131072) >= 3 * 65536 * 8
    assert gwx.workspace_bytes("simulate_batch", 3, 2048, 8192) > 2048 * 144
    assert gwx.workspace_bytes("log_likelihood", 4, 3, 8192, 100) > 0
    assert gwx.workspace_bytes("importance_weights", 64) >= 64 * 16 * 24
    assert gwx.workspace_bytes("importance_weights", 0) == 0


def test_validation_fails_before_any_launch(lib):
    """Bad sizes are rejected on the host, with a message, without touching a device."""
    import paper_2407_19048_gb300 as gwx
    from paper_2407_19048_gb300 import _lib
    st = lib.gwx_generate_waveforms(1, None, 4, 20.0, 0.25, 4097, None, None, None)
    assert st == -6 and b"IMRPhenomD" in lib.gwx_last_error()
    st = lib.gwx_inject(None, 2, 1000, None, None, 4, 1000, 1024.0, None, None)   # N not a power of two
    assert st == -2 and b"power of two" in lib.gwx_last_error()
    st = lib.gwx_welch_psd(None, 9, 4096, 1024.0, 1024, 512, None, None, 0, None)
    assert st == -2
    p = _lib.GwxPrior(*([0.0] * 12))
    st = lib.gwx_sample_prior(p, 1, 0, 16, 100, 200, None, None, None)         # L < N
    assert st == -2
    import ctypes
    st = lib.gwx_rfft(ctypes.c_void_p(0x1004), 1, 256, ctypes.c_void_p(0x2000), None)
    assert st == -1 and b"not 8-byte aligned" in lib.gwx_last_error()
    st = lib.gwx_gemm_bf16(None, None, None, 128, 256, 12, 0, None)
    assert st == -2 and b"K % 8" in lib.gwx_last_error()
    st = lib.gwx_gemm_bf16(ctypes.c_void_p(0x1008), ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000), 8, 8, 8, 0,
                           None)
    assert st == -1 and b"16-byte aligned" in lib.gwx_last_error()
    st = lib.gwx_importance_weights(None, None, None, 0, 5, None, None, None, None, None, 0, None)
    assert st == -2 and b"without events" in lib.gwx_last_error()
    st = lib.gwx_importance_weights(None, None, None, -1, 0, None, None, None, None, None, 0, None)
    assert st == -2
    with pytest.raises(KeyError):
        gwx.detector_geometry("K1")


def test_flow_layout_and_validation(lib):
    """The flow's flat parameter layout (host arithmetic) and its argument checks."""
    import ctypes
    import paper_2407_19048_gb300 as gwx
    import workloads
    shape = workloads.flow_shape(features=128, group=16, embed_hidden=64, context=32, layers=3, hidden=48)
    n, off = gwx.flow_layout(shape)
    sizes = [int(np.prod(s)) for s in workloads.flow_tensor_shapes(shape)]
    assert len(off) == len(sizes) == 6 + 6 * 3
    assert off[0] == 0 and all(o % 64 == 0 for o in off)
    for t in range(len(off) - 1):
        assert off[t + 1] - off[t] == (sizes[t] + 63) // 64 * 64
    assert n == off[-1] + (sizes[-1] + 63) // 64 * 64
    sh = gwx.flow_shape(128, 16, 64, 30, 3, 48)                     # context not a multiple of 8
    assert lib.gwx_flow_layout(ctypes.byref(sh), None, None) == -2
    sh = gwx.flow_shape(128, 16, 64, 32, 0, 48)                     # no layers
    assert lib.gwx_flow_layout(ctypes.byref(sh), None, None) == -2
    sh = gwx.flow_shape(128, 16, 64, 32, 3, 48)
    assert lib.gwx_flow_train_workspace(ctypes.byref(sh), 64, 2, 2048) > 0
    assert lib.gwx_sample_posterior_workspace(ctypes.byref(sh), 4, 2, 2048, 1000) > 0
    m8 = (ctypes.c_double * 8)(*([0.0] * 8))
    s8 = (ctypes.c_double * 8)(*([1.0] * 8))
    # batch not a multiple of 8: rejected before any launch
    st = lib.gwx_flow_train_step(ctypes.byref(sh), None, None, None, None, None, 1, None, 1e-3, 0.9, 0.999, 1e-8, 0.0,
                                 1.0,
                                 m8, s8, None, None, 12, 2, 2048, 1024.0, 20.0, None, None, None, None, 0, None)
    assert st == -2 and b"multiple of 8" in lib.gwx_last_error()
    # too few feature columns for the band
    sh_small = gwx.flow_shape(64, 16, 64, 32, 3, 48)
    st = lib.gwx_flow_log_prob(ctypes.byref(sh_small), None, None, m8, s8, None, None, 8, 2, 2048, 1024.0, 20.0,
                               None, None, None, 0, None)
    assert st == -2 and b"groups" in lib.gwx_last_error()
    bad = (ctypes.c_double * 8)(*([1.0] * 7 + [0.0]))
    st = lib.gwx_flow_targets(None, 4, m8, bad, None, None)
    assert st == -1 and b"scale" in lib.gwx_last_error()


def test_resnet_and_dense_validation(lib):
    """The ResNet pieces keep one grid row per sample and 32-bit index arithmetic within a
    sample, so their shapes are bounded on the host; the dense backward's workspace
    grows with the split-K slices of dW when the batch is long and the output small."""
    import ctypes
    st = lib.gwx_group_norm(None, 65536, 8, 64, 8, None, None, None, None, 1, None, None, None, None)
    assert st == -2 and b"65535" in lib.gwx_last_error()
    st = lib.gwx_group_norm(None, 2, 1 << 20, 4096, 8, None, None, None, None, 1, None, None, None, None)
    assert st == -2                                                  # T C = 2^32
    st = lib.gwx_group_norm(None, 4, 8, 60, 8, None, None, None, None, 1, None, None, None, None)
    assert st == -2 and b"multiple of G" in lib.gwx_last_error()
    st = lib.gwx_im2col(None, 2, 1 << 19, 1024, 5, 1, 2, 5120, None, None)   # T_out K >= 2^31
    assert st == -2 and b"T_out K" in lib.gwx_last_error()
    st = lib.gwx_col2im(None, 65536, 16, 8, 5, 1, 2, 40, None, None, None)
    assert st == -2
    small = lib.gwx_dense_bf16_backward_workspace(512, 64, 320)
    long_batch = lib.gwx_dense_bf16_backward_workspace(262144, 64, 320)
    # the dW slices: at most ~128 work items over 2 tiles, 64 x 320 FP32 each
    assert long_batch >= 262144 * 64 * 4 + 262144 * 320 * 2 + 64 * 64 * 320 * 4
    assert small < long_batch


def test_adamw_at_validation(lib):
    """The device-step AdamW rejects a missing step counter and bad hyper-parameters before
    any launch, and n = 0 is a no-op."""
    dummy = 16   # never dereferenced: the checks come first
    st = lib.gwx_adamw_at(dummy, dummy, dummy, dummy, 10, 1e-3, 0.9, 0.999, 1e-8, 0.0, None, None, None)
    assert st == -1 and b"step" in lib.gwx_last_error()
    st = lib.gwx_adamw_at(dummy, dummy, dummy, dummy, 10, 1e-3, 1.0, 0.999, 1e-8, 0.0, dummy, None, None)
    assert st == -1 and b"hyper-parameters" in lib.gwx_last_error()
    st = lib.gwx_adamw_at(dummy, dummy, dummy, dummy, -1, 1e-3, 0.9, 0.999, 1e-8, 0.0, dummy, None, None)
    assert st == -2
    assert lib.gwx_adamw_at(None, None, None, None, 0, 1e-3, 0.9, 0.999, 1e-8, 0.0, None, None, None) == 0


def test_conv1d_validation(lib):
    """The implicit-GEMM convolutions take whole 128-time tiles and 64-channel blocks; other
    shapes, even kernels, missing arrays and short workspaces fail before any launch."""
    import ctypes
    good = dict(B=2, T=256, C=64, O=64, k=5)
    for bad, word in ((dict(T=200), b"T %"), (dict(C=96), b"C and O"), (dict(O=32), b"C and O"), (dict(k=4), b"k odd"),
                      (dict(k=17), b"k odd"), (dict(B=1 << 19, T=256), b"2^26")):
        a = dict(good, **bad)
        st = lib.gwx_conv1d_bf16(None, a["B"], a["T"], a["C"], a["k"], None, a["O"], None, None, None)
        assert st == -2 and word in lib.gwx_last_error(), (bad, lib.gwx_last_error())
    st = lib.gwx_conv1d_bf16(None, 2, 256, 64, 5, None, 64, None, None, None)
    assert st == -1 and b"NULL" in lib.gwx_last_error()
    ws = lib.gwx_conv1d_bf16_backward_workspace(2, 256, 64, 64, 5)
    # dZ and dZ^T (bfloat16), the transposed weights and the transposed rows 5 C x B T
    assert ws >= 2 * 512 * 64 * 2 + 64 * 5 * 64 * 2 + 5 * 64 * 512 * 2
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    st = lib.gwx_conv1d_bf16_backward(p, p, p, 2, 256, 64, 64, 5, None, None, None, p, 64, None)
    assert st == -4 and b"workspace" in lib.gwx_last_error()


def test_static_whitening_checks_as_gwx_whiten(lib):
    """gwx_whiten_static runs gwx_whiten's own argument checks (before any device work):
    the same statuses and messages for a non-finite sample rate, a band start above the
    last bin, a bad window and too many detectors."""
    import ctypes
    ws = ctypes.c_void_p(0x10000)
    cases = [
        (4096, float("inf"), 20.0, 1, 3, 8192),      # fs = +inf: df = inf
        (4096, 2048.0, float("inf"), 1, 3, 8192),    # f_lo = +inf
        (4096, 2048.0, 2000.0, 1, 3, 8192),          # band starts above the last usable bin
        (4096, 2048.0, 20.0, 1, 3, 8000),            # window not a power of two
        (4096, 2048.0, 20.0, 1, 5, 8192),            # more detectors than GWX_MAX_DET
        (4095, 2048.0, 20.0, 1, 3, 8192),            # Welch segment not a power of two
    ]
    for seg_len, fs, f_lo, B, D, N in cases:
        st_ref = lib.gwx_whiten(None, None, seg_len, fs, f_lo, B, D, N, None, ws, 1 << 20, None)
        msg_ref = lib.gwx_last_error()
        st = lib.gwx_whiten_static(None, None, seg_len, fs, f_lo, B, D, N, None, None)
        assert st == st_ref and st < 0, (seg_len, fs, f_lo, D, N, st, st_ref)
        assert lib.gwx_last_error() == msg_ref
    st = lib.gwx_whiten_static(None, None, 4096, float("inf"), 20.0, 1, 3, 8192, None, None)
    assert st == -1 and b"must be positive" in lib.gwx_last_error()


def test_tmarg_likelihood_validation(lib):
    """The merger-time marginal rejects a bad grid on the host, before any device work."""
    import ctypes
    ids = (ctypes.c_int32 * 2)(0, 1)
    def call(tc_lo, n_tc, u, N=2048):
        return lib.gwx_log_likelihood_tmarg(0, None, 1, 2, N, None, 1024, 1024.0, 20.0, ids, 0.0, tc_lo, n_tc, u,
                                            None, None, 4, None, None, 0, None)
    assert call(1.0, 512, 3) == -2 and b"power of two" in lib.gwx_last_error()
    assert call(1.0, 512, 128) == -2
    assert call(1.0, 0, 16) == -2 and b"n_tc" in lib.gwx_last_error()
    assert call(1.0, 4096, 16) == -2
    assert call(float("nan"), 512, 16) == -1 and b"tc_lo" in lib.gwx_last_error()
    assert call(1.0, 512, 16, N=3000) == -2
    assert call(1.0, 512, 16) == -1 and b"NULL" in lib.gwx_last_error()   # valid grid: the NULL arrays are next

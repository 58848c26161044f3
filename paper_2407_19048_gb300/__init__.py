"""GB300-native on-the-fly simulation and pre-processing of gravitational-wave training data.

Python binding of the libgwx C ABI (``include/gwx.h``).  Each function below
has the name of a C entry point without its ``gwx_`` prefix and only marshals
arguments: it checks tensor devices, dtypes and shapes, allocates outputs and
workspaces with PyTorch on the current CUDA device, and calls the library on
PyTorch's current stream.  All computation happens in the library's CUDA
kernels; nothing here has a CPU path.

The steps follow Sec. 3 of the paper: prior draws (Table 1), TaylorF2
waveforms (Sec. 3.1), detector projection, background crops and injection,
Welch PSD and whitening (Sec. 3.2), plus the standard Gaussian-noise
log-likelihood used by its nested-sampling comparison (Sec. 6).
"""
import ctypes

from . import _lib

TAYLORF2 = 0
IMRPHENOMD = 1
DETECTORS = {"H1": 0, "L1": 1, "V1": 2}
M1, M2, CHI1, CHI2, DIST, TC, PHIC, THETAJN, PSI, RA, DEC = range(11)
NPARAM = 11

__all__ = ["GwxError", "version", "init", "detector_geometry", "sample_prior", "generate_waveforms", "project",
           "colored_noise", "welch_psd", "inject", "inject_padded", "simulate_batch_padded", "whiten", "unwhiten", "simulate_batch", "simulate_shape", "log_likelihood", "log_likelihood_tmarg",
           "importance_weights", "gemm_bf16", "dense_bf16", "dense_bf16_backward", "gemm_autotune", "spectral_features",
           "cross_features", "lag_features", "proposal_targets",
           "gauss_nll", "adamw", "adamw_at", "adamw_clip", "skymap", "vicreg", "retime", "sample_proposal", "device_status", "selftest_bounded_wait", "rfft", "irfft",
           "workspace_bytes", "debug_check", "conv1d_bf16", "conv1d_bf16_backward", "TAYLORF2", "IMRPHENOMD", "DETECTORS"]


class GwxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("libgwx status %d: %s" % (status, message))
        self.status = status


def _check(status):
    if status != 0:
        lib = _lib.load()
        raise GwxError(status, lib.gwx_last_error().decode(errors="replace"))
    if _lib.DEBUG:
        debug_check()


# Debug build (GWX_DEBUG=1): every workspace the binding allocates is followed by a
# guard of _GUARD bytes in a fixed pattern, and after every call the guards of the live
# workspaces and the kernels' index records are checked (synchronising the device; calls
# made while a stream is being captured are checked at the next call outside capture).
_GUARD = 256
_guards = []


def debug_check():
    """Raise GwxError if a kernel of the debug build recorded an out-of-range access or a
    call wrote into the guard after one of the binding's workspaces (no-op otherwise)."""
    if not _lib.DEBUG or _torch().cuda.is_current_stream_capturing():
        return
    lib = _lib.load()
    first = ctypes.c_uint64(0)
    st = lib.gwx_debug_status(ctypes.byref(first))
    if st != 0:
        raise GwxError(st, lib.gwx_last_error().decode(errors="replace"))
    live = []
    for ref, ptr, nbytes in _guards:
        if ref() is None:
            continue
        live.append((ref, ptr, nbytes))
        ok = ctypes.c_int(1)
        st = lib.gwx_debug_check_guard(ctypes.c_void_p(ptr), nbytes, _GUARD, ctypes.byref(ok), _stream())
        if st != 0:
            raise GwxError(st, lib.gwx_last_error().decode(errors="replace"))
        if not ok.value:
            raise GwxError(-2, "a call wrote past the end of a %d-byte workspace" % nbytes)
    _guards[:] = live


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (libgwx has no CPU path)" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _workspace(nbytes, device):
    torch = _torch()
    if nbytes == 0:
        return None, 0
    guard = _GUARD if _lib.DEBUG else 0
    ws = torch.empty(nbytes + 256 + guard, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    if guard:
        import weakref
        ptr = ws.data_ptr() + off
        st = _lib.load().gwx_debug_guard(ctypes.c_void_p(ptr), nbytes, guard, _stream())
        if st != 0:
            raise GwxError(st, _lib.load().gwx_last_error().decode(errors="replace"))
        _guards.append((weakref.ref(ws), ptr, nbytes))
    return ws[off:off + nbytes], nbytes


def _det_ids(dets):
    ids = [DETECTORS[d] if isinstance(d, str) else int(d) for d in dets]
    return (ctypes.c_int32 * len(ids))(*ids), len(ids)


def _prior(p):
    if isinstance(p, _lib.GwxPrior):
        return p
    return _lib.GwxPrior(*[float(p[k]) for k in (
        "m_lo", "m_hi", "chi_lo", "chi_hi", "d_lo", "d_hi", "tc_lo", "tc_hi", "phi_lo", "phi_hi", "psi_lo", "psi_hi")])


def version():
    return _lib.load().gwx_version()


def init():
    """Prepare the per-device tables on the current device (outside stream capture)."""
    _check(_lib.load().gwx_init())


def detector_geometry(det):
    """(tensor [3][3], position [3] m) of a detector, computed on the host."""
    lib = _lib.load()
    T = (ctypes.c_double * 9)()
    r = (ctypes.c_double * 3)()
    _check(lib.gwx_detector_geometry(DETECTORS[det] if isinstance(det, str) else int(det), T, r))
    return [list(T[3 * i:3 * i + 3]) for i in range(3)], list(r)


def workspace_bytes(call, *args):
    """Workspace size of an entry point, e.g. workspace_bytes("whiten", D, N)."""
    return int(getattr(_lib.load(), "gwx_%s_workspace" % call)(*args))


def sample_prior(prior, seed, step, B, L, N, theta=None, offsets=None):
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    theta = torch.empty((NPARAM, B), dtype=torch.float64, device=dev) if theta is None else \
        _dev(theta, torch.float64, "theta")
    offsets = torch.empty(B, dtype=torch.int64, device=dev) if offsets is None else _dev(offsets, torch.int64, "offsets")
    p = _prior(prior)
    _check(_lib.load().gwx_sample_prior(ctypes.byref(p), seed, step, B, L, N, _ptr(theta), _ptr(offsets), _stream()))
    return theta, offsets


def generate_waveforms(theta, f_lo, df, F, approximant=TAYLORF2, hp=None, hc=None):
    torch = _torch()
    _dev(theta, torch.float64, "theta")
    B = theta.shape[1]
    hp = torch.empty((B, F), dtype=torch.complex64, device=theta.device) if hp is None else hp
    hc = torch.empty((B, F), dtype=torch.complex64, device=theta.device) if hc is None else hc
    _check(_lib.load().gwx_generate_waveforms(approximant, _ptr(theta), B, f_lo, df, F, _ptr(hp), _ptr(hc), _stream()))
    return hp, hc


def project(hp, hc, theta, dets, gmst, df, out=None):
    torch = _torch()
    _dev(hp, torch.complex64, "hp")
    _dev(hc, torch.complex64, "hc")
    _dev(theta, torch.float64, "theta")
    B, F = hp.shape
    ids, D = _det_ids(dets)
    out = torch.empty((B, D, F), dtype=torch.complex64, device=hp.device) if out is None else out
    _check(_lib.load().gwx_project(_ptr(hp), _ptr(hc), _ptr(theta), B, ids, D, gmst, df, F, _ptr(out), _stream()))
    return out


def colored_noise(seed, step, D, L, fs, f_lo, out=None):
    torch = _torch()
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((D, L), dtype=torch.float32, device=dev) if out is None else out
    ws, nb = _workspace(lib.gwx_colored_noise_workspace(D, L), dev)
    _check(lib.gwx_colored_noise(seed, step, D, L, fs, f_lo, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def welch_psd(x, fs, seg_len, stride, out=None):
    torch = _torch()
    lib = _lib.load()
    _dev(x, torch.float32, "x")
    D, L = x.shape
    out = torch.empty((D, seg_len // 2 + 1), dtype=torch.float64, device=x.device) if out is None else out
    ws, nb = _workspace(lib.gwx_welch_psd_workspace(D, L, seg_len, stride), x.device)
    _check(lib.gwx_welch_psd(_ptr(x), D, L, fs, seg_len, stride, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def inject(noise, offsets, h_det, N, fs, out=None):
    torch = _torch()
    _dev(noise, torch.float32, "noise")
    _dev(offsets, torch.int64, "offsets")
    _dev(h_det, torch.complex64, "h_det")
    D, L = noise.shape
    B = h_det.shape[0]
    out = torch.empty((B, D, N), dtype=torch.float32, device=noise.device) if out is None else out
    _check(_lib.load().gwx_inject(_ptr(noise), D, L, _ptr(offsets), _ptr(h_det), B, N, fs, _ptr(out), _stream()))
    return out


def inject_padded(noise, offsets, h_td, N, fs, out=None):
    """Definition B injection: d [B][D][N] = noise crops + fs h_td[..., :N] (h_td [B][D][N_pad])."""
    torch = _torch()
    _dev(noise, torch.float32, "noise")
    _dev(offsets, torch.int64, "offsets")
    _dev(h_td, torch.float32, "h_td")
    D, L = noise.shape
    B, _, Np = h_td.shape
    out = torch.empty((B, D, N), dtype=torch.float32, device=noise.device) if out is None else out
    _check(_lib.load().gwx_inject_padded(_ptr(noise), D, L, _ptr(offsets), _ptr(h_td), B, N, Np, fs, _ptr(out),
                                         _stream()))
    return out


def simulate_batch_padded(prior, seed, step, noise, psd, seg_len, fs, f_lo, dets, gmst, B, N, N_pad):
    """One whitened batch with Definition B waveforms: prior draws, waveforms and projection
    on the N_pad-point grid, inverse transforms over the padded segment, injection of their
    first N samples, whitening (each step one libgwx call).  Returns (y, theta, offsets)."""
    D, L = noise.shape
    theta, offsets = sample_prior(prior, seed, step, B, L, N)
    df = fs / N_pad
    hp, hc = generate_waveforms(theta, f_lo, df, N_pad // 2 + 1)
    h = project(hp, hc, theta, dets, gmst, df)
    h_td = irfft(h, N_pad)
    d = inject_padded(noise, offsets, h_td, N, fs)
    return whiten(d, psd, seg_len, fs, f_lo), theta, offsets


def whiten(d, psd, seg_len, fs, f_lo, out=None):
    torch = _torch()
    lib = _lib.load()
    _dev(d, torch.float32, "d")
    _dev(psd, torch.float64, "psd")
    B, D, N = d.shape
    out = torch.empty_like(d) if out is None else out
    ws, nb = _workspace(lib.gwx_whiten_workspace(D, N), d.device)
    _check(lib.gwx_whiten(_ptr(d), _ptr(psd), seg_len, fs, f_lo, B, D, N, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def unwhiten(y, psd, seg_len, fs, f_lo, out=None):
    """Inverse of whiten on the band (for checks): d [B][D][N] from y."""
    torch = _torch()
    lib = _lib.load()
    _dev(y, torch.float32, "y")
    _dev(psd, torch.float64, "psd")
    B, D, N = y.shape
    out = torch.empty_like(y) if out is None else out
    ws, nb = _workspace(lib.gwx_whiten_workspace(D, N), y.device)
    _check(lib.gwx_unwhiten(_ptr(y), _ptr(psd), seg_len, fs, f_lo, B, D, N, _ptr(out), _ptr(ws), nb, _stream()))
    return out


class SimulateBuffers:
    """Preallocated outputs and workspace for repeated simulate_batch calls."""

    def __init__(self, B, D, N, device=None):
        torch = _torch()
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.y = torch.empty((B, D, N), dtype=torch.float32, device=dev)
        self.theta = torch.empty((NPARAM, B), dtype=torch.float64, device=dev)
        self.offsets = torch.empty(B, dtype=torch.int64, device=dev)
        self.ws, self.ws_bytes = _workspace(_lib.load().gwx_simulate_batch_workspace(D, B, N), dev)


def simulate_batch(prior, seed, step, noise, psd, seg_len, fs, f_lo, dets, gmst, B, N, buffers=None):
    """One whitened batch (Sec. 3.2): returns (y [B][D][N], theta [11][B], offsets [B])."""
    torch = _torch()
    _dev(noise, torch.float32, "noise")
    _dev(psd, torch.float64, "psd")
    D, L = noise.shape
    ids, nd = _det_ids(dets)
    bufs = buffers or SimulateBuffers(B, nd, N, noise.device)
    p = _prior(prior)
    _check(_lib.load().gwx_simulate_batch(ctypes.byref(p), seed, step, _ptr(noise), L, _ptr(psd), seg_len, fs, f_lo,
                                          ids, nd, gmst, B, N, _ptr(bufs.y), _ptr(bufs.theta), _ptr(bufs.offsets),
                                          _ptr(bufs.ws), bufs.ws_bytes, _stream()))
    return bufs.y, bufs.theta, bufs.offsets


def log_likelihood(y_data, psd, seg_len, fs, f_lo, dets, gmst, theta, event_offsets, approximant=TAYLORF2,
                   out=None):
    """ln L [S] of samples theta [11][S] against whitened events y_data [E][D][N]."""
    torch = _torch()
    lib = _lib.load()
    _dev(y_data, torch.float32, "y_data")
    _dev(psd, torch.float64, "psd")
    _dev(theta, torch.float64, "theta")
    _dev(event_offsets, torch.int64, "event_offsets")
    E, D, N = y_data.shape
    S = theta.shape[1]
    ids, nd = _det_ids(dets)
    out = torch.empty(S, dtype=torch.float64, device=y_data.device) if out is None else out
    ws, nb = _workspace(lib.gwx_log_likelihood_workspace(E, D, N, S), y_data.device)
    _check(lib.gwx_log_likelihood(approximant, _ptr(y_data), E, D, N, _ptr(psd), seg_len, fs, f_lo, ids, gmst,
                                  _ptr(theta), _ptr(event_offsets), S, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def simulate_shape(N, D, shape=-2):
    """The fused pass's launch shape for windows of N samples and D detectors: shape >= 0
    records one, -1 forgets the record, -2 (default) only asks; returns the shape in use."""
    st = _lib.load().gwx_simulate_shape(int(N), int(D), int(shape))
    if st < 0:
        _check(st)
    return st


def log_likelihood_tmarg(y_data, psd, seg_len, fs, f_lo, dets, gmst, tc_lo, n_tc, oversample, theta, event_offsets,
                         approximant=TAYLORF2, out=None):
    """ln L [S] of samples theta [11][S] with the merger time integrated out over
    [tc_lo, tc_lo + n_tc / fs) on a grid of spacing 1 / (oversample fs) (the tc row of
    theta is not read)."""
    torch = _torch()
    lib = _lib.load()
    _dev(y_data, torch.float32, "y_data")
    _dev(psd, torch.float64, "psd")
    _dev(theta, torch.float64, "theta")
    _dev(event_offsets, torch.int64, "event_offsets")
    E, D, N = y_data.shape
    S = theta.shape[1]
    ids, nd = _det_ids(dets)
    out = torch.empty(S, dtype=torch.float64, device=y_data.device) if out is None else out
    ws, nb = _workspace(lib.gwx_log_likelihood_workspace(E, D, N, S), y_data.device)
    _check(lib.gwx_log_likelihood_tmarg(approximant, _ptr(y_data), E, D, N, _ptr(psd), seg_len, fs, f_lo, ids, gmst,
                                        float(tc_lo), int(n_tc), int(oversample), _ptr(theta), _ptr(event_offsets), S,
                                        _ptr(out), _ptr(ws), nb, _stream()))
    return out


def importance_weights(lnl, event_offsets, log_ratio=None):
    """Per-event importance weights of scored samples: returns (weights [S], ess [E],
    efficiency [E], ln_evidence [E]) as device float64 tensors (see gwx.h)."""
    torch = _torch()
    lib = _lib.load()
    _dev(lnl, torch.float64, "lnl")
    _dev(event_offsets, torch.int64, "event_offsets")
    if log_ratio is not None:
        _dev(log_ratio, torch.float64, "log_ratio")
    S = lnl.shape[0]
    E = event_offsets.shape[0] - 1
    dev = lnl.device
    w = torch.empty(S, dtype=torch.float64, device=dev)
    ess, eff, lnz = (torch.empty(max(E, 0), dtype=torch.float64, device=dev) for _ in range(3))
    ws, nb = _workspace(lib.gwx_importance_weights_workspace(E), dev)
    _check(lib.gwx_importance_weights(_ptr(lnl), _ptr(log_ratio) if log_ratio is not None else None,
                                      _ptr(event_offsets), E, S, _ptr(w), _ptr(ess), _ptr(eff), _ptr(lnz),
                                      _ptr(ws), nb, _stream()))
    return w, ess, eff, lnz


def gemm_bf16(A, B, out=None, out_dtype=None):
    """C = A B^T on the tensor cores: A bfloat16 [M][K], B bfloat16 [N][K], C float32
    (default) or bfloat16 [M][N]."""
    torch = _torch()
    _dev(A, torch.bfloat16, "A")
    _dev(B, torch.bfloat16, "B")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A is [M][K] and B is [N][K]")
    if out is None:
        out = torch.empty((M, N), dtype=out_dtype or torch.float32, device=A.device)
    code = {torch.float32: 0, torch.bfloat16: 1}[out.dtype]
    _check(_lib.load().gwx_gemm_bf16(_ptr(A), _ptr(B), _ptr(out), M, N, K, code, _stream()))
    return out


ACT_NONE, ACT_RELU, ACT_GELU = 0, 1, 2


def dense_bf16(X, W, bias=None, act=ACT_NONE, out=None, out_dtype=None):
    """Y = act(X W^T + bias) on the tensor cores: X bfloat16 [M][K], W bfloat16 [N][K],
    bias float32 [N] or None, Y float32 (default) or bfloat16 [M][N]."""
    torch = _torch()
    _dev(X, torch.bfloat16, "X")
    _dev(W, torch.bfloat16, "W")
    if bias is not None:
        _dev(bias, torch.float32, "bias")
    M, K = X.shape
    N = W.shape[0]
    if W.shape[1] != K or (bias is not None and bias.numel() != N):
        raise ValueError("X is [M][K], W is [N][K], bias is [N]")
    if out is None:
        out = torch.empty((M, N), dtype=out_dtype or torch.float32, device=X.device)
    code = {torch.float32: 0, torch.bfloat16: 1}[out.dtype]
    _check(_lib.load().gwx_dense_bf16(_ptr(X), _ptr(W), _ptr(bias), _ptr(out), M, N, K, act, code, _stream()))
    return out


def dense_bf16_backward(X, W, bias, dY, act=ACT_NONE, want_dx=True, want_db=None):
    """Gradients of Y = act(X W^T + bias) for dL/dY = dY (float32 [M][N]): returns
    (dX float32 [M][K], dW float32 [N][K], db float32 [N]); dX is None when want_dx is
    false and db None when want_db is false (default: db only when there is a bias)."""
    torch = _torch()
    _dev(X, torch.bfloat16, "X")
    _dev(W, torch.bfloat16, "W")
    _dev(dY, torch.float32, "dY")
    if bias is not None:
        _dev(bias, torch.float32, "bias")
    if want_db is None:
        want_db = bias is not None
    M, K = X.shape
    N = W.shape[0]
    dev = X.device
    dX = torch.empty((M, K), dtype=torch.float32, device=dev) if want_dx else None
    dW = torch.empty((N, K), dtype=torch.float32, device=dev)
    db = torch.empty(N, dtype=torch.float32, device=dev) if want_db else None
    lib = _lib.load()
    ws, nb = _workspace(lib.gwx_dense_bf16_backward_workspace(M, N, K), dev)
    _check(lib.gwx_dense_bf16_backward(_ptr(X), _ptr(W), _ptr(bias), _ptr(dY), M, N, K, act, _ptr(dX), _ptr(dW),
                                       _ptr(db), _ptr(ws), nb, _stream()))
    return dX, dW, db


def conv1d_bf16(x, W, k, addend=None, out=None):
    """Stride-1 "same" convolution z [B][T][O] (float32) of bfloat16 x [B][T][C] with
    bfloat16 W [O][k C] (tap-major rows), plus addend if given, as an implicit GEMM."""
    torch = _torch()
    _dev(x, torch.bfloat16, "x")
    _dev(W, torch.bfloat16, "W")
    B, T, C = x.shape
    O = W.shape[0]
    if addend is not None:
        _dev(addend, torch.float32, "addend")
    z = torch.empty((B, T, O), dtype=torch.float32, device=x.device) if out is None else out
    _check(_lib.load().gwx_conv1d_bf16(_ptr(x), B, T, C, int(k), _ptr(W), O, _ptr(addend), _ptr(z), _stream()))
    return z


def conv1d_bf16_backward(dz, x, W, k, addend=None, want_dx=True, want_dW=True, workspace=None):
    """(dx float32 [B][T][C] (+ addend), dW float32 [O][k C]) of z = conv1d_bf16(x, W, k)
    for dL/dz = dz (float32 [B][T][O]); either is None when not wanted."""
    torch = _torch()
    _dev(dz, torch.float32, "dz")
    _dev(x, torch.bfloat16, "x")
    _dev(W, torch.bfloat16, "W")
    B, T, C = x.shape
    O = W.shape[0]
    if addend is not None:
        _dev(addend, torch.float32, "addend")
    dev = x.device
    dx = torch.empty((B, T, C), dtype=torch.float32, device=dev) if want_dx else None
    dW = torch.empty((O, int(k) * C), dtype=torch.float32, device=dev) if want_dW else None
    lib = _lib.load()
    ws, nb = workspace if workspace is not None else _workspace(
        lib.gwx_conv1d_bf16_backward_workspace(B, T, C, O, int(k)), dev)
    _check(lib.gwx_conv1d_bf16_backward(_ptr(dz), _ptr(x), _ptr(W), B, T, C, O, int(k), _ptr(addend), _ptr(dx),
                                        _ptr(dW), _ptr(ws), nb, _stream()))
    return dx, dW


def _host3(v):
    return (ctypes.c_double * 3)(*[float(x) for x in v]) if v is not None else None


def spectral_features(y, fs, f_lo, group, F_pad, out=None):
    """bfloat16 [B][F_pad] log group powers of whitened windows y [B][D][N] (see gwx.h)."""
    torch = _torch()
    lib = _lib.load()
    _dev(y, torch.float32, "y")
    B, D, N = y.shape
    out = torch.empty((B, F_pad), dtype=torch.bfloat16, device=y.device) if out is None else out
    ws, nb = _workspace(lib.gwx_spectral_features_workspace(B, D, N), y.device)
    _check(lib.gwx_spectral_features(_ptr(y), B, D, N, fs, f_lo, group, F_pad, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def cross_features(y, fs, f_lo, group, F_pad, col0, out):
    """Writes the cross-spectral columns of whitened windows y [B][D][N] into out
    (bfloat16 [B][F_pad]) from column col0 (see gwx.h); returns out."""
    torch = _torch()
    lib = _lib.load()
    _dev(y, torch.float32, "y")
    _dev(out, torch.bfloat16, "out")
    B, D, N = y.shape
    ws, nb = _workspace(lib.gwx_spectral_features_workspace(B, D, N), y.device)
    _check(lib.gwx_cross_features(_ptr(y), B, D, N, fs, f_lo, group, F_pad, col0, _ptr(out), _ptr(ws), nb,
                                  _stream()))
    return out


def lag_features(y, fs, f_lo, group, F_pad, col0, out):
    """Writes the lag-one spectral columns of whitened windows y [B][D][N] into out
    (bfloat16 [B][F_pad]) from column col0 (see gwx.h); returns out."""
    torch = _torch()
    lib = _lib.load()
    _dev(y, torch.float32, "y")
    _dev(out, torch.bfloat16, "out")
    B, D, N = y.shape
    ws, nb = _workspace(lib.gwx_spectral_features_workspace(B, D, N), y.device)
    _check(lib.gwx_lag_features(_ptr(y), B, D, N, fs, f_lo, group, F_pad, col0, _ptr(out), _ptr(ws), nb, _stream()))
    return out


def proposal_targets(theta, mean, scale, out=None):
    """float32 [B][3] standardised (Mc, M, D) of draws theta [11][B]."""
    torch = _torch()
    _dev(theta, torch.float64, "theta")
    B = theta.shape[1]
    out = torch.empty((B, 3), dtype=torch.float32, device=theta.device) if out is None else out
    _check(_lib.load().gwx_proposal_targets(_ptr(theta), B, _host3(mean), _host3(scale), _ptr(out), _stream()))
    return out


def gauss_nll(out, targets, grad=None, loss_rows=None, loss_mean=None):
    """Gaussian NLL of targets [B][P] under network outputs out [B][ldo]: returns
    (loss_rows [B], loss_mean [1] float64 on the device, grad [B][ldo])."""
    torch = _torch()
    _dev(out, torch.float32, "out")
    _dev(targets, torch.float32, "targets")
    B, ldo = out.shape
    P = targets.shape[1]
    dev = out.device
    grad = torch.empty_like(out) if grad is None else grad
    loss_rows = torch.empty(B, dtype=torch.float32, device=dev) if loss_rows is None else loss_rows
    loss_mean = torch.empty(1, dtype=torch.float64, device=dev) if loss_mean is None else loss_mean
    _check(_lib.load().gwx_gauss_nll(_ptr(out), ldo, _ptr(targets), P, B, _ptr(loss_rows), _ptr(loss_mean),
                                     _ptr(grad), _stream()))
    return loss_rows, loss_mean, grad


def adamw(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, param_bf16=None):
    """One AdamW step in place on float32 param, m, v (step counts from 1)."""
    _check(_lib.load().gwx_adamw(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2, eps,
                                 weight_decay, step, _ptr(param_bf16), _stream()))


def adamw_at(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, param_bf16=None):
    """adamw with the step number read on the device from step (an int64 device tensor of one
    element, not modified), so that a CUDA graph can replay it."""
    torch = _torch()
    _dev(step, torch.int64, "step")
    _check(_lib.load().gwx_adamw_at(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2, eps,
                                    weight_decay, _ptr(step), _ptr(param_bf16), _stream()))


def adamw_clip(param, grad, m, v, step, lr, clip, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
               param_bf16=None):
    """One AdamW step in place with the gradients scaled to a norm of at most clip."""
    lib = _lib.load()
    ws, nb = _workspace(lib.gwx_adamw_clip_workspace(), param.device)
    _check(lib.gwx_adamw_clip(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2, eps,
                              weight_decay, step, clip, _ptr(param_bf16), _ptr(ws), nb, _stream()))


def vicreg(x, xp, lam=(1.0, 1.0, 5.0), grad_x=None, grad_xp=None):
    """VICReg loss of two views' representations x, x' [B][d] (float32): returns
    (loss [1] float64, terms [5] float64, dL/dx, dL/dx')."""
    torch = _torch()
    _dev(x, torch.float32, "x")
    _dev(xp, torch.float32, "xp")
    B, d = x.shape
    dev = x.device
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    terms = torch.empty(5, dtype=torch.float64, device=dev)
    gx = torch.empty_like(x) if grad_x is None else grad_x
    gxp = torch.empty_like(xp) if grad_xp is None else grad_xp
    _check(_lib.load().gwx_vicreg(_ptr(x), _ptr(xp), B, d, lam[0], lam[1], lam[2], _ptr(loss), _ptr(terms), _ptr(gx),
                                  _ptr(gxp), _stream()))
    return loss, terms, gx, gxp


def retime(theta, tc_lo, tc_hi, seed, counter, out=None):
    """theta [11][B] with the merger time redrawn uniformly in [tc_lo, tc_hi]."""
    torch = _torch()
    _dev(theta, torch.float64, "theta")
    out = torch.empty_like(theta) if out is None else out
    _check(_lib.load().gwx_retime(_ptr(theta), _ptr(out), theta.shape[1], tc_lo, tc_hi, seed, counter, _stream()))
    return out


def skymap(theta, nside, weights=None, out=None):
    """Normalised HEALPix (nested) map [12 nside^2] float64 of the samples' sky positions
    (rows RA, dec of theta [11][S]), each counted with its weight."""
    torch = _torch()
    lib = _lib.load()
    _dev(theta, torch.float64, "theta")
    if weights is not None:
        _dev(weights, torch.float64, "weights")
    S = theta.shape[1]
    out = torch.empty(12 * nside * nside, dtype=torch.float64, device=theta.device) if out is None else out
    ws, nb = _workspace(lib.gwx_skymap_workspace(), theta.device)
    _check(lib.gwx_skymap(_ptr(theta), _ptr(weights) if weights is not None else None, S, nside, _ptr(out), _ptr(ws),
                          nb, _stream()))
    return out


def sample_proposal(prior, truth, event_offsets, seed, counter, net_out=None, mean=None, scale=None,
                    fix_angles=False):
    """Importance-sampling draws: returns (theta [11][S] float64, log_ratio [S] float64)."""
    torch = _torch()
    _dev(truth, torch.float64, "truth")
    _dev(event_offsets, torch.int64, "event_offsets")
    E = event_offsets.shape[0] - 1
    S = int(event_offsets[-1].item())
    dev = truth.device
    theta = torch.empty((NPARAM, S), dtype=torch.float64, device=dev)
    lr = torch.empty(S, dtype=torch.float64, device=dev)
    ldn = 0
    if net_out is not None:
        _dev(net_out, torch.float32, "net_out")
        ldn = net_out.shape[1]
    p = _prior(prior)
    _check(_lib.load().gwx_sample_proposal(_ptr(net_out), ldn, _host3(mean), _host3(scale), ctypes.byref(p),
                                           _ptr(truth), E, _ptr(event_offsets), S, seed, counter,
                                           1 if fix_angles else 0, _ptr(theta), _ptr(lr), _stream()))
    return theta, lr


def gemm_autotune(A, B, out):
    """Tune the product's tile raster for this shape on these buffers (out is
    overwritten); later gemm_bf16 / dense_bf16 calls of the shape use it.  Returns the
    chosen band height."""
    torch = _torch()
    _dev(A, torch.bfloat16, "A")
    _dev(B, torch.bfloat16, "B")
    M, K = A.shape
    N = B.shape[0]
    code = {torch.float32: 0, torch.bfloat16: 1}[out.dtype]
    g = ctypes.c_int(0)
    _check(_lib.load().gwx_gemm_autotune(_ptr(A), _ptr(B), _ptr(out), M, N, K, code, ctypes.byref(g), _stream()))
    return g.value


def device_status():
    """Raise GwxError(GWX_ETIMEOUT) if a kernel gave up a bounded wait since the last
    call (synchronises the device)."""
    _check(_lib.load().gwx_device_status())


def selftest_bounded_wait(polls=256):
    """Launch a kernel whose bounded wait expires (nothing arrives at its mbarrier); the
    next device_status() raises GwxError(GWX_ETIMEOUT)."""
    _check(_lib.load().gwx_selftest_bounded_wait(int(polls), _stream()))


def rfft(x, out=None):
    torch = _torch()
    _dev(x, torch.float32, "x")
    N = x.shape[-1]
    R = x.numel() // N
    out = torch.empty(x.shape[:-1] + (N // 2 + 1,), dtype=torch.complex64, device=x.device) if out is None else out
    _check(_lib.load().gwx_rfft(_ptr(x), R, N, _ptr(out), _stream()))
    return out


def irfft(X, N, out=None):
    torch = _torch()
    _dev(X, torch.complex64, "X")
    R = X.numel() // X.shape[-1]
    out = torch.empty(X.shape[:-1] + (N,), dtype=torch.float32, device=X.device) if out is None else out
    _check(_lib.load().gwx_irfft(_ptr(X), R, N, _ptr(out), _stream()))
    return out


# ---------------------------------------------------------------- conditional coupling flow

FLOW_CROSS, FLOW_LAG = 1, 2


def flow_shape(features, group, embed_hidden, context, layers, hidden, extra=0):
    return _lib.GwxFlowShape(int(features), int(group), int(embed_hidden), int(context), int(layers), int(hidden),
                             int(extra))


def _shape(shape):
    if isinstance(shape, _lib.GwxFlowShape):
        return shape
    return flow_shape(shape["features"], shape["group"], shape["embed_hidden"], shape["context"], shape["layers"],
                      shape["hidden"], shape.get("extra", 0))


def _host8(v):
    return (ctypes.c_double * 8)(*[float(x) for x in v])


def flow_layout(shape):
    """(number of flat parameters, [offset of each tensor]) of a flow shape (see gwx.h)."""
    sh = _shape(shape)
    n = ctypes.c_int64(0)
    off = (ctypes.c_int64 * (6 + 6 * sh.layers))()
    _check(_lib.load().gwx_flow_layout(ctypes.byref(sh), ctypes.byref(n), off))
    return n.value, list(off)


def flow_targets(theta, mean8, scale8, out=None):
    """float32 [B][8] standardised flow coordinates of theta [11][B]."""
    torch = _torch()
    _dev(theta, torch.float64, "theta")
    B = theta.shape[1]
    out = torch.empty((B, 8), dtype=torch.float32, device=theta.device) if out is None else out
    _check(_lib.load().gwx_flow_targets(_ptr(theta), B, _host8(mean8), _host8(scale8), _ptr(out), _stream()))
    return out


def flow_conditioner_input(layer, v, ctx, event_offsets=None, row0=0, out=None):
    """bfloat16 [B][8 + C] conditioner input rows of layer `layer`."""
    torch = _torch()
    _dev(v, torch.float32, "v")
    _dev(ctx, torch.bfloat16, "ctx")
    B = v.shape[0]
    C = ctx.shape[1]
    E = 0
    if event_offsets is not None:
        _dev(event_offsets, torch.int64, "event_offsets")
        E = event_offsets.shape[0] - 1
    out = torch.empty((B, 8 + C), dtype=torch.bfloat16, device=v.device) if out is None else out
    _check(_lib.load().gwx_flow_conditioner_input(layer, _ptr(v), _ptr(ctx), C, _ptr(event_offsets), E, row0, B,
                                                  _ptr(out), _stream()))
    return out


def flow_coupling(layer, direction, v_in, o, sum_s, init, v_out=None):
    """One coupling step (direction +1 sampling, -1 density); returns v_out [B][8]."""
    torch = _torch()
    _dev(v_in, torch.float32, "v_in")
    _dev(o, torch.float32, "o")
    _dev(sum_s, torch.float32, "sum_s")
    v_out = torch.empty_like(v_in) if v_out is None else v_out
    _check(_lib.load().gwx_flow_coupling(layer, direction, _ptr(v_in), _ptr(o), v_in.shape[0], _ptr(v_out),
                                         _ptr(sum_s), 1 if init else 0, _stream()))
    return v_out


def flow_nll(z, sum_s):
    """(loss_rows [B] float32, loss_mean [1] float64, grad [B][8] = z / B)."""
    torch = _torch()
    _dev(z, torch.float32, "z")
    _dev(sum_s, torch.float32, "sum_s")
    B = z.shape[0]
    rows = torch.empty(B, dtype=torch.float32, device=z.device)
    mean = torch.empty(1, dtype=torch.float64, device=z.device)
    grad = torch.empty_like(z)
    _check(_lib.load().gwx_flow_nll(_ptr(z), _ptr(sum_s), B, _ptr(rows), _ptr(mean), _ptr(grad), _stream()))
    return rows, mean, grad


def flow_coupling_backward(layer, w, o, g, row_weight):
    """(d_o [B][8], g_u [B][8]) of a density step (see gwx.h)."""
    torch = _torch()
    for t, n in ((w, "w"), (o, "o"), (g, "g")):
        _dev(t, torch.float32, n)
    d_o, g_u = torch.empty_like(o), torch.empty_like(g)
    _check(_lib.load().gwx_flow_coupling_backward(layer, _ptr(w), _ptr(o), _ptr(g), w.shape[0], float(row_weight),
                                                  _ptr(d_o), _ptr(g_u), _stream()))
    return d_o, g_u


def flow_input_backward(layer, dX, g_u, d_ctx, init):
    """In place: g_u[:, a] += dX[:, 0:4]; d_ctx (=, or += unless init) dX[:, 8:]."""
    torch = _torch()
    for t, n in ((dX, "dX"), (g_u, "g_u"), (d_ctx, "d_ctx")):
        _dev(t, torch.float32, n)
    _check(_lib.load().gwx_flow_input_backward(layer, _ptr(dX), d_ctx.shape[1], dX.shape[0], _ptr(g_u), _ptr(d_ctx),
                                               1 if init else 0, _stream()))


def flow_base(seed, counter, row0, n):
    """float32 [n][8] base normals of global draws row0 .. row0 + n - 1."""
    torch = _torch()
    z = torch.empty((n, 8), dtype=torch.float32, device=torch.device("cuda", torch.cuda.current_device()))
    _check(_lib.load().gwx_flow_base(seed, counter, row0, n, _ptr(z), _stream()))
    return z


def flow_proposal(x, z, sum_s, mean8, scale8, prior, seed, counter):
    """(theta [11][S], log_q [S], log_ratio [S]) of flow draws x with base z and sum_s
    (spins and t_c drawn from the prior)."""
    torch = _torch()
    _dev(x, torch.float32, "x")
    _dev(z, torch.float32, "z")
    _dev(sum_s, torch.float32, "sum_s")
    S = x.shape[0]
    dev = x.device
    theta = torch.empty((NPARAM, S), dtype=torch.float64, device=dev)
    log_q, lr = (torch.empty(S, dtype=torch.float64, device=dev) for _ in range(2))
    p = _prior(prior)
    _check(_lib.load().gwx_flow_proposal(_ptr(x), _ptr(z), _ptr(sum_s), S, _host8(mean8), _host8(scale8),
                                         ctypes.byref(p), seed, counter, _ptr(theta), _ptr(log_q), _ptr(lr),
                                         _stream()))
    return theta, log_q, lr


def flow_train_step(shape, params, params_bf16, grads, m, v, step, lr, mean8, scale8, y, theta, fs, f_lo,
                    beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, clip=0.0, loss_mean=None, workspace=None,
                    step_counter=None, ctx=None, d_ctx=None):
    """One training step (step 0: loss and gradients only).  Returns loss_mean (device
    float64 [1]).  `workspace` may be a preallocated (tensor, bytes) pair.  With ctx
    (bfloat16 [B][C]) the context comes from the caller's summary network and d_ctx
    (float32 [B][C]) receives its gradient."""
    torch = _torch()
    sh = _shape(shape)
    _dev(y, torch.float32, "y")
    _dev(theta, torch.float64, "theta")
    B, D, N = y.shape
    lib = _lib.load()
    loss_mean = torch.empty(1, dtype=torch.float64, device=y.device) if loss_mean is None else loss_mean
    ws, nb = workspace if workspace is not None else _workspace(
        lib.gwx_flow_train_workspace(ctypes.byref(sh), B, D, N), y.device)
    _check(lib.gwx_flow_train_step(ctypes.byref(sh), _ptr(params), _ptr(params_bf16), _ptr(grads), _ptr(m), _ptr(v),
                                   step, _ptr(step_counter) if step_counter is not None else None, lr, beta1, beta2,
                                   eps, weight_decay, clip, _host8(mean8), _host8(scale8), _ptr(y), _ptr(theta), B, D,
                                   N, fs, f_lo, _ptr(ctx) if ctx is not None else None,
                                   _ptr(d_ctx) if d_ctx is not None else None, _ptr(loss_mean), _ptr(ws), nb,
                                   _stream()))
    return loss_mean


def flow_log_prob(shape, params, params_bf16, mean8, scale8, y, theta, fs, f_lo, ctx=None):
    """float64 [B] ln q_r(r(theta_b) | y_b)."""
    torch = _torch()
    sh = _shape(shape)
    _dev(y, torch.float32, "y")
    _dev(theta, torch.float64, "theta")
    B, D, N = y.shape
    lib = _lib.load()
    out = torch.empty(B, dtype=torch.float64, device=y.device)
    ws, nb = _workspace(lib.gwx_flow_log_prob_workspace(ctypes.byref(sh), B, D, N), y.device)
    _check(lib.gwx_flow_log_prob(ctypes.byref(sh), _ptr(params), _ptr(params_bf16), _host8(mean8), _host8(scale8),
                                 _ptr(y), _ptr(theta), B, D, N, fs, f_lo, _ptr(ctx) if ctx is not None else None,
                                 _ptr(out), _ptr(ws), nb, _stream()))
    return out


def sample_posterior(shape, params, params_bf16, mean8, scale8, prior, y, fs, f_lo, event_offsets, seed,
                     counter, out=None, workspace=None, ctx=None, S=None):
    """Posterior draws for events y [E][D][N]: (theta [11][S], log_q [S], log_ratio [S]);
    spins and t_c (not modelled by the flow) are drawn from the prior.  S (the total
    number of draws, event_offsets[-1]) is read from the device when not given."""
    torch = _torch()
    sh = _shape(shape)
    _dev(y, torch.float32, "y")
    _dev(event_offsets, torch.int64, "event_offsets")
    E, D, N = y.shape
    S = int(event_offsets[-1].item()) if S is None else int(S)
    dev = y.device
    lib = _lib.load()
    if out is None:
        out = (torch.empty((NPARAM, S), dtype=torch.float64, device=dev),
               torch.empty(S, dtype=torch.float64, device=dev), torch.empty(S, dtype=torch.float64, device=dev))
    theta, log_q, lr = out
    ws, nb = workspace if workspace is not None else _workspace(
        lib.gwx_sample_posterior_workspace(ctypes.byref(sh), E, D, N, S), dev)
    p = _prior(prior)
    _check(lib.gwx_sample_posterior(ctypes.byref(sh), _ptr(params), _ptr(params_bf16), _host8(mean8), _host8(scale8),
                                    ctypes.byref(p), _ptr(y), E, D, N, fs, f_lo,
                                    _ptr(ctx) if ctx is not None else None, _ptr(event_offsets), S,
                                    seed, counter, _ptr(theta), _ptr(log_q), _ptr(lr), _ptr(ws), nb, _stream()))
    return theta, log_q, lr


def flow_skymap(shape, params, params_bf16, mean8, scale8, y, fs, f_lo, theta, log_q, nside, ctx=None, out=None):
    """The flow's sky density (float64 [12 nside^2], nested HEALPix order, unit sum) for
    one event y [1][D][N]: RA and sin dec at each pixel centre, the other coordinates at
    the draw of largest log_q among theta [11][S]."""
    torch = _torch()
    sh = _shape(shape)
    _dev(y, torch.float32, "y")
    _dev(theta, torch.float64, "theta")
    _dev(log_q, torch.float64, "log_q")
    _, D, N = y.shape
    S = theta.shape[1]
    lib = _lib.load()
    out = torch.empty(12 * nside * nside, dtype=torch.float64, device=y.device) if out is None else out
    ws, nb = _workspace(lib.gwx_flow_skymap_workspace(ctypes.byref(sh), D, N, nside), y.device)
    _check(lib.gwx_flow_skymap(ctypes.byref(sh), _ptr(params), _ptr(params_bf16), _host8(mean8), _host8(scale8),
                               _ptr(y), D, N, fs, f_lo, _ptr(ctx) if ctx is not None else None, _ptr(theta),
                               _ptr(log_q), S, int(nside), _ptr(out), _ptr(ws), nb, _stream()))
    return out


__all__ += ["flow_shape", "flow_layout", "flow_targets", "flow_conditioner_input", "flow_coupling", "flow_nll",
            "flow_coupling_backward", "flow_input_backward", "flow_base", "flow_proposal", "flow_train_step",
            "flow_log_prob", "sample_posterior", "flow_skymap"]

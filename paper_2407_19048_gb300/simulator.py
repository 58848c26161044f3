"""On-the-fly training-data generator built on the libgwx C ABI.

Sec. 3.2 describes the workflow this class runs: a background chunk resident on
the device with its power spectrum fitted to it, then for every batch N prior
draws, their waveforms, N background crops, injection and whitening.  One
``step(i)`` is four C-ABI calls:

1. ``prepare_batch``     -- prior draws and the FP64 per-draw set-up, on a side
   stream (it occupies few SMs, so it runs alongside 2 and 3);
2. ``colored_noise``     -- a fresh synthetic background stretch (stand-in for the
   paper's real strain chunk), or ``set_background`` to use caller data;
3. ``welch_psd``         -- the PSD fitted to that stretch;
4. ``simulate_prepared`` -- waveforms, projection, crops, injection and
   whitening, fused per draw, after the side stream's work (event wait).

All buffers and workspaces are allocated once, so a step performs no
allocation and no host synchronisation.
"""
import ctypes

from . import _lib
from . import DETECTORS, NPARAM, _det_ids, _prior, _ptr, _stream, _workspace, _check


class Simulator:
    def __init__(self, workload, device=None, noise_on_device=True):
        import torch
        self.wl = dict(workload)
        wl = self.wl
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.lib = _lib.load()
        self.D = len(wl["dets"])
        self.B, self.N, self.L = int(wl["B"]), int(wl["N"]), int(wl["L"])
        self.M, self.stride = int(wl["seg_len"]), int(wl["seg_stride"])
        self.fs, self.f_lo = float(wl["fs"]), float(wl["f_lo"])
        self.gmst = float(wl.get("gmst", 0.0))
        self.ids, _ = _det_ids(wl["dets"])
        self.prior = _prior(wl["prior"])
        self.noise_on_device = noise_on_device
        f32, f64 = torch.float32, torch.float64
        self.noise = torch.empty((self.D, self.L), dtype=f32, device=self.dev)
        self.psd = torch.empty((self.D, self.M // 2 + 1), dtype=f64, device=self.dev)
        self.y = torch.empty((self.B, self.D, self.N), dtype=f32, device=self.dev)
        self.theta = torch.empty((NPARAM, self.B), dtype=f64, device=self.dev)
        self.offsets = torch.empty(self.B, dtype=torch.int64, device=self.dev)
        lib = self.lib
        self.ws_noise = _workspace(lib.gwx_colored_noise_workspace(self.D, self.L), self.dev)
        self.ws_welch = _workspace(lib.gwx_welch_psd_workspace(self.D, self.L, self.M, self.stride), self.dev)
        self.ws_sim = _workspace(lib.gwx_simulate_batch_workspace(self.D, self.B, self.N), self.dev)
        self.side = torch.cuda.Stream(device=self.dev)
        self.ev_start = torch.cuda.Event()
        self.ev_prep = torch.cuda.Event()
        _check(lib.gwx_init())

    # kernels one step launches: prepare 2, colored noise 3, Welch 2, simulate_prepared 2
    LAUNCHES_PER_STEP = 9

    def set_background(self, strain):
        """Use caller strain [D][L] (device float32) as the background of later steps."""
        self.noise.copy_(strain)
        self.noise_on_device = False

    def background(self, step):
        lib, s = self.lib, _stream()
        if self.noise_on_device:
            ws, nb = self.ws_noise
            _check(lib.gwx_colored_noise(int(self.wl["noise_seed"]), step & 0xFFFFFFFF, self.D, self.L, self.fs,
                                         self.f_lo, _ptr(self.noise), _ptr(ws), nb, s))
        ws, nb = self.ws_welch
        _check(lib.gwx_welch_psd(_ptr(self.noise), self.D, self.L, self.fs, self.M, self.stride, _ptr(self.psd),
                                 _ptr(ws), nb, s))

    def prepare(self, step):
        ws, nb = self.ws_sim
        _check(self.lib.gwx_prepare_batch(ctypes.byref(self.prior), int(self.wl["param_seed"]), step & 0xFFFFFFFF,
                                          self.L, self.N, self.fs, self.f_lo, self.ids, self.D, self.gmst, self.B,
                                          _ptr(self.theta), _ptr(self.offsets), _ptr(ws), nb, _stream()))

    def simulate_prepared(self):
        ws, nb = self.ws_sim
        _check(self.lib.gwx_simulate_prepared(_ptr(self.noise), self.L, _ptr(self.psd), self.M, self.fs, self.f_lo,
                                              self.D, self.B, self.N, _ptr(self.offsets), _ptr(self.y), _ptr(ws),
                                              nb, _stream()))

    def simulate(self, step):
        """prepare + simulate_prepared on the current stream (the single-call gwx_simulate_batch)."""
        ws, nb = self.ws_sim
        _check(self.lib.gwx_simulate_batch(ctypes.byref(self.prior), int(self.wl["param_seed"]), step & 0xFFFFFFFF,
                                           _ptr(self.noise), self.L, _ptr(self.psd), self.M, self.fs, self.f_lo,
                                           self.ids, self.D, self.gmst, self.B, self.N, _ptr(self.y),
                                           _ptr(self.theta), _ptr(self.offsets), _ptr(ws), nb, _stream()))

    def step(self, step, mark=None):
        """One batch: returns (y [B][D][N], theta [11][B], offsets [B]) (device tensors, reused).

        The preparation runs on the side stream after everything already queued on the
        current stream (so earlier readers of theta/offsets are done); the fused pass
        waits for it.  ``mark``, if given, is recorded on the current stream after the
        background and PSD."""
        import torch
        main = torch.cuda.current_stream(self.dev)
        self.ev_start.record(main)
        self.side.wait_event(self.ev_start)
        with torch.cuda.stream(self.side):
            self.prepare(step)
            self.ev_prep.record(self.side)
        self.background(step)
        if mark is not None:
            mark.record(main)
        main.wait_event(self.ev_prep)
        self.simulate_prepared()
        return self.y, self.theta, self.offsets


__all__ = ["Simulator", "DETECTORS"]

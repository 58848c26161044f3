"""On-the-fly training-data generator built on the libgwx C ABI.

Sec. 3.2 describes the workflow this class runs: a background chunk resident on
the device with its power spectrum fitted to it, then for every batch N prior
draws, their waveforms, N background crops, injection and whitening.  One
``step(i)`` is up to four C-ABI calls:

1. ``prepare_batch``     -- prior draws and the FP64 per-draw set-up, on a side
   stream;
2. ``colored_noise``     -- a fresh synthetic background stretch (stand-in for the
   paper's real strain chunk), or ``set_background`` to use caller data;
3. ``welch_psd``         -- the PSD fitted to that stretch;
4. ``simulate_prepared`` -- waveforms, projection, crops, injection and
   whitening, fused per draw, after the side stream's work (event wait).

2 and 3 run every ``background_every`` batches (the paper keeps one background
for many batches).  With ``pipeline=True`` the side stream prepares batch i + 1
while batch i's fused pass runs (two buffer sets, used alternately), so the
latency-bound FP64 set-up overlaps the previous pass instead of delaying the next;
the passes then run on a high-priority stream so the preparation fills the SMs the
fused pass leaves idle rather than taking them first.
All buffers and workspaces are allocated once: a step performs no allocation and
no host synchronisation.
"""
import ctypes

from . import _lib
from . import DETECTORS, NPARAM, _det_ids, _prior, _ptr, _stream, _workspace, _check


class Simulator:
    # kernels per call: prepare 2, colored noise 2, Welch 2, simulate_prepared 2 (1 when the
    # whitening filter of its workspace is still current)
    LAUNCHES = {"prepare": 2, "colored_noise": 2, "welch": 2, "simulate": 2, "simulate_reuse": 1}

    def __init__(self, workload, device=None, noise_on_device=True, pipeline=False, background_every=1):
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
        self.pipeline = bool(pipeline)
        self.background_every = max(1, int(background_every))
        f32, f64 = torch.float32, torch.float64
        nbuf = 2 if self.pipeline else 1
        self.noise = torch.empty((self.D, self.L), dtype=f32, device=self.dev)
        self.psd = torch.empty((self.D, self.M // 2 + 1), dtype=f64, device=self.dev)
        self._y = [torch.empty((self.B, self.D, self.N), dtype=f32, device=self.dev) for _ in range(nbuf)]
        self._theta = [torch.empty((NPARAM, self.B), dtype=f64, device=self.dev) for _ in range(nbuf)]
        self._offsets = [torch.empty(self.B, dtype=torch.int64, device=self.dev) for _ in range(nbuf)]
        lib = self.lib
        self.ws_noise = _workspace(lib.gwx_colored_noise_workspace(self.D, self.L), self.dev)
        self.ws_welch = _workspace(lib.gwx_welch_psd_workspace(self.D, self.L, self.M, self.stride), self.dev)
        self._ws_sim = [_workspace(lib.gwx_simulate_batch_workspace(self.D, self.B, self.N), self.dev)
                        for _ in range(nbuf)]
        self.side = torch.cuda.Stream(device=self.dev)
        # pipelined passes run on a high-priority stream, so that when both are pending
        # the block scheduler dispatches the fused pass before the next batch's preparation
        self.work = torch.cuda.Stream(device=self.dev, priority=-1) if self.pipeline else None
        self.ev_start = torch.cuda.Event()
        self.ev_done = torch.cuda.Event()
        self._ev_prep = [torch.cuda.Event() for _ in range(nbuf)]
        self._slot = 0
        self._psd_version = 0     # incremented whenever the PSD is recomputed
        self._filter_version = [-1] * nbuf   # PSD version each workspace's whitening filter was built from
        self._ready = None        # step counter already prepared in the current slot (pipeline)
        self._since_bg = None     # batches since the last background
        self.launches = 0         # kernels launched so far (all calls of this object)
        _check(lib.gwx_init())

    # current buffer set (the one the last or next step uses)
    @property
    def y(self):
        return self._y[self._slot]

    @property
    def theta(self):
        return self._theta[self._slot]

    @property
    def offsets(self):
        return self._offsets[self._slot]

    @property
    def ws_sim(self):
        return self._ws_sim[self._slot]

    def set_background(self, strain):
        """Use caller strain [D][L] (device float32) as the background of later steps."""
        self.noise.copy_(strain)
        self.noise_on_device = False
        self._since_bg = None

    def background(self, step):
        lib, s = self.lib, _stream()
        if self.noise_on_device:
            ws, nb = self.ws_noise
            _check(lib.gwx_colored_noise(int(self.wl["noise_seed"]), step & 0xFFFFFFFF, self.D, self.L, self.fs,
                                         self.f_lo, _ptr(self.noise), _ptr(ws), nb, s))
            self.launches += self.LAUNCHES["colored_noise"]
        ws, nb = self.ws_welch
        _check(lib.gwx_welch_psd(_ptr(self.noise), self.D, self.L, self.fs, self.M, self.stride, _ptr(self.psd),
                                 _ptr(ws), nb, s))
        self.launches += self.LAUNCHES["welch"]
        self._psd_version += 1

    def prepare(self, step, slot=None):
        slot = self._slot if slot is None else slot
        ws, nb = self._ws_sim[slot]
        _check(self.lib.gwx_prepare_batch(ctypes.byref(self.prior), int(self.wl["param_seed"]), step & 0xFFFFFFFF,
                                          self.L, self.N, self.fs, self.f_lo, self.ids, self.D, self.gmst, self.B,
                                          _ptr(self._theta[slot]), _ptr(self._offsets[slot]), _ptr(ws), nb,
                                          _stream()))
        self.launches += self.LAUNCHES["prepare"]

    def simulate_prepared(self, slot=None):
        slot = self._slot if slot is None else slot
        ws, nb = self._ws_sim[slot]
        ready = self._filter_version[slot] == self._psd_version
        _check(self.lib.gwx_simulate_prepared(_ptr(self.noise), self.L, _ptr(self.psd), self.M, self.fs, self.f_lo,
                                              self.D, self.B, self.N, _ptr(self._offsets[slot]),
                                              _ptr(self._y[slot]), 1 if ready else 0, _ptr(ws), nb, _stream()))
        self._filter_version[slot] = self._psd_version
        self.launches += self.LAUNCHES["simulate_reuse" if ready else "simulate"]

    def simulate(self, step):
        """prepare + simulate_prepared on the current stream (the single-call gwx_simulate_batch)."""
        ws, nb = self.ws_sim
        _check(self.lib.gwx_simulate_batch(ctypes.byref(self.prior), int(self.wl["param_seed"]), step & 0xFFFFFFFF,
                                           _ptr(self.noise), self.L, _ptr(self.psd), self.M, self.fs, self.f_lo,
                                           self.ids, self.D, self.gmst, self.B, self.N, _ptr(self.y),
                                           _ptr(self.theta), _ptr(self.offsets), _ptr(ws), nb, _stream()))
        self._filter_version[self._slot] = self._psd_version
        self.launches += self.LAUNCHES["prepare"] + self.LAUNCHES["simulate"]

    def autotune(self, step=0):
        """Time the fused pass's launch shapes (bit-identical outputs) on a batch of this
        simulator's workload and record the fastest for its (N, D); returns the shape.
        Synchronises; call it before timing or capturing steps."""
        import torch
        if self._since_bg is None:
            self.background(step)
            self._since_bg = 0
        slot = self._slot
        self.prepare(step, slot)
        ws, nb = self._ws_sim[slot]
        shape = ctypes.c_int(-1)
        _check(self.lib.gwx_simulate_autotune(_ptr(self.noise), self.L, _ptr(self.psd), self.M, self.fs, self.f_lo,
                                              self.D, self.B, self.N, _ptr(self._offsets[slot]), _ptr(self._y[slot]),
                                              _ptr(ws), nb, ctypes.byref(shape), _stream()))
        self._filter_version[slot] = self._psd_version
        self._ready = None
        torch.cuda.current_stream(self.dev).synchronize()
        return shape.value

    def step(self, step, mark=None):
        """One batch: returns (y [B][D][N], theta [11][B], offsets [B]) (device tensors).

        Preparations run on the side stream after everything already queued on the
        current stream (so earlier readers of the buffers they overwrite are done);
        the fused pass waits for them.  The background is regenerated on the first
        step and then every ``background_every`` steps.  With ``pipeline`` the returned
        tensors alternate between two buffer sets: batch i stays valid until step i + 2
        is called.  ``mark``, if given, is recorded on the current stream after the
        background, the PSD and the wait for the preparation, just before the fused
        pass."""
        import torch
        caller = torch.cuda.current_stream(self.dev)
        self.ev_start.record(caller)
        self.side.wait_event(self.ev_start)
        main = self.work if self.pipeline else caller
        if main is not caller:
            main.wait_event(self.ev_start)
        slot = self._slot
        if not self.pipeline or self._ready != step:
            with torch.cuda.stream(self.side):
                self.prepare(step, slot)
                self._ev_prep[slot].record(self.side)
        with torch.cuda.stream(main):
            if self._since_bg is None or self._since_bg >= self.background_every:
                self.background(step)
                self._since_bg = 0
            self._since_bg += 1
            main.wait_event(self._ev_prep[slot])
            if mark is not None:
                mark.record(main)
            self.simulate_prepared(slot)
        if main is not caller:
            self.ev_done.record(main)
            caller.wait_event(self.ev_done)
        out = (self._y[slot], self._theta[slot], self._offsets[slot])
        if self.pipeline:
            nxt = 1 - slot
            with torch.cuda.stream(self.side):
                self.prepare(step + 1, nxt)
                self._ev_prep[nxt].record(self.side)
            self._ready = step + 1
            self._slot = nxt
        return out


__all__ = ["Simulator", "DETECTORS"]

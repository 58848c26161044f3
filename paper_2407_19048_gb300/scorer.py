"""Low-latency scoring of single events (the serving side of the likelihood path).

An event arrives as a whitened window y [D][N]; the scorer draws S samples from a
proposal (the prior, or a trained `flow.FlowPosterior` through `gwx_sample_posterior`),
scores them with the standard likelihood (Sec. 6; optionally with the merger time
integrated out, `gwx_log_likelihood_tmarg`) and weighs them, then reads the
event's effective sample size and evidence back to the host.  Every buffer and workspace is allocated once
for the largest S, the calls go straight to the C ABI on one stream, and the only host
synchronisation is the final read of two doubles from pinned memory.
"""
import ctypes

from . import _lib
from . import NPARAM, _check, _det_ids, _prior, _ptr, _workspace


class Scorer:
    def __init__(self, workload, max_samples, psd, device=None, seed=55, flow=None, tmarg=None):
        import torch
        self.wl = dict(workload)
        wl = self.wl
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.lib = _lib.load()
        self.D, self.N, self.L = len(wl["dets"]), int(wl["N"]), int(wl["L"])
        self.M, self.fs, self.f_lo = int(wl["seg_len"]), float(wl["fs"]), float(wl["f_lo"])
        self.ids, _ = _det_ids(wl["dets"])
        self.prior = _prior(wl["prior"])
        self.seed = int(seed)
        self.psd = psd
        self.smax = int(max_samples)
        f64 = torch.float64
        self.theta = torch.empty(NPARAM * self.smax, dtype=f64, device=self.dev)
        self.offsets_draw = torch.empty(self.smax, dtype=torch.int64, device=self.dev)
        self.lnl = torch.empty(self.smax, dtype=f64, device=self.dev)
        self.w = torch.empty(self.smax, dtype=f64, device=self.dev)
        self.out = torch.empty(4, dtype=f64, device=self.dev)          # ess, efficiency, ln Z, spare
        self.host = torch.empty(4, dtype=f64, pin_memory=True)
        self.ev = torch.empty(2, dtype=torch.int64, device=self.dev)
        self.ev_host = torch.empty(2, dtype=torch.int64, pin_memory=True)
        self.ws_ll = _workspace(self.lib.gwx_log_likelihood_workspace(1, self.D, self.N, self.smax), self.dev)
        self.ws_iw = _workspace(self.lib.gwx_importance_weights_workspace(1), self.dev)
        self.flow = flow
        # (tc_lo, n_tc, oversample): score with the merger time integrated out over that grid
        self.tmarg = None if tmarg is None else (float(tmarg[0]), int(tmarg[1]), int(tmarg[2]))
        if flow is not None:
            from . import _shape
            self.shape = _shape(flow.shape)
            self.ws_fl = _workspace(self.lib.gwx_sample_posterior_workspace(ctypes.byref(self.shape), 1, self.D, self.N,
                                                                            self.smax), self.dev)
            self.log_q = torch.empty(self.smax, dtype=f64, device=self.dev)
            self.log_ratio = torch.empty(self.smax, dtype=f64, device=self.dev)
            self.mean8 = (ctypes.c_double * 8)(*flow.mean)
            self.scale8 = (ctypes.c_double * 8)(*flow.scale)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.done = torch.cuda.Event()

    def score(self, y_event, S, step):
        """(ess, efficiency, ln_evidence) of one event y_event [D][N] (device float32)
        from S samples drawn with Philox counter `step`: from the prior, or from the flow
        (whose draws take the spins and merger time, which it does not model, from the
        prior)."""
        import torch
        if S > self.smax:
            raise ValueError("S exceeds max_samples")
        lib, s = self.lib, ctypes.c_void_p(self.stream.cuda_stream)
        self.stream.wait_stream(torch.cuda.current_stream(self.dev))
        self.ev_host[0], self.ev_host[1] = 0, S
        with torch.cuda.stream(self.stream):
            self.ev.copy_(self.ev_host, non_blocking=True)
        theta = ctypes.c_void_p(self.theta.data_ptr())
        ratio = None
        if self.flow is None:
            _check(lib.gwx_sample_prior(ctypes.byref(self.prior), self.seed, step & 0xFFFFFFFF, S, self.L, self.N,
                                        theta, _ptr(self.offsets_draw), s))
        else:
            ws, nb = self.ws_fl
            fp = self.flow
            _check(lib.gwx_sample_posterior(ctypes.byref(self.shape), _ptr(fp.params), _ptr(fp.params16), self.mean8,
                                            self.scale8, ctypes.byref(self.prior), _ptr(y_event), 1, self.D, self.N,
                                            self.fs, self.f_lo, None, _ptr(self.ev), S, self.seed,
                                            step & 0xFFFFFFFF, theta, _ptr(self.log_q), _ptr(self.log_ratio),
                                            _ptr(ws), nb, s))
            ratio = _ptr(self.log_ratio)
        ws, nb = self.ws_ll
        if self.tmarg is None:
            _check(lib.gwx_log_likelihood(0, _ptr(y_event), 1, self.D, self.N, _ptr(self.psd), self.M, self.fs,
                                          self.f_lo, self.ids, 0.0, theta, _ptr(self.ev), S, _ptr(self.lnl), _ptr(ws),
                                          nb, s))
        else:
            tc_lo, n_tc, u = self.tmarg
            _check(lib.gwx_log_likelihood_tmarg(0, _ptr(y_event), 1, self.D, self.N, _ptr(self.psd), self.M, self.fs,
                                                self.f_lo, self.ids, 0.0, tc_lo, n_tc, u, theta, _ptr(self.ev), S,
                                                _ptr(self.lnl), _ptr(ws), nb, s))
        ws, nb = self.ws_iw
        o = self.out.data_ptr()
        _check(lib.gwx_importance_weights(_ptr(self.lnl), ratio, _ptr(self.ev), 1, S, _ptr(self.w),
                                          ctypes.c_void_p(o), ctypes.c_void_p(o + 8), ctypes.c_void_p(o + 16),
                                          _ptr(ws), nb, s))
        with torch.cuda.stream(self.stream):
            self.host.copy_(self.out, non_blocking=True)
            self.done.record(self.stream)
        self.done.synchronize()
        return float(self.host[0]), float(self.host[1]), float(self.host[2])


__all__ = ["Scorer"]

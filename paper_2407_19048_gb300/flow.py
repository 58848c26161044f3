"""The conditional coupling flow as a trainable posterior estimator.

Sec. 5 of the paper trains a normalizing flow q(theta | d) on the simulated batches by
maximising ln q(theta_i | d_i) with AdamW, conditioned on a summary of the whitened
strain (Sec. 4), and then draws posterior samples for new data; Sec. 6 judges those
samples with the standard likelihood.  `FlowPosterior` holds the flow's parameters as
one flat FP32 array with its bfloat16 copy and AdamW moments (the layout of
`gwx_flow_layout`), and drives three library calls: `flow_train_step` (features,
embedding, the K coupling layers in the density direction, loss, backward, AdamW: one
C-ABI call), `sample_posterior` (draws with ln q and the prior-to-proposal log ratio
for importance sampling) and `log_prob`.
"""
import math

from . import _lib


class FlowPosterior:
    def __init__(self, workload, layers=16, hidden=256, context=64, embed_hidden=512, group=4, seed=0,
                 device=None, lr=1e-3, weight_decay=2e-3, cross=True, lag=True, clip=1.0, embedding="spectral",
                 resnet_stages=None):
        import torch
        import paper_2407_19048_gb300 as gwx
        self.gwx = gwx
        self.wl = dict(workload)
        wl = self.wl
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.D, self.N, self.fs, self.f_lo = len(wl["dets"]), int(wl["N"]), float(wl["fs"]), float(wl["f_lo"])
        k_lo = math.ceil(self.f_lo * self.N / self.fs - 1e-9)
        ng = (self.N // 2 - k_lo) // group
        cross = 1 if (cross and self.D > 1) else 0
        lag = 1 if lag else 0
        cols = self.D * ng * (1 + (self.D - 1) * cross + 2 * lag)
        F = ((cols + 7) // 8) * 8
        self.shape = {"features": F, "group": group, "embed_hidden": embed_hidden, "context": context,
                      "layers": layers, "hidden": hidden, "extra": gwx.FLOW_CROSS * cross + gwx.FLOW_LAG * lag}
        self.n_params, self.offsets = gwx.flow_layout(self.shape)
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device=self.dev)
        self.params16 = torch.zeros(self.n_params, dtype=torch.bfloat16, device=self.dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.lr, self.wd, self.clip = float(lr), float(weight_decay), float(clip)
        self.steps = 0
        self._ws = {}
        self._loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.init_random(seed)
        # standardisation of the flow's coordinates from prior draws (computed by the library)
        # the data summary: the built-in dense network on spectral features, or the
        # ResNet-1D of Sec. 4 on the whitened strain (trained here, its context fed in)
        self.embedding = embedding
        self.resnet = None
        if embedding == "resnet":
            from .resnet import ResNet1D, STAGES
            self.resnet = ResNet1D(self.D, context, stages=resnet_stages or STAGES, device=self.dev, seed=seed + 1)
            self.rmom = {name: (torch.zeros_like(p), torch.zeros_like(p)) for name, p, _ in self.resnet.tensors()}
        elif embedding != "spectral":
            raise ValueError("embedding must be 'spectral' or 'resnet'")
        th, _ = gwx.sample_prior(wl["prior"], 12345, 0, 100000, wl["L"], self.N)
        r = gwx.flow_targets(th, [0.0] * 8, [1.0] * 8).double()
        self.mean = [float(x) for x in r.mean(dim=0).cpu()]
        self.scale = [float(x) for x in r.std(dim=0).cpu()]

    # ------------------------------------------------------------ parameters
    def tensor_shapes(self):
        sh = self.shape
        F, He, C, H = sh["features"], sh["embed_hidden"], sh["context"], sh["hidden"]
        out = [(He, F), (He,), (He, He), (He,), (C, He), (C,)]
        for _ in range(sh["layers"]):
            out += [(H, 8 + C), (H,), (H, H), (H,), (8, H), (8,)]
        return out

    def tensor(self, t, bf16=False):
        """View of parameter tensor t (storage order) in the flat array."""
        shape = self.tensor_shapes()[t]
        n = 1
        for s in shape:
            n *= s
        base = self.params16 if bf16 else self.params
        return base[self.offsets[t]:self.offsets[t] + n].view(shape)

    def set_tensors(self, arrays):
        """Load parameter tensors (storage order; numpy or torch) and refresh the copy."""
        import torch
        for t, a in enumerate(arrays):
            self.tensor(t).copy_(torch.as_tensor(a, dtype=torch.float32))
        self.params16.copy_(self.params.to(torch.bfloat16))

    def init_random(self, seed):
        """Weights N(0, 1 / fan_in), the last layer of each conditioner scaled by 0.01 (the
        flow starts near the identity), biases zero."""
        import torch
        g = torch.Generator(device=self.dev)
        g.manual_seed(int(seed))
        self.params.zero_()
        for t, shape in enumerate(self.tensor_shapes()):
            if len(shape) == 2:
                gain = 0.01 if (t >= 6 and t % 6 == 4) else 1.0
                w = torch.randn(shape, generator=g, device=self.dev) * (gain / math.sqrt(shape[1]))
                self.tensor(t).copy_(w)
        self.params16.copy_(self.params.to(torch.bfloat16))

    def _workspace(self, key, nbytes):
        import paper_2407_19048_gb300 as gwx
        if key not in self._ws or self._ws[key][1] < nbytes:
            self._ws[key] = gwx._workspace(nbytes, self.dev)
        return self._ws[key]

    # ------------------------------------------------------------ training and use
    def train_step(self, y, theta, update=True):
        """One AdamW step (or, with update False, the loss and gradients only) on a
        simulated batch y [B][D][N] with parameters theta [11][B]; returns the batch-mean
        loss as a device tensor (no host synchronisation)."""
        import ctypes
        gwx = self.gwx
        B = y.shape[0]
        sh = gwx._shape(self.shape)
        nb = _lib.load().gwx_flow_train_workspace(ctypes.byref(sh), B, self.D, self.N)
        ws = self._workspace(("train", B), nb)
        step = self.steps + 1 if update else 0
        ctx = d_ctx = None
        if self.resnet is not None:
            import torch
            ctx = self.resnet.forward(y, out_dtype=torch.bfloat16)
            d_ctx = torch.empty(ctx.shape, dtype=torch.float32, device=self.dev)
        gwx.flow_train_step(self.shape, self.params, self.params16, self.grads, self.m, self.v, step, self.lr,
                            self.mean, self.scale, y, theta, self.fs, self.f_lo, weight_decay=self.wd, clip=self.clip,
                            loss_mean=self._loss, workspace=ws, ctx=ctx, d_ctx=d_ctx)
        if update:
            self.steps += 1
            if self.resnet is not None:
                G = self.resnet.backward(d_ctx)
                for name, p, p16 in self.resnet.tensors():
                    mm, vv = self.rmom[name]
                    gwx.adamw(p, G[name].contiguous(), mm, vv, self.steps, self.lr, weight_decay=self.wd,
                              param_bf16=p16)
        return self._loss

    def context(self, y):
        """The ResNet-1D summary of y (bfloat16 [rows][C]), or None for the built-in one."""
        import torch
        return None if self.resnet is None else self.resnet.forward(y, out_dtype=torch.bfloat16)

    def capture_train_step(self, y, theta):
        """Capture one training step on the batch buffers y [B][D][N], theta [11][B] into a
        CUDA graph and return it: each replay runs forward, backward and the AdamW update
        of whatever batch those buffers hold, with the step count kept on the device
        (call note_replay() after each replay to keep the host count in step)."""
        import ctypes
        import torch
        gwx = self.gwx
        if getattr(self, "step_dev", None) is None:
            self.step_dev = torch.tensor([self.steps], dtype=torch.int64, device=self.dev)
        else:
            self.step_dev.fill_(self.steps)
        B = y.shape[0]
        sh = gwx._shape(self.shape)
        nb = _lib.load().gwx_flow_train_workspace(ctypes.byref(sh), B, self.D, self.N)
        ws = self._workspace(("train", B), nb)
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph):
            ctx = d_ctx = None
            if self.resnet is not None:
                # the ResNet-1D summary: forward, the flow's step (which advances the step
                # counter), backward, and AdamW on every summary tensor at that step
                ctx = self.resnet.forward(y, out_dtype=torch.bfloat16)
                d_ctx = torch.empty(ctx.shape, dtype=torch.float32, device=self.dev)
            gwx.flow_train_step(self.shape, self.params, self.params16, self.grads, self.m, self.v, 1, self.lr,
                                self.mean, self.scale, y, theta, self.fs, self.f_lo, weight_decay=self.wd,
                                clip=self.clip, loss_mean=self._loss, workspace=ws, step_counter=self.step_dev,
                                ctx=ctx, d_ctx=d_ctx)
            if self.resnet is not None:
                G = self.resnet.backward(d_ctx)
                for name, p, p16 in self.resnet.tensors():
                    mm, vv = self.rmom[name]
                    gwx.adamw_at(p, G[name].contiguous(), mm, vv, self.step_dev, self.lr, weight_decay=self.wd,
                                 param_bf16=p16)
        return graph

    def note_replay(self):
        self.steps += 1

    def validation_loss(self, y, theta):
        """Mean of -ln q_r over a fixed validation set (y [B][D][N], theta [11][B]), as a
        host float (one synchronisation)."""
        lq = self.log_prob(y, theta)
        return float(-lq.mean().item())

    def fit(self, sim, steps, counter0, val, epoch_sims=160000, patience=10, stop_patience=50, factor=0.1,
            threshold=1e-4, min_lr=None, graph=True, log=None):
        """Train on the simulator's batches (counters counter0, counter0 + 1, ...) for at most
        `steps` steps with the schedule of Sec. 5: an epoch is `epoch_sims` simulations
        (the paper: 200 batches of 800); after every epoch the validation loss of `val`
        (y, theta) is evaluated, the learning rate is divided by 1/factor when it has not
        improved (by more than `threshold`, relative) for `patience` epochs, and training
        stops when it has not improved for `stop_patience` epochs or the learning rate
        falls below `min_lr` (default: initial / 1000).  The parameters of the best epoch
        are restored at the end.  With graph=True each step is one CUDA-graph replay per
        simulator buffer set (recaptured when the learning rate changes).  Returns the
        history: (step, validation loss, learning rate) per epoch and the stop reason."""
        import torch
        B = sim.B
        per_epoch = max(1, round(epoch_sims / B))
        lr0 = self.lr
        min_lr = lr0 * 1e-3 if min_lr is None else min_lr
        best, best_step, bad, bad_stop = float("inf"), 0, 0, 0
        best_params = self.params.clone()
        graphs = {}
        hist, reason = [], "step budget"
        yv, thv = val
        for i in range(steps):
            y, th, _ = sim.step(counter0 + i)
            if graph:
                g = graphs.get(y.data_ptr())
                if g is None:
                    g = graphs[y.data_ptr()] = self.capture_train_step(y, th)
                    # the capture itself runs no step; replay it now
                g.replay()
                self.note_replay()
            else:
                self.train_step(y, th)
            if (i + 1) % per_epoch == 0 or i == steps - 1:
                vl = self.validation_loss(yv, thv)
                hist.append((i + 1, vl, self.lr))
                if log is not None:
                    log(i + 1, vl, self.lr)
                improved = (not math.isfinite(best)) or vl < best - threshold * abs(best)
                if improved:
                    best, best_step, bad, bad_stop = vl, i + 1, 0, 0
                    best_params.copy_(self.params)
                else:
                    bad += 1
                    bad_stop += 1
                    if bad_stop >= stop_patience:
                        reason = "validation loss saturated"
                        break
                    if bad >= patience:
                        bad = 0
                        self.lr *= factor
                        graphs.clear()
                        if self.lr < min_lr:
                            reason = "learning rate below its floor"
                            break
        torch.cuda.synchronize()
        self.params.copy_(best_params)
        self.params16.copy_(self.params.to(torch.bfloat16))
        return {"epochs": hist, "best_step": best_step, "best_val_loss": best, "steps_run": hist[-1][0] if hist else 0,
                "stop": reason, "steps_per_epoch": per_epoch}

    def sample(self, y_events, event_offsets, seed, counter, S=None):
        """Posterior draws for events y_events [E][D][N] (spins and t_c, which the flow does
        not model, from the prior): (theta [11][S], ln q_r [S], ln prior_r - ln q_r [S])."""
        return self.gwx.sample_posterior(self.shape, self.params, self.params16, self.mean, self.scale,
                                         self.wl["prior"], y_events, self.fs, self.f_lo, event_offsets, seed,
                                         counter, ctx=self.context(y_events), S=S)

    def skymap(self, y_event, theta, log_q, nside):
        """The flow's sky density for one event y_event [1][D][N] over the HEALPix pixels
        of nside (nested order, unit sum): RA and sin dec at each pixel centre, the other
        coordinates at the event's draw of largest log_q among theta [11][S]."""
        return self.gwx.flow_skymap(self.shape, self.params, self.params16, self.mean, self.scale, y_event, self.fs,
                                    self.f_lo, theta, log_q, nside, ctx=self.context(y_event))

    def log_prob(self, y, theta):
        return self.gwx.flow_log_prob(self.shape, self.params, self.params16, self.mean, self.scale, y, theta,
                                      self.fs, self.f_lo, ctx=self.context(y))

    # ------------------------------------------------------------ checkpoints
    _MAGIC = b"GWXFLOW1"

    def save(self, path, next_step=None):
        """Flat binary checkpoint (built-in summary only): magic, little-endian int64 header (7 shape fields, steps,
        next_step, n_params), 16 float64 (mean, scale), then params, m and v as float32."""
        import numpy as np
        sh = self.shape
        with open(path, "wb") as fh:
            fh.write(self._MAGIC)
            np.array([sh["features"], sh["group"], sh["embed_hidden"], sh["context"], sh["layers"], sh["hidden"],
                      sh["extra"], self.steps, -1 if next_step is None else next_step, self.n_params],
                     dtype="<i8").tofile(fh)
            np.array(self.mean + self.scale, dtype="<f8").tofile(fh)
            for t in (self.params, self.m, self.v):
                t.detach().cpu().numpy().astype("<f4").tofile(fh)

    def load(self, path):
        """Restore a checkpoint written by save() (same shape); returns the stored next
        data-stream counter (None if none was stored)."""
        import numpy as np
        import torch
        with open(path, "rb") as fh:
            if fh.read(len(self._MAGIC)) != self._MAGIC:
                raise ValueError("not a flow checkpoint: %s" % path)
            hdr = [int(v) for v in np.fromfile(fh, dtype="<i8", count=10)]
            sh = self.shape
            want = [sh["features"], sh["group"], sh["embed_hidden"], sh["context"], sh["layers"], sh["hidden"],
                    sh["extra"]]
            if hdr[:7] != want or hdr[9] != self.n_params:
                raise ValueError("checkpoint shape %s differs from this flow %s" % (hdr[:7], want))
            ms = np.fromfile(fh, dtype="<f8", count=16)
            self.mean, self.scale = [float(v) for v in ms[:8]], [float(v) for v in ms[8:]]
            for t in (self.params, self.m, self.v):
                t.copy_(torch.from_numpy(np.fromfile(fh, dtype="<f4", count=self.n_params)))
            self.params16.copy_(self.params.to(torch.bfloat16))
            self.steps = hdr[7]
        return None if hdr[8] < 0 else hdr[8]


__all__ = ["FlowPosterior"]

"""Self-supervised pre-training of the flow's data summary (Sec. 4.1).

The paper pre-trains its embedding network so that two views of one simulated source,
identical but for the time of arrival, get the same representation: both views are
summarised, expanded by a small network to 24 dimensions, and the VICReg loss of the two
expanded batches (weights 1, 1, 5) is minimised; the expander is then dropped and the
summary keeps training with the flow.  `VICRegPretrainer` does this for a
`flow.FlowPosterior`'s summary: per step it draws B sources from the prior, redraws
their merger times for the second view (`retime`), renders both views into one 2B batch
against the same background crops (`prepare_theta` + `simulate_prepared`), summarises the
2B rows, runs the expander (tcgen05 dense layers), the loss and its gradient (`vicreg`),
the backward pass, and AdamW on the summary's tensors (updated in place in the flow's
parameter arrays) and the expander's.  The summary is the flow's own: the spectral-feature
network, or the ResNet-1D over the raw whitened strain (the paper's case, where nothing but
the pre-training makes the representation insensitive to the arrival time).
"""
import ctypes
import math

from . import _lib


class VICRegPretrainer:
    def __init__(self, flow, batch=1024, expander=(128, 24), lam=(1.0, 1.0, 5.0), lr=1e-3, weight_decay=2e-3,
                 seed=7, background_every=16):
        import torch
        import paper_2407_19048_gb300 as gwx
        self.gwx, self.fp = gwx, flow
        wl = flow.wl
        self.wl, self.B, self.lam = wl, int(batch), tuple(lam)
        self.lr, self.wd, self.seed = float(lr), float(weight_decay), int(seed)
        self.dev = flow.dev
        self.D, self.N = flow.D, flow.N
        self.L = int(wl["L"])
        self.ids = (ctypes.c_int32 * self.D)(*[gwx.DETECTORS[d] if isinstance(d, str) else int(d)
                                                for d in wl["dets"]])
        C = flow.shape["context"]
        g = torch.Generator(device=self.dev)
        g.manual_seed(self.seed)
        dims = [(expander[0], C), (expander[1], expander[0])]
        self.X, self.X16, self.c = [], [], []
        for (o, i) in dims:
            w = torch.randn((o, i), generator=g, device=self.dev) / math.sqrt(i)
            self.X.append(w)
            self.X16.append(w.to(torch.bfloat16))
            self.c.append(torch.zeros(o, device=self.dev))
        # AdamW moments: the summary's tensors (the embedding's six, or the ResNet's) and
        # the expander's four
        self.resnet = flow.resnet
        if self.resnet is None:
            summary = [("e%d" % t, flow.tensor(t)) for t in range(6)]
        else:
            summary = [("r:" + name, p) for name, p, _ in self.resnet.tensors()]
        self.mom = {}
        for key, t in summary + [("X%d" % i, self.X[i]) for i in range(2)] + [("c%d" % i, self.c[i]) for i in range(2)]:
            self.mom[key] = (torch.zeros_like(t), torch.zeros_like(t))
        self.steps = 0
        self.y = torch.empty((2 * self.B, self.D, self.N), dtype=torch.float32, device=self.dev)
        self.ws = gwx._workspace(gwx.workspace_bytes("simulate_batch", self.D, self.B, self.N), self.dev)
        self.bg_every, self.noise, self.psd = int(background_every), None, None

    def _background(self, step):
        gwx, wl = self.gwx, self.wl
        self.noise = gwx.colored_noise(wl["noise_seed"] + 1000, step, self.D, self.L, wl["fs"], wl["f_lo"])
        self.psd = gwx.welch_psd(self.noise, wl["fs"], wl["seg_len"], wl["seg_stride"])

    def _render(self, theta, offsets, y):
        gwx, wl, lib = self.gwx, self.wl, _lib.load()
        ws, nb = self.ws
        s = gwx._stream()
        gwx._check(lib.gwx_prepare_theta(gwx._ptr(theta), self.L, self.N, wl["fs"], wl["f_lo"], self.ids, self.D,
                                         wl.get("gmst", 0.0), self.B, gwx._ptr(ws), nb, s))
        gwx._check(lib.gwx_simulate_prepared(gwx._ptr(self.noise), self.L, gwx._ptr(self.psd), wl["seg_len"],
                                             wl["fs"], wl["f_lo"], self.D, self.B, self.N, gwx._ptr(offsets),
                                             gwx._ptr(y), 0, gwx._ptr(ws), nb, s))

    def views(self, step):
        """Two views [2B][D][N] of B prior draws (rows b and B + b differ only in tc)."""
        gwx, wl = self.gwx, self.wl
        if self.noise is None or step % self.bg_every == 0:
            self._background(step)
        th1, off = gwx.sample_prior(wl["prior"], self.seed, step, self.B, self.L, self.N)
        th2 = gwx.retime(th1, wl["prior"]["tc_lo"], wl["prior"]["tc_hi"], self.seed, step)
        self._render(th1, off, self.y[:self.B])
        self._render(th2, off, self.y[self.B:])
        return self.y

    def features(self, y):
        gwx, fp = self.gwx, self.fp
        sh = fp.shape
        F, G = sh["features"], sh["group"]
        k_lo = math.ceil(fp.f_lo * fp.N / fp.fs - 1e-9)
        ng = (fp.N // 2 - k_lo) // G
        f = gwx.spectral_features(y, fp.fs, fp.f_lo, G, F)
        col = fp.D * ng
        if sh["extra"] & gwx.FLOW_CROSS:
            gwx.cross_features(y, fp.fs, fp.f_lo, G, F, col, f)
            col += fp.D * (fp.D - 1) * ng
        if sh["extra"] & gwx.FLOW_LAG:
            gwx.lag_features(y, fp.fs, fp.f_lo, G, F, col, f)
        return f

    def represent(self, y):
        """(context [rows][C] bfloat16, expanded [rows][24] float32, activations)."""
        import torch
        gwx, fp = self.gwx, self.fp
        R, N = gwx.ACT_RELU, gwx.ACT_NONE
        if self.resnet is not None:
            ctx = self.resnet.forward(y, out_dtype=torch.bfloat16)
            acts = (None, None, None)
        else:
            f = self.features(y)
            h1 = gwx.dense_bf16(f, fp.tensor(0, True), fp.tensor(1), act=R, out_dtype=torch.bfloat16)
            h2 = gwx.dense_bf16(h1, fp.tensor(2, True), fp.tensor(3), act=R, out_dtype=torch.bfloat16)
            ctx = gwx.dense_bf16(h2, fp.tensor(4, True), fp.tensor(5), act=N, out_dtype=torch.bfloat16)
            acts = (f, h1, h2)
        e1 = gwx.dense_bf16(ctx, self.X16[0], self.c[0], act=R, out_dtype=torch.bfloat16)
        x = gwx.dense_bf16(e1, self.X16[1], self.c[1], act=N, out_dtype=torch.float32)
        return ctx, x, acts + (e1,)

    def step(self, step):
        """One pre-training step; returns (loss [1], terms [5]) as device tensors."""
        import torch
        gwx, fp, B = self.gwx, self.fp, self.B
        y = self.views(step)
        ctx, x, (f, h1, h2, e1) = self.represent(y)
        g = torch.empty_like(x)
        loss, terms, _, _ = gwx.vicreg(x[:B], x[B:], self.lam, grad_x=g[:B], grad_xp=g[B:])
        de1, dX1, dc1 = gwx.dense_bf16_backward(e1, self.X16[1], self.c[1], g, act=gwx.ACT_NONE)
        dctx, dX0, dc0 = gwx.dense_bf16_backward(ctx, self.X16[0], self.c[0], de1, act=gwx.ACT_RELU)
        self.steps += 1
        k = self.steps
        if self.resnet is not None:
            G = self.resnet.backward(dctx.float().contiguous())
            upd = [("r:" + name, p, G[name], p16) for name, p, p16 in self.resnet.tensors()]
        else:
            dh2, dW3, db3 = gwx.dense_bf16_backward(h2, fp.tensor(4, True), fp.tensor(5), dctx, act=gwx.ACT_NONE)
            dh1, dW2, db2 = gwx.dense_bf16_backward(h1, fp.tensor(2, True), fp.tensor(3), dh2, act=gwx.ACT_RELU)
            _, dW1, db1 = gwx.dense_bf16_backward(f, fp.tensor(0, True), fp.tensor(1), dh1, act=gwx.ACT_RELU)
            upd = [("e0", fp.tensor(0), dW1, fp.tensor(0, True)), ("e1", fp.tensor(1), db1, None),
                   ("e2", fp.tensor(2), dW2, fp.tensor(2, True)), ("e3", fp.tensor(3), db2, None),
                   ("e4", fp.tensor(4), dW3, fp.tensor(4, True)), ("e5", fp.tensor(5), db3, None)]
        upd += [("X0", self.X[0], dX0, self.X16[0]), ("X1", self.X[1], dX1, self.X16[1]),
                ("c0", self.c[0], dc0, None), ("c1", self.c[1], dc1, None)]
        for key, p, grad, p16 in upd:
            m, v = self.mom[key]
            gwx.adamw(p, grad.contiguous(), m, v, k, self.lr, weight_decay=self.wd, param_bf16=p16)
        return loss, terms


__all__ = ["VICRegPretrainer"]

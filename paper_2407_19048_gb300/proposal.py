"""A learned proposal trained on the on-the-fly simulated batches.

The paper's estimator (Sec. 4 embedding network, Sec. 5 normalizing flow) is trained
with AdamW on batches the simulator produces, and its samples can be corrected by
importance sampling with the standard likelihood (Sec. 6).  This module is the first
step of that learned part, built only from libgwx kernels: a dense network (the
tcgen05 layers `dense_bf16` / `dense_bf16_backward`) maps spectral features of the
whitened strain (`spectral_features`) to the mean and log-scale of a Gaussian over
chirp mass, total mass and distance -- the one-layer case of a conditional affine flow.
`train_step` runs forward, the Gaussian loss (`gauss_nll`), backward and `adamw`;
`proposal_samples` draws importance-sampling samples (`sample_proposal`) whose log
prior-to-proposal ratio feeds `importance_weights`.
"""
import math

from . import ACT_GELU, ACT_NONE

N_OUT = 8   # mu (3), log-scale (3), two unused columns (the layer widths are multiples of 8)


class LearnedProposal:
    def __init__(self, workload, hidden=512, group=4, seed=0, device=None, lr=1e-3, weight_decay=1e-4):
        import torch
        import paper_2407_19048_gb300 as gwx
        self.gwx = gwx
        self.wl = dict(workload)
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        wl = self.wl
        self.D, self.N, self.fs, self.f_lo = len(wl["dets"]), int(wl["N"]), float(wl["fs"]), float(wl["f_lo"])
        k_lo = math.ceil(self.f_lo * self.N / self.fs - 1e-9)   # first band bin
        self.group = int(group)
        ng = (self.N // 2 - k_lo) // self.group
        self.F = ((self.D * ng + 7) // 8) * 8
        self.H = int(hidden)
        self.lr, self.wd = float(lr), float(weight_decay)
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        shapes = [(self.H, self.F), (self.H, self.H), (N_OUT, self.H)]
        self.W, self.b, self.W16, self.mW, self.vW, self.mb, self.vb = [], [], [], [], [], [], []
        for (n_out, n_in) in shapes:
            w = torch.randn((n_out, n_in), generator=g, device=self.dev) * (1.0 / n_in) ** 0.5
            self.W.append(w)
            self.W16.append(w.to(torch.bfloat16))
            self.b.append(torch.zeros(n_out, device=self.dev))
            self.mW.append(torch.zeros_like(w))
            self.vW.append(torch.zeros_like(w))
            self.mb.append(torch.zeros(n_out, device=self.dev))
            self.vb.append(torch.zeros(n_out, device=self.dev))
        # standardisation of (Mc, M, D) from the prior (the scale the network works in)
        import numpy as np
        th, _ = gwx.sample_prior(wl["prior"], 12345, 0, 100000, wl["L"], self.N)
        t = th.cpu().numpy()
        m1, m2, dist = t[0], t[1], t[4]
        raw = np.stack([(m1 * m2) ** 0.6 / (m1 + m2) ** 0.2, m1 + m2, dist])
        self.mean = [float(x) for x in raw.mean(axis=1)]
        self.scale = [float(x) for x in raw.std(axis=1)]
        self.steps = 0

    def features(self, y):
        return self.gwx.spectral_features(y, self.fs, self.f_lo, self.group, self.F)

    def forward(self, feat):
        """Network outputs [B][8] (FP32) and the hidden activations (bfloat16)."""
        import torch
        gwx = self.gwx
        h1 = gwx.dense_bf16(feat, self.W16[0], self.b[0], act=ACT_GELU, out_dtype=torch.bfloat16)
        h2 = gwx.dense_bf16(h1, self.W16[1], self.b[1], act=ACT_GELU, out_dtype=torch.bfloat16)
        out = gwx.dense_bf16(h2, self.W16[2], self.b[2], act=ACT_NONE, out_dtype=torch.float32)
        return out, (feat, h1, h2)

    def train_step(self, y, theta):
        """One AdamW step on a simulated batch (y [B][D][N], theta [11][B]); returns the
        batch-mean loss as a device tensor (no host synchronisation)."""
        gwx = self.gwx
        feat = self.features(y)
        t = gwx.proposal_targets(theta, self.mean, self.scale)
        out, (x0, h1, h2) = self.forward(feat)
        _, loss, g = gwx.gauss_nll(out, t)
        acts = [ACT_GELU, ACT_GELU, ACT_NONE]
        inputs = [x0, h1, h2]
        grads = []
        for i in (2, 1, 0):
            dx, dw, db = gwx.dense_bf16_backward(inputs[i], self.W16[i], self.b[i], g, act=acts[i])
            grads.append((i, dw, db))
            g = dx
        self.steps += 1
        for i, dw, db in grads:
            gwx.adamw(self.W[i], dw, self.mW[i], self.vW[i], self.steps, self.lr, weight_decay=self.wd,
                      param_bf16=self.W16[i])
            gwx.adamw(self.b[i], db, self.mb[i], self.vb[i], self.steps, self.lr)
        return loss

    def net_out(self, y):
        out, _ = self.forward(self.features(y))
        return out

    def proposal_samples(self, y_events, truth, event_offsets, seed, counter, learned=True, fix_angles=False):
        """Importance-sampling draws for events y_events [E][D][N] with known spins and
        merger times (and, with fix_angles, known angles) from truth [11][E]:
        (theta [11][S], log_ratio [S])."""
        net = self.net_out(y_events) if learned else None
        return self.gwx.sample_proposal(self.wl["prior"], truth, event_offsets, seed, counter, net_out=net,
                                        mean=self.mean, scale=self.scale, fix_angles=fix_angles)


    # ---------------------------------------------------------------- checkpoints
    _MAGIC = b"GWXPROP1"

    def save(self, path, next_step=None):
        """Write weights, AdamW moments, step count, standardisation and the caller's
        next data-stream counter to a flat binary file: magic, a little-endian int64
        header (layers, hidden, features, steps, next_step), 6 float64 (mean, scale),
        then per layer the FP32 arrays W, b, m_W, v_W, m_b, v_b in C order."""
        import numpy as np
        with open(path, "wb") as fh:
            fh.write(self._MAGIC)
            np.array([len(self.W), self.H, self.F, self.steps, -1 if next_step is None else next_step],
                     dtype="<i8").tofile(fh)
            np.array(self.mean + self.scale, dtype="<f8").tofile(fh)
            for i in range(len(self.W)):
                for t in (self.W[i], self.b[i], self.mW[i], self.vW[i], self.mb[i], self.vb[i]):
                    t.detach().cpu().numpy().astype("<f4").tofile(fh)

    def load(self, path):
        """Restore a checkpoint written by save() into this object (same shapes); returns
        the stored next data-stream counter (None if none was stored)."""
        import numpy as np
        import torch
        with open(path, "rb") as fh:
            if fh.read(len(self._MAGIC)) != self._MAGIC:
                raise ValueError("not a learned-proposal checkpoint: %s" % path)
            layers, H, F, steps, nxt = (int(v) for v in np.fromfile(fh, dtype="<i8", count=5))
            if (layers, H, F) != (len(self.W), self.H, self.F):
                raise ValueError("checkpoint shapes (%d, %d, %d) differ from this network" % (layers, H, F))
            ms = np.fromfile(fh, dtype="<f8", count=6)
            self.mean, self.scale = [float(v) for v in ms[:3]], [float(v) for v in ms[3:]]
            for i in range(layers):
                for t in (self.W[i], self.b[i], self.mW[i], self.vW[i], self.mb[i], self.vb[i]):
                    a = np.fromfile(fh, dtype="<f4", count=t.numel()).reshape(tuple(t.shape))
                    t.copy_(torch.from_numpy(a))
                self.W16[i].copy_(self.W[i].to(torch.bfloat16))
            self.steps = steps
        return None if nxt < 0 else nxt


__all__ = ["LearnedProposal"]

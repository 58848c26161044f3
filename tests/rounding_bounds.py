"""Element-wise bounds on |GPU - oracle| for the learned part (test infrastructure).

The GPU keeps activations, weights and the products' operands in bfloat16 and
accumulates in FP32; the oracle (oracle.flow) rounds to bfloat16 at the same points but
accumulates in FP64.  The two therefore differ by (i) FP32 accumulation error in every
product and FP32 operation, and (ii) "flips": a value whose FP32 and FP64 versions lie on
either side of a bfloat16 rounding boundary rounds one ulp apart on the two sides, and
that difference propagates through the rest of the chain (as does a ReLU mask of the
backward pass whose pre-activation sits within its accumulation error of zero).

A worst-case propagation of (ii) is useless through a deep chain: it lets every
ambiguous element flip adversarially at once.  Instead the oracle's own chain is
re-evaluated in `TRIALS` perturbed runs (the `Chain` class below mirrors oracle.flow
operation by operation; its unperturbed run reproduces the oracle's values):

* every product sum_k a_k b_k gets an error drawn uniformly within +-4 x 2^-24 sum_k |a_k b_k|
  (recursive FP32 summation of K terms whose partial sums grow like a random walk errs
  by about 2^-24 sum |a b| in r.m.s.; the tensor cores add exact products in wider
  registers within each K-block, so this is several times the expected error; the worst
  case K 2^-24 sum |a b| is not used here, because letting every product err by its worst
  case at once floods the chain with flips no FP32 sum makes);
* every FP32 elementwise result (add, multiply, tanhf, expf) an error within +-4 ulp;
* the features (computed on the GPU from its own FP32 FFT) an error within
  +-FEATURE_ERR before their rounding: 8x the largest deviation of an FP32 FFT's features
  from FP64 on the same kind of input (2.6e-7, measured on the host with a
  single-precision FFT);

and each run then rounds to bfloat16 wherever the GPU does, so the near-boundary
elements flip as they may on the GPU.  The bound of an element is SAFETY x the largest
deviation over the runs plus the deterministic FP32 bound 2 K 2^-24 sum |a b| of the
final contraction that produces it.  It is derived from the oracle alone (no GPU value
enters it) and, because rounding absorbs small differences, it stays a small multiple of
the FP32 error for nearly every element, so each element is checked on its own.
"""
import numpy as np

from oracle import flow as fl

U32 = 2.0 ** -24
FEATURE_ERR = 2e-6
TRIALS = 12
SAFETY = 4.0


class Chain:
    """The flow's training step, density and sampling pass with optional perturbations."""

    def __init__(self, rng=None, scales=None):
        self.rng = rng
        # sum |a b| of every product, recorded by the unperturbed run and reused by the
        # perturbed runs (which make the same products in the same order)
        self.scales = [] if scales is None else scales
        self._i = 0

    # -- primitives
    def _u(self, shape):
        return self.rng.uniform(-1.0, 1.0, shape)

    def prod(self, A, B):
        """A @ B of bfloat16 operands accumulated in FP32; returns (value, sum |a b|)."""
        v = A @ B
        if self.rng is None:
            s = np.abs(A) @ np.abs(B)
            self.scales.append(s)
        else:
            s = self.scales[self._i]
            self._i += 1
            v = v + self._u(v.shape) * 4.0 * U32 * s
        return v, s

    def f32(self, v):
        """One FP32 elementwise result."""
        v = np.asarray(v, dtype=np.float64)
        return v if self.rng is None else v * (1.0 + 4.0 * U32 * self._u(v.shape))

    def rnd(self, v):
        return fl.round_bf16(v)

    # -- layers (the oracle's operations in its order)
    def dense(self, X, W, b, act_relu, out_bf16):
        z, _ = self.prod(X, W.T)
        z = self.f32(z + b[None, :])
        y = np.maximum(z, 0.0) if act_relu else z
        return self.rnd(y) if out_bf16 else y

    def dense_back(self, X, W, b, dy, act_relu):
        if act_relu:
            z, _ = self.prod(X, W.T)                 # recomputed on the tensor cores
            z = self.f32(z + b[None, :])
            dz = dy * (z > 0.0)
        else:
            dz = dy
        dzp = self.rnd(dz)
        dX, _ = self.prod(dzp, W)
        dW, sW = self.prod(dzp.T, X)
        db = np.sum(dz, axis=0)
        sb = np.sum(np.abs(dz), axis=0)
        if self.rng is not None:
            db = db + self._u(db.shape) * 4.0 * U32 * sb
        return dX, dW, db, (dzp.shape[0], sW, sb)

    def embed(self, feat, emb):
        W1, b1, W2, b2, W3, b3 = emb
        h1 = self.dense(feat, W1, b1, True, True)
        h2 = self.dense(h1, W2, b2, True, True)
        c = self.dense(h2, W3, b3, False, True)
        return c, (h1, h2)

    def conditioner_input(self, v, c, l):
        a, _ = fl.SPLITS[l % 4]
        X = np.zeros((len(v), 8 + c.shape[1]))
        X[:, 0:4] = self.rnd(v[:, list(a)])
        X[:, 8:] = c
        return X

    def conditioner(self, X, layer):
        V1, e1, V2, e2, V3, e3 = layer
        g1 = self.dense(X, V1, e1, True, True)
        g2 = self.dense(g1, V2, e2, True, True)
        return self.dense(g2, V3, e3, False, False), (g1, g2)

    def shift_logscale(self, o):
        t = self.f32(np.tanh(self.f32(o[:, 4:8] / fl.S_MAX)))
        return o[:, 0:4], self.f32(fl.S_MAX * t), t

    def coupling(self, v, o, l, direction):
        _, b = fl.SPLITS[l % 4]
        b = list(b)
        mu, s, _ = self.shift_logscale(o)
        w = v.copy()
        if direction > 0:
            w[:, b] = self.f32(v[:, b] * self.f32(np.exp(s)) + mu)
        else:
            w[:, b] = self.f32(self.f32(v[:, b] - mu) * self.f32(np.exp(-s)))
        tot = s[:, 0]
        for j in range(1, 4):
            tot = self.f32(tot + s[:, j])
        return w, tot

    def density(self, x, c, layers):
        v = x
        tot = np.zeros(len(x))
        tape = [None] * len(layers)
        for l in reversed(range(len(layers))):
            X = self.conditioner_input(v, c, l)
            o, (g1, g2) = self.conditioner(X, layers[l])
            v, ss = self.coupling(v, o, l, -1)
            tot = self.f32(tot + ss)
            tape[l] = (X, g1, g2, o, v)
        return v, tot, tape

    def sample(self, z, c, layers):
        v = z
        tot = np.zeros(len(z))
        for l in range(len(layers)):
            o, _ = self.conditioner(self.conditioner_input(v, c, l), layers[l])
            v, ss = self.coupling(v, o, l, +1)
            tot = self.f32(tot + ss)
        return v, tot

    def coupling_backward(self, l, w, o, G, row_weight):
        a, b = (list(t) for t in fl.SPLITS[l % 4])
        _, s, t = self.shift_logscale(o)
        e = self.f32(np.exp(-s))
        Gb = G[:, b]
        dmu = self.f32(-Gb * e)
        ds = self.f32(self.f32(row_weight - self.f32(Gb * w[:, b])) * self.f32(1.0 - self.f32(t * t)))
        Gu = G.copy()
        Gu[:, b] = self.f32(Gb * e)
        return np.concatenate([dmu, ds], axis=1), Gu

    # -- whole passes
    def features(self, feat_pre):
        f = feat_pre if self.rng is None else feat_pre + self._u(feat_pre.shape) * FEATURE_ERR
        return self.rnd(f)

    def loss_and_grads(self, feat_pre, x, params, K):
        emb, layers = fl.split_params(params, K)
        feat = self.features(feat_pre)
        x = self.f32(x)
        c, (h1, h2) = self.embed(feat, emb)
        z, ss, tape = self.density(x, c, layers)
        rows = -fl.log_normal(z) + ss
        B = len(z)
        G = self.f32(z / B)
        dc = np.zeros_like(c)
        layer_grads, sums = [None] * K, [None] * K
        for l in range(K):
            X, g1, g2, o, w = tape[l]
            do, Gu = self.coupling_backward(l, w, o, G, 1.0 / B)
            V1, e1, V2, e2, V3, e3 = layers[l]
            dg2, dV3, de3, s3 = self.dense_back(g2, V3, e3, do, False)
            dg1, dV2, de2, s2 = self.dense_back(g1, V2, e2, dg2, True)
            dX, dV1, de1, s1 = self.dense_back(X, V1, e1, dg1, True)
            a, _ = fl.SPLITS[l % 4]
            G = Gu.copy()
            G[:, list(a)] = self.f32(Gu[:, list(a)] + dX[:, 0:4])
            dc = self.f32(dc + dX[:, 8:])
            layer_grads[l] = [dV1, de1, dV2, de2, dV3, de3]
            sums[l] = [s1, s2, s3]
        W1, b1, W2, b2, W3, b3 = emb
        dh2, dW3, db3, t3 = self.dense_back(h2, W3, b3, dc, False)
        dh1, dW2, db2, t2 = self.dense_back(h1, W2, b2, dh2, True)
        _, dW1, db1, t1 = self.dense_back(feat, W1, b1, dh1, True)
        grads = [dW1, db1, dW2, db2, dW3, db3]
        fsum = [t1, t2, t3]
        for l in range(K):
            grads += layer_grads[l]
            fsum += sums[l]
        return rows.mean(), rows, grads, fsum

    def log_prob(self, feat_pre, x, params, K, log_scale_sum, ctx=None):
        emb, layers = fl.split_params(params, K)
        c = ctx if ctx is not None else self.embed(self.features(feat_pre), emb)[0]
        z, ss, _ = self.density(self.f32(x), c, layers)
        return fl.log_normal(z) - ss - log_scale_sum

    def draws(self, feat_pre, z, ev, params, K):
        emb, layers = fl.split_params(params, K)
        c, _ = self.embed(self.features(feat_pre), emb)
        if self.rng is not None:
            z = z + self._u(z.shape) * 8.0 * U32 * (np.abs(z) + 4.0)   # FP32 Box-Muller of radius <= ~6
        return self.sample(z, c[ev], layers)


def _final_bound(n, s):
    """2 K 2^-24 sum |a b| of an FP32 contraction of K = n terms."""
    return 2.0 * n * U32 * s


def _spread(run, trials=TRIALS, seed=0):
    """(unperturbed result, max |perturbed - unperturbed| over the trials) of run(chain),
    element by element for each array of the (nested) result."""
    ch0 = Chain()
    base = run(ch0)
    flat = [np.asarray(a, dtype=np.float64) for a in (base if isinstance(base, (list, tuple)) else [base])]
    dev = [np.zeros_like(a) for a in flat]
    for t in range(trials):
        out = run(Chain(np.random.default_rng(seed + 1000 * t + 17), ch0.scales))
        out = out if isinstance(out, (list, tuple)) else [out]
        for i, a in enumerate(out):
            dev[i] = np.maximum(dev[i], np.abs(np.asarray(a, dtype=np.float64) - flat[i]))
    return flat, dev


def loss_and_grads(feat_pre, x, params, K):
    """(mean, bound of mean, grads, bounds of grads) of the training step, for the
    unrounded FP64 features feat_pre and FP64 targets x."""
    _, _, _, fsum = Chain().loss_and_grads(feat_pre, x, params, K)

    def run(ch):
        m, _, g, _ = ch.loss_and_grads(feat_pre, x, params, K)
        return [np.array([m])] + list(g)

    vals, dev = _spread(run)
    mean, mean_b = float(vals[0][0]), SAFETY * float(dev[0][0]) + 1e-12 * abs(float(vals[0][0]))
    grads, bounds = vals[1:], []
    # fsum in grads order: per dense layer (n, sum |dZ||X| of dW, sum |dZ| of db)
    for i, g in enumerate(grads):
        n, sW, sb = fsum[i // 2]
        fb = _final_bound(n, sW if i % 2 == 0 else sb)
        bounds.append(SAFETY * dev[1 + i] + fb)
    return mean, mean_b, grads, bounds


def log_prob(feat_pre, x, params, K, log_scale_sum, ctx=None):
    vals, dev = _spread(lambda ch: ch.log_prob(feat_pre, x, params, K, log_scale_sum, ctx))
    return vals[0], SAFETY * dev[0] + 1e-12 * np.abs(vals[0])


def draws(feat_pre, z, ev, params, K):
    """((x, sum_s), (bound x, bound sum_s)) of the sampling pass from base normals z."""
    vals, dev = _spread(lambda ch: list(ch.draws(feat_pre, z, ev, params, K)))
    return vals, [SAFETY * d + 1e-12 * np.abs(v) for v, d in zip(vals, dev)]


# ---------------------------------------------------------------- the ResNet-1D summary

class ResChain(Chain):
    """oracle.resnet's forward and backward pass with the same perturbations as Chain:
    products (convolutions as im2col rows times W^T, their backward products), the
    group-norm arithmetic, the FP32 sums of col2im and pooling; bfloat16 roundings where
    the GPU rounds.  Unperturbed, it reproduces oracle.resnet's values."""

    def __init__(self, rng=None, scales=None):
        super().__init__(rng, scales)
        self.sums = {}

    def conv(self, x, W, k, s, p):
        from oracle import resnet as rn
        cols = rn.im2col(x, k, s, p, W.shape[1])
        B, To, K = cols.shape
        z, _ = self.prod(cols.reshape(B * To, K), W.T)
        return z.reshape(B, To, -1), cols

    def gn(self, z, gamma, beta):
        from oracle import resnet as rn
        y, xh, rstd = rn.gn(z, gamma, beta)
        if self.rng is not None:
            B, T, C = z.shape
            r = np.repeat(rstd, C // rn.GROUPS, axis=1)[:, None, :]
            y = y + self._u(y.shape) * 4.0 * U32 * (np.abs(y) + np.abs(gamma)[None, None, :] * np.abs(z) * r)
        return y, xh, rstd

    def gn_back(self, dy, xh, rstd, gamma):
        from oracle import resnet as rn
        dz, dg, db = rn.gn_back(dy, xh, rstd, gamma)
        if self.rng is not None:
            B, T, C = dy.shape
            r = np.repeat(rstd, C // rn.GROUPS, axis=1)[:, None, :]
            dz = dz + self._u(dz.shape) * 8.0 * U32 * (np.abs(dz) + r * np.abs(dy * gamma[None, None, :]))
            dg = dg + self._u(dg.shape) * 4.0 * U32 * np.sum(np.abs(dy * xh), axis=(0, 1))
            db = db + self._u(db.shape) * 4.0 * U32 * np.sum(np.abs(dy), axis=(0, 1))
        return dz, dg, db

    def col2im(self, dcols, T, C, k, s, p):
        from oracle import resnet as rn
        return self.f32(rn.col2im(dcols, T, C, k, s, p))

    def forward(self, y, P):
        from oracle import resnet as rn
        x = self.rnd(np.transpose(np.asarray(y, dtype=np.float64), (0, 2, 1)))
        tape = {"x": x}
        z0, cols0 = self.conv(x, P["W0"], 7, 2, 3)
        a0p, xh0, r0 = self.gn(z0, P["g0"], P["b0"])
        a0 = self.rnd(np.maximum(a0p, 0.0))
        h, arg = rn.maxpool(a0)
        tape["stem"] = (cols0, xh0, r0, a0, arg)
        tb = []
        for blk in P["blocks"]:
            s = blk["s"]
            z1, c1 = self.conv(h, blk["W1"], 5, s, 2)
            h1p, xh1, r1 = self.gn(z1, blk["g1"], blk["b1"])
            h1 = self.rnd(np.maximum(h1p, 0.0))
            z2, c2 = self.conv(h1, blk["W2"], 5, 1, 2)
            o, xh2, r2 = self.gn(z2, blk["g2"], blk["b2"])
            if "Wd" in blk:
                zd, cd = self.conv(h, blk["Wd"], 1, s, 0)
                sc, xhd, rd = self.gn(zd, blk["gd"], blk["bd"])
            else:
                sc, cd, xhd, rd = h, None, None, None
            out = self.rnd(np.maximum(self.f32(o + sc), 0.0))
            tb.append((h, c1, xh1, r1, h1, c2, xh2, r2, cd, xhd, rd, out))
            h = out
        tape["blocks"] = tb
        m = self.rnd(self.f32(h.mean(axis=1)))
        tape["m"] = m
        c, _ = self.prod(m, P["Wf"].T)
        return self.f32(c + P["bf"][None, :]), tape

    def _wgrad(self, name, dzr, cols):
        g, sW = self.prod(dzr.T, cols.reshape(dzr.shape[0], -1))
        if self.rng is None:
            self.sums[name] = (dzr.shape[0], sW)
        return g

    def backward(self, dc, P, tape):
        from oracle import resnet as rn
        G = {}
        m = tape["m"]
        G["Wf"] = self._wgrad("Wf", self.rnd(dc), m)
        G["bf"] = dc.sum(axis=0)
        self.sums["bf"] = (len(dc), np.abs(dc).sum(axis=0))
        dm, _ = self.prod(self.rnd(dc), P["Wf"])
        hT = tape["blocks"][-1][-1]
        dh = self.f32(np.repeat(dm[:, None, :], hT.shape[1], axis=1) / hT.shape[1])
        gblocks = [None] * len(P["blocks"])
        for i in reversed(range(len(P["blocks"]))):
            blk = P["blocks"][i]
            h, c1, xh1, r1, h1, c2, xh2, r2, cd, xhd, rd, out = tape["blocks"][i]
            s = blk["s"]
            dsum = dh * (out > 0)
            g = {}
            dz2, g["g2"], g["b2"] = self.gn_back(dsum, xh2, r2, blk["g2"])
            B, T2, C2 = dz2.shape
            dzr = self.rnd(dz2).reshape(B * T2, C2)
            g["W2"] = self._wgrad("%d.W2" % i, dzr, c2)
            dcol, _ = self.prod(dzr, blk["W2"])
            dh1 = self.col2im(dcol.reshape(B, T2, -1), h1.shape[1], h1.shape[2], 5, 1, 2)
            dh1 = dh1 * (h1 > 0)
            dz1, g["g1"], g["b1"] = self.gn_back(dh1, xh1, r1, blk["g1"])
            B, T1, C1 = dz1.shape
            dzr = self.rnd(dz1).reshape(B * T1, C1)
            g["W1"] = self._wgrad("%d.W1" % i, dzr, c1)
            dcol, _ = self.prod(dzr, blk["W1"])
            dx = self.col2im(dcol.reshape(B, T1, -1), h.shape[1], h.shape[2], 5, s, 2)
            if "Wd" in blk:
                dzd, g["gd"], g["bd"] = self.gn_back(dsum, xhd, rd, blk["gd"])
                B, Td, Cd = dzd.shape
                dzr = self.rnd(dzd).reshape(B * Td, Cd)
                g["Wd"] = self._wgrad("%d.Wd" % i, dzr, cd)
                dcol, _ = self.prod(dzr, blk["Wd"])
                dx = self.f32(dx + self.col2im(dcol.reshape(B, Td, -1), h.shape[1], h.shape[2], 1, s, 0))
            else:
                dx = self.f32(dx + dsum)
            gblocks[i] = g
            dh = dx
        G["blocks"] = gblocks
        cols0, xh0, r0, a0, arg = tape["stem"]
        da0 = self.f32(rn.maxpool_back(dh, arg, a0.shape[1])) * (a0 > 0)
        dz0, G["g0"], G["b0"] = self.gn_back(da0, xh0, r0, P["g0"])
        B, T0, C0 = dz0.shape
        G["W0"] = self._wgrad("W0", self.rnd(dz0).reshape(B * T0, C0), cols0)
        return G


def _flat_grads(G):
    out = {k: G[k] for k in ("W0", "g0", "b0", "Wf", "bf")}
    for i, g in enumerate(G["blocks"]):
        for k, v in g.items():
            out["%d.%s" % (i, k)] = v
    return out


def resnet(y, P, dc, trials=8):
    """(summary c, its bound, gradients, their bounds) of the ResNet-1D for whitened
    windows y [B][D][N] and dL/dc = dc, gradients keyed like the binding's ("W0", "3.W1",
    ...).  The representation's bound is SAFETY x the spread over the perturbed runs plus
    the FP32 bound of the head's product; each weight gradient's adds the FP32 bound
    2 K 2^-24 sum |dZ| |cols| of its own product over the K = B T rows."""
    base = ResChain()
    c0, tape0 = base.forward(y, P)
    G0 = _flat_grads(base.backward(dc, P, tape0))
    dc_dev = np.zeros_like(c0)
    g_dev = {k: np.zeros_like(v) for k, v in G0.items()}
    for t in range(trials):
        ch = ResChain(np.random.default_rng(7000 + 31 * t), base.scales)
        c, tape = ch.forward(y, P)
        dc_dev = np.maximum(dc_dev, np.abs(c - c0))
        G = _flat_grads(ch.backward(dc, P, tape))
        for k in G0:
            g_dev[k] = np.maximum(g_dev[k], np.abs(G[k] - G0[k]))
    K = P["Wf"].shape[1]
    c_bound = SAFETY * dc_dev + 2.0 * K * U32 * (np.abs(tape0["m"]) @ np.abs(P["Wf"].T)) + 1e-12 * np.abs(c0)
    bounds = {}
    for k, g in G0.items():
        b = SAFETY * g_dev[k] + 1e-12 * np.abs(g)
        if k in base.sums:
            n, s = base.sums[k]
            b = b + _final_bound(n, s)
        bounds[k] = b
    return c0, c_bound, G0, bounds

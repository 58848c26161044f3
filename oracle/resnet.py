"""ResNet-1D data summary (oracle; test infrastructure).

Sec. 4 of the paper summarises the whitened two-detector strain with a ResNet adapted to
time series: 1-D convolutions, group normalisation instead of batch normalisation,
stacks of basic residual blocks with 64, 128 and 256 channels ((5, 3, 3) blocks, kernel
size 5 in the best configuration), and a final fully connected layer to the
representation.  This module states that network in FP64, channels-last:

* conv_direct(x, W, k, s, p): y[b][t][o] = sum_{j, c} W[o][j C + c] x[b][s t + j - p][c]
  (zero outside 0 <= index < T), summed tap by tap as written; T_out = (T + 2 p - k) // s
  + 1; its backward conv_backward_direct is the same sums transposed.  (im2col / col2im,
  the same product as rows of all taps times W^T and its adjoint, are kept as helpers for
  tests and are checked against the direct form);
* gn(z, gamma, beta, G): per sample and group of C / G consecutive channels, over all
  times and those channels: (z - mean) / sqrt(var + 1e-5) (biased variance), then
  gamma_c z + beta_c;
* stem: conv(k 7, s 2, p 3) of the D detector channels (taps padded to a multiple of 8
  columns with zero weights), gn, ReLU, max pool (k 3, s 2, p 1; the first maximum of
  a window on ties);
* block(x; C_out, s): h = relu(gn(conv(x, W1, 5, s, 2))), o = gn(conv(h, W2, 5, 1, 2)),
  shortcut x, or gn(conv(x, Wd, 1, s, 0)) when s > 1 or the width changes;
  out = relu(o + shortcut);
* head: the mean over time of the last stage, then c = Wf m + bf.

Rounding (`rnd`, as in oracle.flow): the GPU holds the input of every convolution, the
block outputs and the pooled mean in bfloat16; convolution and group-norm arithmetic is
FP32 there, FP64 here.  The backward pass is the chain rule of the above, with the
products of the convolutions' backward taking rnd(dZ) as the GPU's do.
"""
import numpy as np

from .flow import exact, round_bf16

EPS = 1e-5
STAGES = ((64, 5, 1), (128, 3, 2), (256, 3, 2))
GROUPS = 8


def stem_k(D):
    """Columns of the stem's im2col rows: 7 D taps rounded up to a multiple of 8."""
    return (7 * D + 7) // 8 * 8


def im2col(x, k, s, p, K=None):
    """x [B][T][C] -> cols [B][T_out][K] (K >= k C, extra columns zero)."""
    x = np.asarray(x, dtype=np.float64)
    B, T, C = x.shape
    To = (T + 2 * p - k) // s + 1
    K = k * C if K is None else K
    cols = np.zeros((B, To, K))
    for j in range(k):
        src = s * np.arange(To) + j - p
        ok = (src >= 0) & (src < T)
        cols[:, ok, j * C:(j + 1) * C] = x[:, src[ok], :]
    return cols


def col2im(dcols, T, C, k, s, p):
    """Adjoint of im2col: dx [B][T][C] from dcols [B][T_out][>= k C]."""
    B, To, _ = dcols.shape
    dx = np.zeros((B, T, C))
    for j in range(k):
        src = s * np.arange(To) + j - p
        ok = (src >= 0) & (src < T)
        np.add.at(dx, (slice(None), src[ok], slice(None)), dcols[:, ok, j * C:(j + 1) * C])
    return dx


def conv(x, W, k, s, p):
    cols = im2col(x, k, s, p, W.shape[1])
    return cols @ W.T, cols


def conv_direct(x, W, k, s, p):
    """The convolution as its definition, tap by tap: y[b][t][o] = sum over j < k and c of
    W[o][j C + c] x[b][s t + j - p][c] (zero outside 0 <= index < T); columns of W past
    k C (the stem's padding) do not enter."""
    x = np.asarray(x, dtype=np.float64)
    B, T, C = x.shape
    To = (T + 2 * p - k) // s + 1
    y = np.zeros((B, To, W.shape[0]))
    for j in range(k):
        src = s * np.arange(To) + j - p
        ok = (src >= 0) & (src < T)
        y[:, ok, :] += np.einsum("btc,oc->bto", x[:, src[ok], :], W[:, j * C:(j + 1) * C])
    return y


def conv_backward_direct(dz, x, W, k, s, p):
    """(dx [B][T][C], dW with the shape of W) of y = conv_direct(x, W, k, s, p) for
    dL/dy = dz, tap by tap: dx[b][s t + j - p][c] += sum_o dz[b][t][o] W[o][j C + c] and
    dW[o][j C + c] = sum_{b, t} dz[b][t][o] x[b][s t + j - p][c]; padded columns of W get
    zero."""
    x = np.asarray(x, dtype=np.float64)
    B, T, C = x.shape
    To = dz.shape[1]
    dx = np.zeros_like(x)
    dW = np.zeros(W.shape)
    for j in range(k):
        src = s * np.arange(To) + j - p
        ok = (src >= 0) & (src < T)
        Wj = W[:, j * C:(j + 1) * C]
        np.add.at(dx, (slice(None), src[ok], slice(None)), np.einsum("bto,oc->btc", dz[:, ok, :], Wj))
        dW[:, j * C:(j + 1) * C] = np.einsum("bto,btc->oc", dz[:, ok, :], x[:, src[ok], :])
    return dx, dW


def gn(z, gamma, beta, G=GROUPS):
    """(y, xhat, rstd [B][G])."""
    B, T, C = z.shape
    zg = z.reshape(B, T, G, C // G)
    mean = zg.mean(axis=(1, 3), keepdims=True)
    var = ((zg - mean) ** 2).mean(axis=(1, 3), keepdims=True)
    rstd = 1.0 / np.sqrt(var + EPS)
    xhat = ((zg - mean) * rstd).reshape(B, T, C)
    return xhat * gamma[None, None, :] + beta[None, None, :], xhat, rstd.reshape(B, G)


def gn_back(dy, xhat, rstd, gamma, G=GROUPS):
    """(dz, dgamma, dbeta) of y = gamma xhat + beta."""
    B, T, C = dy.shape
    dgamma = np.sum(dy * xhat, axis=(0, 1))
    dbeta = np.sum(dy, axis=(0, 1))
    dxh = (dy * gamma[None, None, :]).reshape(B, T, G, C // G)
    xh = xhat.reshape(B, T, G, C // G)
    m1 = dxh.mean(axis=(1, 3), keepdims=True)
    m2 = (dxh * xh).mean(axis=(1, 3), keepdims=True)
    dz = rstd.reshape(B, 1, G, 1) * (dxh - m1 - xh * m2)
    return dz.reshape(B, T, C), dgamma, dbeta


def maxpool(x):
    """k 3, s 2, p 1 over time: (y [B][T_out][C], argmax offsets in {0, 1, 2})."""
    B, T, C = x.shape
    To = (T + 2 - 3) // 2 + 1
    xp = np.full((B, T + 2, C), -np.inf)
    xp[:, 1:T + 1] = x
    win = np.stack([xp[:, 2 * np.arange(To) + j] for j in range(3)], axis=0)
    arg = np.argmax(win, axis=0)
    return np.max(win, axis=0), arg


def maxpool_back(dy, arg, T):
    B, To, C = dy.shape
    dx = np.zeros((B, T + 2, C))
    b, t, c = np.meshgrid(np.arange(B), np.arange(To), np.arange(C), indexing="ij")
    np.add.at(dx, (b, 2 * t + arg, c), dy)
    return dx[:, 1:T + 1]


def init_params(rng, D, C_out, stages=STAGES):
    """Random parameters (weights N(0, 2 / fan_in), gamma 1 + N(0, 0.1^2), beta
    N(0, 0.1^2), FC N(0, 1 / 256)) as a dict of float64 arrays (test inputs)."""
    def w(o, i):
        return rng.normal(0, np.sqrt(2.0 / i), (o, i))

    def g(c):
        return 1.0 + rng.normal(0, 0.1, c), rng.normal(0, 0.1, c)

    P = {"W0": np.zeros((stages[0][0], stem_k(D)))}
    P["W0"][:, :7 * D] = w(stages[0][0], 7 * D)
    P["g0"], P["b0"] = g(stages[0][0])
    cin = stages[0][0]
    blocks = []
    for (c, n, s) in stages:
        for i in range(n):
            stride = s if i == 0 else 1
            blk = {"s": stride, "W1": w(c, 5 * cin), "W2": w(c, 5 * c)}
            blk["g1"], blk["b1"] = g(c)
            blk["g2"], blk["b2"] = g(c)
            if stride != 1 or cin != c:
                blk["Wd"] = w(c, cin)
                blk["gd"], blk["bd"] = g(c)
            blocks.append(blk)
            cin = c
    P["blocks"] = blocks
    P["Wf"] = rng.normal(0, np.sqrt(1.0 / cin), (C_out, cin))
    P["bf"] = rng.normal(0, 0.1, C_out)
    return P


def forward(y, P, rnd=round_bf16):
    """Summary c [B][C_out] of whitened windows y [B][D][N]; returns (c, tape)."""
    x = rnd(np.transpose(np.asarray(y, dtype=np.float64), (0, 2, 1)))      # [B][N][D]
    tape = {"x": x}
    z0 = conv_direct(x, P["W0"], 7, 2, 3)
    a0p, xh0, r0 = gn(z0, P["g0"], P["b0"])
    a0 = rnd(np.maximum(a0p, 0.0))
    h, arg = maxpool(a0)
    tape["stem"] = (x, xh0, r0, a0, arg)
    tb = []
    for blk in P["blocks"]:
        s = blk["s"]
        z1 = conv_direct(h, blk["W1"], 5, s, 2)
        h1p, xh1, r1 = gn(z1, blk["g1"], blk["b1"])
        h1 = rnd(np.maximum(h1p, 0.0))
        z2 = conv_direct(h1, blk["W2"], 5, 1, 2)
        o, xh2, r2 = gn(z2, blk["g2"], blk["b2"])
        if "Wd" in blk:
            zd = conv_direct(h, blk["Wd"], 1, s, 0)
            sc, xhd, rd = gn(zd, blk["gd"], blk["bd"])
        else:
            sc, xhd, rd = h, None, None
        out = rnd(np.maximum(o + sc, 0.0))
        tb.append((h, xh1, r1, h1, xh2, r2, xhd, rd, out))
        h = out
    tape["blocks"] = tb
    m = rnd(h.mean(axis=1))
    tape["m"] = m
    return m @ P["Wf"].T + P["bf"][None, :], tape


def backward(dc, P, tape, rnd=round_bf16):
    """Gradients of a loss with dL/dc = dc: dict with the keys of P (blocks: list)."""
    G = {}
    m = tape["m"]
    G["Wf"] = rnd(dc).T @ m
    G["bf"] = dc.sum(axis=0)
    dm = rnd(dc) @ P["Wf"]
    hT = tape["blocks"][-1][-1]
    dh = np.repeat(dm[:, None, :], hT.shape[1], axis=1) / hT.shape[1]
    gblocks = [None] * len(P["blocks"])
    for i in reversed(range(len(P["blocks"]))):
        blk = P["blocks"][i]
        h, xh1, r1, h1, xh2, r2, xhd, rd, out = tape["blocks"][i]
        s = blk["s"]
        dsum = dh * (out > 0)
        g = {}
        dz2, g["g2"], g["b2"] = gn_back(dsum, xh2, r2, blk["g2"])
        dh1, g["W2"] = conv_backward_direct(rnd(dz2), h1, blk["W2"], 5, 1, 2)
        dh1 = dh1 * (h1 > 0)
        dz1, g["g1"], g["b1"] = gn_back(dh1, xh1, r1, blk["g1"])
        dx, g["W1"] = conv_backward_direct(rnd(dz1), h, blk["W1"], 5, s, 2)
        if "Wd" in blk:
            dzd, g["gd"], g["bd"] = gn_back(dsum, xhd, rd, blk["gd"])
            dxd, g["Wd"] = conv_backward_direct(rnd(dzd), h, blk["Wd"], 1, s, 0)
            dx = dx + dxd
        else:
            dx = dx + dsum
        gblocks[i] = g
        dh = dx
    G["blocks"] = gblocks
    x0, xh0, r0, a0, arg = tape["stem"]
    da0 = maxpool_back(dh, arg, a0.shape[1]) * (a0 > 0)
    dz0, G["g0"], G["b0"] = gn_back(da0, xh0, r0, P["g0"])
    _, G["W0"] = conv_backward_direct(rnd(dz0), x0, P["W0"], 7, 2, 3)
    return G

"""Inverse-autoregressive flow, the paper's flow family (oracle; test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline and
reference legs use the oracle; the library never imports it.

Sec. 5.1 builds its estimator from inverse-autoregressive affine transforms (Kingma et al.
2016, "Improved variational inference with inverse autoregressive flow"): 60 of them, each
with a masked autoencoder (Germain et al. 2015, "MADE") of 6 masked linear layers of 100
hidden units, over the D = 8 source parameters; the whole stack holds ~3.2 M trainable
parameters.  A draw takes one pass of each transform; the density of a given theta takes
D sequential passes of each, one per coordinate.  The library's flow is the coupling
flow of ``oracle.flow`` (one pass each way); this module states the paper's variant, in
the same coordinates x (``oracle.flow.standardise``) and with the same context c, the
data summary.

MADE of one transform (readings where the paper is silent):
  input      u = [v (D values), c (C values)]
  hidden     g_1 = relu(W_1 u + b_1), g_l = relu(W_l g_{l-1} + b_l), l = 2 .. 6 (H each)
  output     o = W_7 g_6 + b_7 (2 D values): shift mu_i = o_i, log-scale
             s_i = S_MAX tanh(o_{D+i} / S_MAX) (the coupling flow's soft clamp)
  with every W_l multiplied element-wise by a fixed 0/1 mask.  Degrees: input coordinate i
  (0-based) has degree i + 1; hidden unit h of every layer has degree (h mod (D - 1)) + 1;
  shift and log-scale of coordinate i have degree i + 1.  A weight from degree a to a
  hidden unit of degree b is kept when b >= a, to an output of degree b when b > a; the
  context reaches every unit of the first layer.  So mu_i and s_i depend on v_0 .. v_{i-1}
  and c only.  With C = 8 (the representation dimension gamma of Sec. 4) the stack has
  60 x (16 x 100 + 5 x 100^2 + 100 x 16 + 6 x 100 + 16) = 3,228,960 parameters, the
  paper's ~3.2 M.
Transform (sampling direction, one pass):  y_i = v_i e^{s_i(v)} + mu_i(v),  ln|det| = sum_i s_i.
Inverse (density direction, D passes):  v_i = (y_i - mu_i) e^{-s_i}, i = 0 .. D-1 in turn,
  mu_i and s_i from the v_0 .. v_{i-1} found so far.
Stack: z ~ N(0, I_D) goes through transforms 0 .. K-1, the coordinate order reversed
between consecutive transforms (a reading: the paper does not state its permutations);
ln q(x) = ln N(z; 0, I_D) - sum over transforms of sum_i s_i.
"""
import math

import numpy as np

from . import flow
from .flow import S_MAX, exact, relu

N_HIDDEN = 6      # masked hidden layers per transform (Sec. 5.1)
HIDDEN = 100      # units per hidden layer (Sec. 5.1)
N_TRANSFORMS = 60  # transforms in the stack (Sec. 5.1)
LN_2PI = math.log(2.0 * math.pi)


def degrees(D, H=HIDDEN, n_hidden=N_HIDDEN):
    """(input degrees [D], hidden degrees [n_hidden][H], output degrees [2 D])."""
    d_in = np.arange(1, D + 1)
    d_h = [(np.arange(H) % max(D - 1, 1)) + 1 for _ in range(n_hidden)]
    return d_in, d_h, np.concatenate([d_in, d_in])


def masks(D, C, H=HIDDEN, n_hidden=N_HIDDEN):
    """0/1 masks of W_1 .. W_{n_hidden + 1}: [H][D + C], [H][H] ..., [2 D][H]."""
    d_in, d_h, d_out = degrees(D, H, n_hidden)
    m = [np.concatenate([(d_h[0][:, None] >= d_in[None, :]).astype(np.float64), np.ones((H, C))], axis=1)]
    for l in range(1, n_hidden):
        m.append((d_h[l][:, None] >= d_h[l - 1][None, :]).astype(np.float64))
    m.append((d_out[:, None] > d_h[-1][None, :]).astype(np.float64))
    return m


def n_params(D, C, H=HIDDEN, n_hidden=N_HIDDEN, K=N_TRANSFORMS):
    """Trainable weights and biases of the stack (masked entries included, as stored)."""
    per = (D + C) * H + (n_hidden - 1) * H * H + H * 2 * D + n_hidden * H + 2 * D
    return K * per


def init(D, C, H=HIDDEN, n_hidden=N_HIDDEN, K=N_TRANSFORMS, seed=0, out_scale=0.1):
    """Random stack: per transform [W_1, b_1, ..., W_{n_hidden + 1}, b_{n_hidden + 1}], the
    masks applied; weights ~ N(0, 1 / fan_in), the output layer's scaled by out_scale so
    the untrained stack is near the identity."""
    rng = np.random.default_rng(seed)
    ms = masks(D, C, H, n_hidden)
    stack = []
    for _ in range(K):
        layer = []
        for l, m in enumerate(ms):
            fan_in = m.shape[1]
            w = rng.standard_normal(m.shape) / math.sqrt(fan_in)
            if l == len(ms) - 1:
                w *= out_scale
            layer += [w * m, 0.01 * rng.standard_normal(m.shape[0])]
        stack.append(layer)
    return stack


def made(layer, v, c, rnd=exact, stats=None):
    """(mu [B][D], s [B][D]) of one transform's autoencoder at rows v [B][D], context c [B][C]."""
    if stats is not None:
        stats["made"] = stats.get("made", 0) + 1
    v = np.asarray(v, dtype=np.float64)
    D = v.shape[1]
    g = rnd(np.concatenate([v, np.asarray(c, dtype=np.float64)], axis=1))
    n = len(layer) // 2
    for l in range(n - 1):
        g = rnd(relu(g @ layer[2 * l].T + layer[2 * l + 1][None, :]))
    o = g @ layer[2 * n - 2].T + layer[2 * n - 1][None, :]
    return o[:, :D], S_MAX * np.tanh(o[:, D:] / S_MAX)


def forward(layer, v, c, rnd=exact, stats=None):
    """One transform, sampling direction: (y, sum_i s_i per row)."""
    mu, s = made(layer, v, c, rnd, stats)
    return np.asarray(v, dtype=np.float64) * np.exp(s) + mu, s.sum(axis=1)


def inverse(layer, y, c, rnd=exact, stats=None):
    """One transform, density direction (D autoencoder passes): (v, sum_i s_i per row)."""
    y = np.asarray(y, dtype=np.float64)
    D = y.shape[1]
    v = np.zeros_like(y)
    for i in range(D):
        mu, s = made(layer, v, c, rnd, stats)
        v[:, i] = (y[:, i] - mu[:, i]) * np.exp(-s[:, i])
    return v, s.sum(axis=1)


def log_normal(z):
    z = np.asarray(z, dtype=np.float64)
    return -0.5 * np.sum(z * z, axis=1) - 0.5 * z.shape[1] * LN_2PI


def sample(stack, z, c, rnd=exact, stats=None):
    """Draws x [B][D] from base normals z [B][D] and ln q(x) [B]: one pass per transform."""
    v = np.asarray(z, dtype=np.float64)
    tot = np.zeros(len(v))
    for k, layer in enumerate(stack):
        if k:
            v = v[:, ::-1]
        v, ss = forward(layer, v, c, rnd, stats)
        tot += ss
    return v, log_normal(z) - tot


def log_prob(stack, x, c, rnd=exact, stats=None):
    """(ln q(x) [B], z [B][D]) for x [B][D]: D passes per transform."""
    v = np.asarray(x, dtype=np.float64)
    tot = np.zeros(len(v))
    for k in reversed(range(len(stack))):
        v, ss = inverse(stack[k], v, c, rnd, stats)
        tot += ss
        if k:
            v = v[:, ::-1]
    return log_normal(v) - tot, v


# ---------------------------------------------------------------- training gradient
# The loss of a row is -ln q(x) = |z|^2 / 2 + (D / 2) ln 2 pi + sum over transforms of
# sum_i s_i, evaluated in the density direction.  Its gradient follows that direction's
# passes backwards: pass i of a transform read the partial v (entries i .. D-1 still zero),
# set v_i = (y_i - mu_i) e^{-s_i} and contributed s_i to the log-determinant, so it sends
#   dy_i = g_i e^{-s_i},  dmu_i = -g_i e^{-s_i},  ds_i = -g_i v_i + (the loss's weight on s)
# back, its autoencoder turns (dmu_i, ds_i) into gradients of the weights, the context and
# the partial v, and entry i of g is consumed.  The weights' gradients are masked (a masked
# weight stays zero under any update); a rounding hook, where given, counts as the identity.


def made_tape(layer, v, c, rnd=exact):
    """(mu, s, tape) with tape = (layer inputs [n], pre-activations [n - 1], s)."""
    v = np.asarray(v, dtype=np.float64)
    D = v.shape[1]
    g = rnd(np.concatenate([v, np.asarray(c, dtype=np.float64)], axis=1))
    n = len(layer) // 2
    ins, pre = [g], []
    for l in range(n - 1):
        a = g @ layer[2 * l].T + layer[2 * l + 1][None, :]
        pre.append(a)
        g = rnd(relu(a))
        ins.append(g)
    o = g @ layer[2 * n - 2].T + layer[2 * n - 1][None, :]
    s = S_MAX * np.tanh(o[:, D:] / S_MAX)
    return o[:, :D], s, (ins, pre, s)


def made_backward(layer, ms, tape, dmu, ds):
    """Gradients (dW [n], db [n], du) of one autoencoder pass from those of mu and s; du is
    the gradient of its input row [v, c]."""
    ins, pre, s = tape
    n = len(layer) // 2
    do = np.concatenate([dmu, ds * (1.0 - (s / S_MAX) ** 2)], axis=1)
    dW, db = [None] * n, [None] * n
    for l in reversed(range(n)):
        dW[l] = (do.T @ ins[l]) * ms[l]
        db[l] = do.sum(axis=0)
        d_in = do @ layer[2 * l]
        if l:
            do = d_in * (pre[l - 1] > 0.0)
    return dW, db, d_in


def inverse_tape(layer, y, c, rnd=exact):
    """The density direction of one transform with the passes' tapes: (v, sum_s, tape)."""
    y = np.asarray(y, dtype=np.float64)
    D = y.shape[1]
    v = np.zeros_like(y)
    tot = np.zeros(len(y))
    passes = []
    for i in range(D):
        mu, s, t = made_tape(layer, v, c, rnd)
        v = v.copy()
        v[:, i] = (y[:, i] - mu[:, i]) * np.exp(-s[:, i])
        tot += s[:, i]
        passes.append((t, s[:, i].copy()))
    return v, tot, passes


def inverse_backward(layer, ms, passes, v, g, ws):
    """Back through one transform's density direction: g = d loss / d v (its output), ws =
    the loss's weight on its sum_s per row.  Returns (d loss / d y, dW, db, dc)."""
    D = v.shape[1]
    g = np.array(g, dtype=np.float64)
    dy = np.zeros_like(g)
    n = len(layer) // 2
    dW = [np.zeros_like(layer[2 * l]) for l in range(n)]
    db = [np.zeros_like(layer[2 * l + 1]) for l in range(n)]
    dc = 0.0
    for i in reversed(range(D)):
        t, s_i = passes[i]
        e = np.exp(-s_i)
        dy[:, i] = g[:, i] * e
        dmu = np.zeros_like(g)
        ds = np.zeros_like(g)
        dmu[:, i] = -g[:, i] * e
        ds[:, i] = -g[:, i] * v[:, i] + ws
        g[:, i] = 0.0                       # entry i was an input zero, overwritten
        w_l, b_l, du = made_backward(layer, ms, t, dmu, ds)
        for l in range(n):
            dW[l] += w_l[l]
            db[l] += b_l[l]
        g += du[:, :D]
        dc = dc + du[:, D:]
    return dy, dW, db, dc


def loss_and_grads(stack, x, c, rnd=exact):
    """Mean over rows of -ln q(x) and its gradients: (loss, grads per transform as
    [dW_1, db_1, ...] (masked), dc [B][C], dx [B][D])."""
    x = np.asarray(x, dtype=np.float64)
    B, D = x.shape
    C = np.asarray(c).shape[1]
    H = stack[0][0].shape[0]
    ms = masks(D, C, H, len(stack[0]) // 2 - 1)
    v = x
    tot = np.zeros(B)
    tapes = [None] * len(stack)
    for k in reversed(range(len(stack))):
        v_out, ss, passes = inverse_tape(stack[k], v, c, rnd)
        tapes[k] = (passes, v_out)
        tot += ss
        v = v_out[:, ::-1] if k else v_out
    z = v
    loss = np.mean(0.5 * np.sum(z * z, axis=1) + 0.5 * D * LN_2PI + tot)
    g = z / B
    ws = np.full(B, 1.0 / B)
    grads = [None] * len(stack)
    dc = np.zeros((B, C))
    for k in range(len(stack)):
        if k:
            g = g[:, ::-1]
        passes, v_out = tapes[k]
        g, dW, db, dck = inverse_backward(stack[k], ms, passes, v_out, g, ws)
        grads[k] = [t for pair in zip(dW, db) for t in pair]
        dc += dck
    return loss, grads, dc, g


# ---------------------------------------------------------------- posterior draws
# The same proposal as the coupling flow's (oracle.flow): base normals z and the ordering
# coin from Philox (flow.base_normals), x from the stack, r = mean + scale x mapped to
# theta with the prior-to-proposal log ratio (flow.proposal_params); only the map z -> x
# and its log-determinant differ.


def sample_posterior(stack, c_events, mean, scale, prior, offsets, seed, counter, rnd=exact):
    """Draws of event e in rows offsets[e] .. offsets[e+1]-1 with context c_events[e]:
    (theta [11][S], ln q_r [S], ln pi_r - ln q_r [S])."""
    S = int(np.asarray(offsets)[-1])
    ev = flow.event_of(offsets, S)
    z, coin = flow.base_normals(seed, counter, np.arange(S))
    x, lq = sample(stack, z, np.asarray(c_events, dtype=np.float64)[ev], rnd)
    return flow.proposal_params(x, z, log_normal(z) - lq, mean, scale, prior, coin,
                                flow.nuisance_uniforms(seed, counter, np.arange(S)))


def log_prob_theta(stack, c, theta, mean, scale, rnd=exact):
    """ln q_r(r(theta) | c) for each column of theta [11][B] with its context row (the
    density over the eight modelled coordinates; D passes per transform)."""
    x = flow.standardise(flow.coords(theta), mean, scale)
    lq, _ = log_prob(stack, x, c, rnd)
    return lq - np.sum(np.log(np.asarray(scale)))

"""Conditional coupling flow over the eight source parameters (oracle; test infrastructure).

The paper's estimator (Sec. 5) is a normalizing flow: a standard normal over an
eight-dimensional parameter vector theta = (Mc, q, D_L, theta_JN, alpha, delta, psi,
phi_c) pushed through a stack of invertible affine transforms whose shifts and
log-scales are functions of the data summary of Sec. 4; training maximises the mean
ln q(theta_i | d_i) over simulations (the loss of Sec. 5), with AdamW.  The paper's
transforms are inverse-autoregressive (one pass to sample, eight sequential passes
for a density).  This oracle states the flow the library builds instead: affine
coupling transforms (Dinh, Sohl-Dickstein and Bengio 2017, "Density estimation using
Real NVP"), for which sampling and density each take one pass.

Coordinates.  r = (Mc, q, D_L, cos theta_JN, alpha, sin delta, psi, phi_c) with chirp
mass Mc = (m1 m2)^{3/5} / (m1 + m2)^{1/5} and q = min(m1, m2) / max(m1, m2) in (0, 1];
the flow works in x = (r - mean) / scale (given per coordinate).

Embedding (the data summary).  From the spectral features f of the whitened strain
(oracle.learn.features and cross_features):  c = W3 h2 + b3,  h2 = relu(W2 h1 + b2),
h1 = relu(W1 f + b1), relu(z) = max(z, 0) (the activation of the autoregressive
networks in the library the paper builds its flow with, and of the ResNet it adapts).

Coupling layer l (l = 0 .. K-1) uses the split SPLITS[l % 4] = (a, b) of the eight
coordinates into four conditioning coordinates a and four transformed coordinates b.
Its conditioner reads the row X = [v_a (4 values), 0, 0, 0, 0, c (C values)] and gives
o = V3 g2 + e3 (8 values), g2 = relu(V2 g1 + e2), g1 = relu(V1 X + e1); the shift is
mu_j = o_j and the log-scale s_j = S_MAX tanh(o_{4+j} / S_MAX), j = 0..3, acting on
coordinate b[j]:
  sampling direction  v_b <- v_b e^{s} + mu,
  density direction   v_b <- (v_b - mu) e^{-s}   (v_a unchanged in both).
Sampling applies layers 0 .. K-1 to z ~ N(0, I_8); the density applies K-1 .. 0 to x.
With sum_s = sum over layers of sum_j s_j:  ln q_x(x) = ln N(z; 0, I_8) - sum_s, and in
r-coordinates ln q_r(r) = ln q_x(x) - sum_p ln scale_p.

Training loss of one row: -ln q_x(x) = |z|^2 / 2 + 4 ln(2 pi) + sum_s; the batch mean is
minimised.  Its gradient with respect to every weight is stated below by the chain rule.

Rounding.  The GPU holds the conditioner and embedding activations, the features, the
context and the conditioner inputs in bfloat16 and the weights as bfloat16 copies; each
function takes `rnd`, applied where the GPU rounds (round_bf16 for parity, `exact` for
the pins that need a smooth function).

Importance-sampling proposal.  A draw x gives r = mean + scale x; inside the prior's
support m_big = Mc (1 + q)^{1/5} q^{-3/5} and m_small = q m_big, ordered by a fair coin,
theta_JN = acos(r_3), delta = asin(r_5).  The flow does not model the spins or t_c (the
paper ignores spins and marginalises t_c, Sec. 5): they are drawn from their own prior,
chi_i = chi_lo + (chi_hi - chi_lo) u, t_c = tc_lo + (tc_hi - tc_lo) u, so their prior
and proposal densities are equal and cancel in the log ratio below.  The prior of the
workloads is uniform in (m1, m2) on [m_lo, m_hi]^2 and in D, cos theta_JN, alpha,
sin delta, psi, phi_c; in r-coordinates its density is
  pi_r = 2 m_big^2 / (Mc (m_hi - m_lo)^2) / ((d_hi - d_lo) 2 (2 pi) 2 (psi_hi - psi_lo)
         (phi_hi - phi_lo)),
the factor 2 for the two mass orderings and m_big^2 / Mc = |d(m1, m2) / d(Mc, q)|.
The log ratio of a draw is ln pi_r - ln q_r (-inf outside the support).

Base normals.  Draw s uses Philox4x32-10 counters (s, j, TAG_FLOW, counter), j = 0..4,
block j giving u_{2j} = uniform52(w0, w1) and u_{2j+1} = uniform52(w2, w3); the normals
are Box-Muller pairs z_{2i}, z_{2i+1} = sqrt(-2 ln u_{2i}) (cos, sin)(2 pi u_{2i+1}),
i = 0..3, and u_8 is the ordering coin (masses swapped when u_8 < 1/2).  The parameters
the flow does not model take u_9 (t_c) and block 5's u_10, u_11 (chi_1, chi_2).
"""
import math

import numpy as np

from .gemm import bf16_to_f64, f64_to_bf16
from .philox import key_of, philox4x32_10, uniform52

TAG_FLOW = 4
S_MAX = 3.0
NDIM = 8
LN_2PI = math.log(2.0 * math.pi)

SPLITS = (((0, 1, 2, 3), (4, 5, 6, 7)),
          ((4, 5, 6, 7), (0, 1, 2, 3)),
          ((0, 2, 4, 6), (1, 3, 5, 7)),
          ((1, 3, 5, 7), (0, 2, 4, 6)))


def round_bf16(x):
    return bf16_to_f64(f64_to_bf16(x))


def exact(x):
    return np.asarray(x, dtype=np.float64)


def relu(z):
    return np.maximum(z, 0.0)


def relu_grad(z):
    return (np.asarray(z) > 0.0).astype(np.float64)


def split_params(params, K):
    """(embedding [W1, b1, W2, b2, W3, b3], [per layer [V1, e1, V2, e2, V3, e3]]) as FP64."""
    p = [np.asarray(t, dtype=np.float64) for t in params]
    if len(p) != 6 + 6 * K:
        raise ValueError("expected %d tensors" % (6 + 6 * K))
    return p[:6], [p[6 + 6 * l:12 + 6 * l] for l in range(K)]


# ---------------------------------------------------------------- coordinates

def coords(theta):
    """r [B][8] from theta [11][B] (rows m1, m2, chi1, chi2, D, tc, phic, theta_JN, psi, RA, dec)."""
    th = np.asarray(theta, dtype=np.float64)
    m1, m2 = th[0], th[1]
    big, small = np.maximum(m1, m2), np.minimum(m1, m2)
    Mc = (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2
    return np.stack([Mc, small / big, th[4], np.cos(th[7]), th[9], np.sin(th[10]), th[8], th[6]], axis=1)


def standardise(r, mean, scale):
    return (np.asarray(r, dtype=np.float64) - np.asarray(mean)[None, :]) / np.asarray(scale)[None, :]


def masses(Mc, q):
    """(m_big, m_small) with chirp mass Mc and ratio q = m_small / m_big."""
    big = Mc * (1.0 + q) ** 0.2 * q ** -0.6
    return big, q * big


def log_prior_r(r, prior):
    """ln pi_r(r) of the workloads' prior in r-coordinates (-inf outside its support)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.full(len(r), -np.inf)
    for i in range(len(r)):
        Mc, q, D, ct, al, sd, psi, phi = r[i]
        if not (Mc > 0.0 and 0.0 < q <= 1.0):
            continue
        big, small = masses(Mc, q)
        inside = (prior["m_lo"] <= small and big <= prior["m_hi"] and prior["d_lo"] <= D <= prior["d_hi"]
                  and -1.0 <= ct <= 1.0 and 0.0 <= al < 2.0 * math.pi and -1.0 <= sd <= 1.0
                  and prior["psi_lo"] <= psi <= prior["psi_hi"] and prior["phi_lo"] <= phi <= prior["phi_hi"])
        if not inside:
            continue
        out[i] = (math.log(2.0) + 2.0 * math.log(big) - math.log(Mc) - 2.0 * math.log(prior["m_hi"] - prior["m_lo"])
                  - math.log(prior["d_hi"] - prior["d_lo"]) - math.log(2.0) - math.log(2.0 * math.pi)
                  - math.log(2.0) - math.log(prior["psi_hi"] - prior["psi_lo"])
                  - math.log(prior["phi_hi"] - prior["phi_lo"]))
    return out


# ---------------------------------------------------------------- network pieces

def embed(feat, emb, rnd=round_bf16):
    """Context c [B][C] from features feat [B][F]; returns (c, (h1, h2))."""
    W1, b1, W2, b2, W3, b3 = emb
    f = np.asarray(feat, dtype=np.float64)
    h1 = rnd(relu(f @ W1.T + b1[None, :]))
    h2 = rnd(relu(h1 @ W2.T + b2[None, :]))
    c = rnd(h2 @ W3.T + b3[None, :])
    return c, (h1, h2)


def conditioner_input(v, c, l, rnd=round_bf16):
    """X [B][8 + C] = [v_a, 0, 0, 0, 0, c] for layer l."""
    a, _ = SPLITS[l % 4]
    v = np.asarray(v, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    X = np.zeros((len(v), 8 + c.shape[1]))
    X[:, 0:4] = rnd(v[:, list(a)])
    X[:, 8:] = c
    return X


def conditioner(X, layer, rnd=round_bf16):
    """o [B][8] of one conditioner; returns (o, (g1, g2))."""
    V1, e1, V2, e2, V3, e3 = layer
    g1 = rnd(relu(X @ V1.T + e1[None, :]))
    g2 = rnd(relu(g1 @ V2.T + e2[None, :]))
    return g2 @ V3.T + e3[None, :], (g1, g2)


def shift_logscale(o):
    o = np.asarray(o, dtype=np.float64)
    return o[:, 0:4], S_MAX * np.tanh(o[:, 4:8] / S_MAX)


def coupling(v, o, l, direction):
    """One coupling step of layer l: direction +1 samples, -1 evaluates the density.
    Returns (v', sum_j s_j per row)."""
    _, b = SPLITS[l % 4]
    b = list(b)
    mu, s = shift_logscale(o)
    v = np.asarray(v, dtype=np.float64)
    w = v.copy()
    if direction > 0:
        w[:, b] = v[:, b] * np.exp(s) + mu
    else:
        w[:, b] = (v[:, b] - mu) * np.exp(-s)
    return w, s.sum(axis=1)


def sample(z, c, layers, rnd=round_bf16):
    """x [B][8] and sum_s [B] from base draws z [B][8] and per-row context c."""
    v = np.asarray(z, dtype=np.float64)
    tot = np.zeros(len(v))
    for l in range(len(layers)):
        o, _ = conditioner(conditioner_input(v, c, l, rnd), layers[l], rnd)
        v, ss = coupling(v, o, l, +1)
        tot += ss
    return v, tot


def density(x, c, layers, rnd=round_bf16):
    """(z, sum_s, tape) for x [B][8]; tape[l] = (X, g1, g2, o, w) of layer l, w its output."""
    v = np.asarray(x, dtype=np.float64)
    tot = np.zeros(len(v))
    tape = [None] * len(layers)
    for l in reversed(range(len(layers))):
        X = conditioner_input(v, c, l, rnd)
        o, (g1, g2) = conditioner(X, layers[l], rnd)
        v, ss = coupling(v, o, l, -1)
        tot += ss
        tape[l] = (X, g1, g2, o, v)
    return v, tot, tape


def log_normal(z):
    z = np.asarray(z, dtype=np.float64)
    return -0.5 * np.sum(z * z, axis=1) - 0.5 * NDIM * LN_2PI


def nll(z, sum_s):
    """Per-row -ln q_x(x) = |z|^2 / 2 + 4 ln(2 pi) + sum_s and its batch mean."""
    rows = -log_normal(z) + np.asarray(sum_s, dtype=np.float64)
    return rows, rows.mean()


def _dense_back(X, W, b, dy, act_relu, rnd_dz):
    """Chain rule of y = act(X W^T + b): (dX, dW, db).  The products take rnd_dz(dZ)."""
    z = X @ W.T + b[None, :]
    dz = dy * (relu_grad(z) if act_relu else 1.0)
    dzp = rnd_dz(dz)
    return dzp @ W, dzp.T @ X, dz.sum(axis=0)


def coupling_backward(l, w, o, G, row_weight):
    """Chain rule through one density step of layer l with output w and conditioner
    output o, given G = dL/dw and the weight of sum_s in the loss: returns
    (dL/do [B][8], dL/dv_in [B][8] without the conditioner's share)."""
    a, b = (list(t) for t in SPLITS[l % 4])
    _, s = shift_logscale(o)
    e = np.exp(-s)
    G = np.asarray(G, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Gb = G[:, b]
    dmu = -Gb * e
    ds = -Gb * w[:, b] + row_weight
    do = np.concatenate([dmu, ds * (1.0 - (s / S_MAX) ** 2)], axis=1)
    Gu = G.copy()
    Gu[:, b] = Gb * e
    return do, Gu


def input_backward(l, dX, Gu, dc):
    """Adds the conditioner input's gradient dX [B][8 + C] into the conditioning half of
    Gu and into the context gradient dc (both returned as new arrays)."""
    a, _ = SPLITS[l % 4]
    Gu = np.array(Gu, dtype=np.float64)
    Gu[:, list(a)] += dX[:, 0:4]
    return Gu, np.asarray(dc, dtype=np.float64) + dX[:, 8:]


def loss_and_grads(feat, x, params, K, rnd=round_bf16):
    """Mean training loss over rows (feat [B][F], x [B][8] standardised targets) and its
    gradient with respect to every parameter tensor (storage order)."""
    emb, layers = split_params(params, K)
    c, (h1, h2) = embed(feat, emb, rnd)
    z, ss, tape = density(x, c, layers, rnd)
    rows, mean = nll(z, ss)
    B = len(z)
    G = z / B                       # d mean / d z
    dc = np.zeros_like(c)
    layer_grads = [None] * K
    for l in range(K):              # the density pass applied K-1 .. 0, so 0 is undone first
        X, g1, g2, o, w = tape[l]
        do, Gu = coupling_backward(l, w, o, G, 1.0 / B)
        V1, e1, V2, e2, V3, e3 = layers[l]
        dg2, dV3, de3 = _dense_back(g2, V3, e3, do, False, rnd)
        dg1, dV2, de2 = _dense_back(g1, V2, e2, dg2, True, rnd)
        dX, dV1, de1 = _dense_back(X, V1, e1, dg1, True, rnd)
        G, dc = input_backward(l, dX, Gu, dc)
        layer_grads[l] = [dV1, de1, dV2, de2, dV3, de3]
    W1, b1, W2, b2, W3, b3 = emb
    dh2, dW3, db3 = _dense_back(h2, W3, b3, dc, False, rnd)
    dh1, dW2, db2 = _dense_back(h1, W2, b2, dh2, True, rnd)
    _, dW1, db1 = _dense_back(np.asarray(feat, dtype=np.float64), W1, b1, dh1, True, rnd)
    grads = [dW1, db1, dW2, db2, dW3, db3]
    for g in layer_grads:
        grads += g
    return mean, rows, grads


# ---------------------------------------------------------------- proposal

def base_uniforms(seed, counter, idx):
    """u [S][12]: u_{2j}, u_{2j+1} from Philox block j = 0..5 of each draw in idx."""
    k0, k1 = key_of(seed)
    idx = np.asarray(idx, dtype=np.uint64)
    u = np.zeros((len(idx), 12))
    for j in range(6):
        w = philox4x32_10((idx & np.uint64(0xFFFFFFFF)).astype(np.uint32), np.uint32(j), np.uint32(TAG_FLOW),
                          np.uint32(counter & 0xFFFFFFFF), k0, k1)
        u[:, 2 * j] = uniform52(w[0], w[1])
        u[:, 2 * j + 1] = uniform52(w[2], w[3])
    return u


def base_normals(seed, counter, idx):
    """(z [S][8], coin [S]) for global draw indices idx."""
    u = base_uniforms(seed, counter, idx)
    z = np.zeros((len(u), 8))
    for i in range(4):
        rad = np.sqrt(-2.0 * np.log(u[:, 2 * i]))
        z[:, 2 * i] = rad * np.cos(2.0 * math.pi * u[:, 2 * i + 1])
        z[:, 2 * i + 1] = rad * np.sin(2.0 * math.pi * u[:, 2 * i + 1])
    return z, u[:, 8]


def nuisance_uniforms(seed, counter, idx):
    """[S][3]: the uniforms of t_c, chi_1 and chi_2 (u_9, u_10, u_11) of draws idx."""
    return base_uniforms(seed, counter, idx)[:, 9:12]


def proposal_params(x, z, sum_s, mean, scale, prior, coin, nuis):
    """theta [11][S], ln q_r [S] and ln pi_r - ln q_r [S] of flow draws x (see the module
    docstring); nuis [S][3] the uniforms of t_c, chi_1, chi_2.  Rows outside the prior's
    support get -inf and in-range placeholder masses (m_lo), distance (d_lo) and clipped
    angles."""
    x = np.asarray(x, dtype=np.float64)
    S = len(x)
    r = np.asarray(mean)[None, :] + np.asarray(scale)[None, :] * x
    log_q = log_normal(z) - np.asarray(sum_s, dtype=np.float64) - np.sum(np.log(np.asarray(scale)))
    lp = log_prior_r(r, prior)
    nuis = np.asarray(nuis, dtype=np.float64)
    th = np.zeros((11, S))
    for i in range(S):
        Mc, q, D, ct, al, sd, psi, phi = r[i]
        if np.isfinite(lp[i]):
            big, small = masses(Mc, q)
            m1, m2 = (small, big) if coin[i] < 0.5 else (big, small)
            dist = D
        else:
            m1 = m2 = prior["m_lo"]
            dist = prior["d_lo"]
        th[0, i], th[1, i], th[4, i] = m1, m2, dist
        th[5, i] = prior["tc_lo"] + (prior["tc_hi"] - prior["tc_lo"]) * nuis[i, 0]
        th[2, i] = prior["chi_lo"] + (prior["chi_hi"] - prior["chi_lo"]) * nuis[i, 1]
        th[3, i] = prior["chi_lo"] + (prior["chi_hi"] - prior["chi_lo"]) * nuis[i, 2]
        th[6, i], th[8, i], th[9, i] = phi, psi, al
        th[7, i] = math.acos(min(1.0, max(-1.0, ct)))
        th[10, i] = math.asin(min(1.0, max(-1.0, sd)))
    return th, log_q, lp - log_q


def event_of(offsets, S):
    offsets = np.asarray(offsets, dtype=np.int64)
    E = len(offsets) - 1
    ev = np.searchsorted(offsets, np.arange(S), side="right") - 1
    return np.minimum(np.maximum(ev, 0), E - 1)


def sample_posterior(feat_events, params, K, mean, scale, prior, offsets, seed, counter, rnd=round_bf16):
    """Samples of event e in rows offsets[e] .. offsets[e+1]-1: (theta [11][S], ln q_r [S],
    ln pi_r - ln q_r [S])."""
    emb, layers = split_params(params, K)
    c, _ = embed(feat_events, emb, rnd)
    S = int(np.asarray(offsets)[-1])
    ev = event_of(offsets, S)
    z, coin = base_normals(seed, counter, np.arange(S))
    x, ss = sample(z, c[ev], layers, rnd)
    return proposal_params(x, z, ss, mean, scale, prior, coin, nuisance_uniforms(seed, counter, np.arange(S)))


def log_prob(feat, theta, params, K, mean, scale, rnd=round_bf16):
    """ln q_r(r(theta) | d) for each column of theta [11][B] with its row of features."""
    emb, layers = split_params(params, K)
    c, _ = embed(feat, emb, rnd)
    x = standardise(coords(theta), mean, scale)
    z, ss, _ = density(x, c, layers, rnd)
    return log_normal(z) - ss - np.sum(np.log(np.asarray(scale)))

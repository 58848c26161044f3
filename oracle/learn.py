"""The learned proposal's elementwise pieces (oracle; test infrastructure).

The paper trains a network on the simulated batches to produce a posterior estimator
(Sec. 4 embedding network, Sec. 5 normalizing flow, AdamW training) whose samples the
standard likelihood (Sec. 6) can judge.  The first learned proposal built here is the
simplest conditional flow: one affine (Gaussian) layer over three parameters, chirp mass
Mc, total mass M and luminosity distance D, whose mean and log-scale come from a dense
network of spectral features of the whitened strain.  This module states, in FP64:

* features  -- log of the mean power |Y_k|^2 / N of the whitened strain's rfft over
  groups of G consecutive bins from k_lo, per detector, zero-padded to F_pad columns;
* targets   -- (Mc, M, D) of each draw, standardised by given means and scales;
* gauss_nll -- per-row negative log-density of standardised targets t under
  N(mu, exp(s)^2) (without the constant): sum_p [ (t_p - mu_p)^2 e^{-2 s_p} / 2 + s_p ],
  its batch mean, and its gradient with respect to the network output (mu, s);
* adamw     -- one AdamW step (Loshchilov & Hutter 2019): moments, bias correction,
  decoupled weight decay;
* proposal  -- a draw of (m1, m2, D) from the Gaussian through (Mc, M) and the log ratio
  ln pi - ln q of the uniform prior in (m1, m2, D) to the proposal density.

Chirp mass Mc = (m1 m2)^{3/5} / M^{1/5}; the map (m1, m2) -> (Mc, M) is two-to-one
(m1 <-> m2) with |d(Mc, M)/d(m1, m2)| = (3/5) Mc |m1 - m2| / (m1 m2).
"""
import math

import numpy as np


def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def features(y, k_lo, G, F_pad):
    """[B][F_pad] FP64 features of whitened windows y [B][D][N]."""
    y = np.asarray(y, dtype=np.float64)
    B, D, N = y.shape
    P = np.abs(np.fft.rfft(y, axis=-1)) ** 2 / N
    ng = (N // 2 - k_lo) // G
    out = np.zeros((B, F_pad))
    for d in range(D):
        for g in range(ng):
            k = k_lo + g * G
            out[:, d * ng + g] = np.log(P[:, d, k:k + G].mean(axis=-1))
    return out


def targets(theta, mean, scale):
    """[B][3] standardised (Mc, M, D) from theta [11][B] (rows m1, m2, chi1, chi2, D, ...)."""
    th = np.asarray(theta, dtype=np.float64)
    m1, m2, D = th[0], th[1], th[4]
    raw = np.stack([chirp_mass(m1, m2), m1 + m2, D], axis=1)
    return (raw - np.asarray(mean)[None, :]) / np.asarray(scale)[None, :]


def gauss_nll(out, t):
    """out [B][>= 2P] (mu in columns 0..P-1, s in P..2P-1), t [B][P].  Returns (per-row
    loss [B], mean loss, gradient of the mean loss w.r.t. out (zero in other columns))."""
    out = np.asarray(out, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B, P = t.shape
    mu, s = out[:, :P], out[:, P:2 * P]
    r = (t - mu) * np.exp(-s)
    loss = np.sum(0.5 * r * r + s, axis=1)
    g = np.zeros_like(out)
    g[:, :P] = -(t - mu) * np.exp(-2.0 * s) / B
    g[:, P:2 * P] = (1.0 - r * r) / B
    return loss, loss.mean(), g


def adamw(p, g, m, v, lr, beta1, beta2, eps, wd, step):
    """One AdamW step (step counts from 1).  Returns (p', m', v')."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v


def proposal(mu, s, mean, scale, z, u, prior):
    """One draw per row: x = mean + scale (mu + e^s z) gives (Mc, M, D); m1 >= m2 solve
    Mc, M and are swapped when u < 1/2.  Returns (m1, m2, D, log_ratio) where log_ratio =
    ln pi(m1, m2, D) - ln q(m1, m2, D) (uniform prior box; -inf outside it or where
    (Mc, M) has no masses)."""
    mu, s, z = (np.asarray(a, dtype=np.float64) for a in (mu, s, z))
    x = np.asarray(mean)[None, :] + np.asarray(scale)[None, :] * (mu + np.exp(s) * z)
    Mc, M, D = x[:, 0], x[:, 1], x[:, 2]
    n = len(Mc)
    m1 = np.full(n, np.nan)
    m2 = np.full(n, np.nan)
    lr = np.full(n, -np.inf)
    log_box = -math.log((prior["m_hi"] - prior["m_lo"]) ** 2 * (prior["d_hi"] - prior["d_lo"]))
    for i in range(n):
        if not (M[i] > 0 and Mc[i] > 0):
            continue
        eta = (Mc[i] / M[i]) ** (5.0 / 3.0)
        if eta > 0.25:
            continue
        root = math.sqrt(1.0 - 4.0 * eta)
        a, b = 0.5 * M[i] * (1.0 + root), 0.5 * M[i] * (1.0 - root)
        if u[i] < 0.5:
            a, b = b, a
        m1[i], m2[i] = a, b
        inside = (prior["m_lo"] <= a <= prior["m_hi"] and prior["m_lo"] <= b <= prior["m_hi"]
                  and prior["d_lo"] <= D[i] <= prior["d_hi"] and a != b)
        if not inside:
            continue
        # density of x (three independent normals, physical units) and the two-to-one Jacobian
        log_qx = 0.0
        for p in range(3):
            zz = (x[i, p] - (mean[p] + scale[p] * mu[i, p])) / (scale[p] * math.exp(s[i, p]))
            log_qx += -0.5 * zz * zz - math.log(scale[p] * math.exp(s[i, p])) - 0.5 * math.log(2.0 * math.pi)
        jac = 0.6 * Mc[i] * abs(a - b) / (a * b)
        lr[i] = log_box - (log_qx + math.log(jac) - math.log(2.0))
    return m1, m2, D, lr

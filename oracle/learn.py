"""The learned proposal's elementwise pieces (oracle; test infrastructure).

The paper trains a network on the simulated batches to produce a posterior estimator
(Sec. 4 embedding network, Sec. 5 normalizing flow, AdamW training) whose samples the
standard likelihood (Sec. 6) can judge.  The first learned proposal built here is the
simplest conditional flow: one affine (Gaussian) layer over three parameters, chirp mass
Mc, total mass M and luminosity distance D, whose mean and log-scale come from a dense
network of spectral features of the whitened strain.  This module states, in FP64:

* features  -- log of the mean power |Y_k|^2 / N of the whitened strain's rfft over
  groups of G consecutive bins from k_lo, per detector, zero-padded to F_pad columns;
* cross_features -- per detector pair (d1 < d2) and group, the normalised cross spectrum
  rho = sum_k Y_d1,k conj(Y_d2,k) / sqrt(sum_k |Y_d1,k|^2 sum_k |Y_d2,k|^2) (real and
  imaginary parts): unchanged by a common time shift of all detectors (the shift's phase
  factor cancels in the product), so it carries the inter-detector delay and amplitude
  ratio that localise the source without the arrival time;
* lag_features -- per detector and group, the normalised lag-one spectral product
  lam = sum_k Y_k conj(Y_{k+1}) / sqrt(sum_k |Y_k|^2 sum_k |Y_{k+1}|^2) (real and imaginary
  parts): for a signal its phase is 2 pi t(f) / T, t(f) the time at which the signal
  passes frequency f (the chirp's time-frequency track, which fixes the chirp mass); a
  common time shift by s samples adds 2 pi s / N to every phase;
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


def detector_pairs(D):
    return [(a, b) for a in range(D) for b in range(a + 1, D)]


def cross_features(y, k_lo, G):
    """[B][2 P ng] normalised cross spectra of whitened windows y [B][D][N]: for pair p
    (detector_pairs order) and group g, column 2 p ng + g holds Re rho, (2 p + 1) ng + g
    holds Im rho."""
    y = np.asarray(y, dtype=np.float64)
    B, D, N = y.shape
    Y = np.fft.rfft(y, axis=-1)
    ng = (N // 2 - k_lo) // G
    pairs = detector_pairs(D)
    out = np.zeros((B, 2 * len(pairs) * ng))
    for p, (a, b) in enumerate(pairs):
        for g in range(ng):
            k = k_lo + g * G
            ya, yb = Y[:, a, k:k + G], Y[:, b, k:k + G]
            rho = np.sum(ya * np.conj(yb), axis=-1) / np.sqrt(np.sum(np.abs(ya) ** 2, axis=-1) *
                                                             np.sum(np.abs(yb) ** 2, axis=-1))
            out[:, 2 * p * ng + g] = rho.real
            out[:, (2 * p + 1) * ng + g] = rho.imag
    return out


def lag_features(y, k_lo, G):
    """[B][2 D ng] normalised lag-one spectral products of whitened windows y [B][D][N]:
    for detector d and group g (bins k = k_lo + g G .. k_lo + g G + G - 1, each paired with
    k + 1), column 2 d ng + g holds Re lam, (2 d + 1) ng + g holds Im lam."""
    y = np.asarray(y, dtype=np.float64)
    B, D, N = y.shape
    Y = np.fft.rfft(y, axis=-1)
    ng = (N // 2 - k_lo) // G
    out = np.zeros((B, 2 * D * ng))
    for d in range(D):
        for g in range(ng):
            k = k_lo + g * G
            a, b = Y[:, d, k:k + G], Y[:, d, k + 1:k + G + 1]
            lam = np.sum(a * np.conj(b), axis=-1) / np.sqrt(np.sum(np.abs(a) ** 2, axis=-1) *
                                                           np.sum(np.abs(b) ** 2, axis=-1))
            out[:, 2 * d * ng + g] = lam.real
            out[:, (2 * d + 1) * ng + g] = lam.imag
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


def adamw(p, g, m, v, lr, beta1, beta2, eps, wd, step, clip=None):
    """One AdamW step (step counts from 1).  Returns (p', m', v').  With clip, the
    gradient is first scaled by min(1, clip / |g|) (global Euclidean norm)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    if clip is not None:
        norm = math.sqrt(float(np.sum(g * g)))
        if norm > clip:
            g = g * (clip / norm)
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


TAG_PROPOSAL = 3


def proposal_uniforms(seed, counter, idx):
    """Ten uniforms per sample from Philox4x32-10: block j (0..4) of sample s has counter
    (s, j, TAG_PROPOSAL, counter) and gives uniform52(w0, w1), uniform52(w2, w3)."""
    from .philox import key_of, philox4x32_10, uniform52
    k0, k1 = key_of(seed)
    idx = np.asarray(idx, dtype=np.uint64)
    out = np.zeros((len(idx), 10))
    for j in range(5):
        w = philox4x32_10((idx & np.uint64(0xFFFFFFFF)).astype(np.uint32), np.uint32(j), np.uint32(TAG_PROPOSAL),
                          np.uint32(counter & 0xFFFFFFFF), k0, k1)
        out[:, 2 * j] = uniform52(w[0], w[1])
        out[:, 2 * j + 1] = uniform52(w[2], w[3])
    return out


def sample_proposal(net_out, mean, scale, prior, truth, offsets, seed, counter, fix_angles=False):
    """Samples for importance sampling, event e owning rows offsets[e] .. offsets[e+1]-1.

    Uniforms u[0..9] of sample s (proposal_uniforms): normals z0, z1 = r (cos, sin)(2 pi u1)
    with r = sqrt(-2 ln u0), z2 = sqrt(-2 ln u2) cos(2 pi u3); u4 orders the masses; phic,
    psi, RA = lo + (hi - lo) u5, u6, 2 pi u8 (psi, phic ranges from the prior, RA in
    [0, 2 pi)); theta_JN = acos(2 u7 - 1); dec = asin(2 u9 - 1); spins and t_c are the
    event's own (truth [11][E]); with fix_angles so are phic, theta_JN, psi, RA and dec
    (the proposal then covers m1, m2, D only).  With net_out (rows per event: mu in columns 0..2, s in
    3..5) the masses and distance come from proposal() with log ratio ln pi - ln q;
    without it (the prior as proposal) m1 = lo + (hi - lo) u0, m2 likewise with u2,
    D = d_lo + (d_hi - d_lo) u1, log ratio 0.  Returns (theta [11][S], log_ratio [S])."""
    offsets = np.asarray(offsets, dtype=np.int64)
    S = int(offsets[-1])
    E = len(offsets) - 1
    ev = np.searchsorted(offsets, np.arange(S), side="right") - 1
    ev = np.minimum(np.maximum(ev, 0), E - 1)
    u = proposal_uniforms(seed, counter, np.arange(S))
    truth = np.asarray(truth, dtype=np.float64)
    th = np.zeros((11, S))
    th[2], th[3], th[5] = truth[2][ev], truth[3][ev], truth[5][ev]
    th[6] = prior["phi_lo"] + (prior["phi_hi"] - prior["phi_lo"]) * u[:, 5]
    th[8] = prior["psi_lo"] + (prior["psi_hi"] - prior["psi_lo"]) * u[:, 6]
    th[7] = np.arccos(2.0 * u[:, 7] - 1.0)
    th[9] = 2.0 * math.pi * u[:, 8]
    th[10] = np.arcsin(2.0 * u[:, 9] - 1.0)
    if fix_angles:
        for r in (6, 7, 8, 9, 10):
            th[r] = truth[r][ev]
    if net_out is None:
        th[0] = prior["m_lo"] + (prior["m_hi"] - prior["m_lo"]) * u[:, 0]
        th[1] = prior["m_lo"] + (prior["m_hi"] - prior["m_lo"]) * u[:, 2]
        th[4] = prior["d_lo"] + (prior["d_hi"] - prior["d_lo"]) * u[:, 1]
        return th, np.zeros(S)
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    z = np.stack([r01 * np.cos(2.0 * math.pi * u[:, 1]), r01 * np.sin(2.0 * math.pi * u[:, 1]),
                  np.sqrt(-2.0 * np.log(u[:, 2])) * np.cos(2.0 * math.pi * u[:, 3])], axis=1)
    out = np.asarray(net_out, dtype=np.float64)[ev]
    m1, m2, D, lr = proposal(out[:, 0:3], out[:, 3:6], mean, scale, z, u[:, 4], prior)
    bad = ~np.isfinite(m1)
    th[0] = np.where(bad, prior["m_lo"], m1)
    th[1] = np.where(bad, prior["m_lo"], m2)
    th[4] = np.where(np.isfinite(D), D, prior["d_lo"])
    return th, lr

"""VICReg loss of two views' representations (oracle; test infrastructure).

Sec. 4.1 of the paper pre-trains its data summary so that two views of the same signal,
differing only in the time of arrival, map to the same representation, using the
Variance-Invariance-Covariance Regularisation loss of Bardes, Ponce and LeCun (2022) on
expanded representations x, x' [B][d] of the two views, with weights (lambda1, lambda2,
lambda3) = (1, 1, 5) in the paper's best configuration:

  L = lambda1 inv(x, x') + lambda2 (v(x) + v(x')) + lambda3 (c(x) + c(x')),
  inv(x, x') = (1 / (B d)) sum_b sum_j (x_bj - x'_bj)^2                    (mean squared error),
  v(x)       = (1 / d) sum_j max(0, gamma - sqrt(Var_j(x) + eps))        (variance hinge),
  c(x)       = (1 / d) sum_{i != j} C_ij(x)^2                             (off-diagonal covariance),

with Var_j and C the unbiased (B - 1) sample variance and covariance over the batch,
gamma = 1 and eps = 1e-4 (VICReg's values).  The paper prints the variance term without
the hinge; it is read here as VICReg defines it (without the hinge, minimising the term
would collapse the representation, the failure the term exists to prevent).

Gradient (chain rule, stated for x; x' is symmetric):
  d inv / d x_bj = 2 (x_bj - x'_bj) / (B d),
  d v / d x_bj   = -(1 / d) [S_j < gamma] (x_bj - mean_j) / ((B - 1) S_j),  S_j = sqrt(Var_j + eps),
  d c / d x_bk   = (4 / (d (B - 1))) sum_{j != k} C_kj (x_bj - mean_j).
"""
import numpy as np

GAMMA = 1.0
EPS = 1e-4


def _stats(x):
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    xc = x - x.mean(axis=0)[None, :]
    C = xc.T @ xc / (B - 1)
    return xc, C


def terms(x, xp):
    """(inv, v(x), v(x'), c(x), c(x'))."""
    x = np.asarray(x, dtype=np.float64)
    xp = np.asarray(xp, dtype=np.float64)
    B, d = x.shape
    inv = np.sum((x - xp) ** 2) / (B * d)
    out = [inv]
    for z in (x, xp):
        _, C = _stats(z)
        S = np.sqrt(np.diag(C) + EPS)
        out.append(np.sum(np.maximum(0.0, GAMMA - S)) / d)
    for z in (x, xp):
        _, C = _stats(z)
        off = C - np.diag(np.diag(C))
        out.append(np.sum(off ** 2) / d)
    return tuple(out)


def loss(x, xp, lam=(1.0, 1.0, 5.0)):
    inv, vx, vxp, cx, cxp = terms(x, xp)
    return lam[0] * inv + lam[1] * (vx + vxp) + lam[2] * (cx + cxp)


def grad(x, xp, lam=(1.0, 1.0, 5.0)):
    """(dL/dx, dL/dx') [B][d]."""
    x = np.asarray(x, dtype=np.float64)
    xp = np.asarray(xp, dtype=np.float64)
    B, d = x.shape
    out = []
    for z, other in ((x, xp), (xp, x)):
        g = lam[0] * 2.0 * (z - other) / (B * d)
        zc, C = _stats(z)
        S = np.sqrt(np.diag(C) + EPS)
        active = (S < GAMMA).astype(np.float64)
        g = g - lam[1] * (active / ((B - 1) * S))[None, :] * zc / d
        off = C - np.diag(np.diag(C))
        g = g + lam[2] * 4.0 / (d * (B - 1)) * (zc @ off)
        out.append(g)
    return out[0], out[1]


TAG_RETIME = 5


def retime(theta, tc_lo, tc_hi, seed, counter):
    """The second view's parameters: theta [11][B] with tc redrawn uniformly in
    [tc_lo, tc_hi]; u = uniform52 of Philox4x32-10 words 0, 1 at counter
    (b, 0, TAG_RETIME, counter), key seed."""
    from .philox import key_of, philox4x32_10, uniform52
    th = np.array(theta, dtype=np.float64, copy=True)
    B = th.shape[1]
    k0, k1 = key_of(seed)
    w = philox4x32_10(np.arange(B, dtype=np.uint64).astype(np.uint32), np.uint32(0), np.uint32(TAG_RETIME),
                      np.uint32(counter & 0xFFFFFFFF), k0, k1)
    th[5] = tc_lo + (tc_hi - tc_lo) * uniform52(w[0], w[1])
    return th

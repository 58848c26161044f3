"""Pins of the VICReg oracle (oracle/vicreg.py): the gradient against central
differences, and the special cases that fix each term."""
import math

import numpy as np

from oracle import vicreg as vr


def test_gradient_by_central_differences():
    rng = np.random.default_rng(1)
    B, d = 9, 5
    x = rng.normal(0, 0.6, (B, d))            # std below gamma: the hinge is active
    xp = x + rng.normal(0, 0.3, (B, d))
    xp[:, 0] *= 3.0                            # one dimension above gamma: inactive there
    gx, gxp = vr.grad(x, xp)
    h = 1e-6
    for arr, g in ((x, gx), (xp, gxp)):
        for _ in range(12):
            b, j = rng.integers(0, B), rng.integers(0, d)
            ap, am = arr.copy(), arr.copy()
            ap[b, j] += h
            am[b, j] -= h
            if arr is x:
                fd = (vr.loss(ap, xp) - vr.loss(am, xp)) / (2 * h)
            else:
                fd = (vr.loss(x, ap) - vr.loss(x, am)) / (2 * h)
            assert abs(fd - g[b, j]) < 1e-6 + 1e-5 * abs(g[b, j]), (fd, g[b, j])


def test_special_cases():
    rng = np.random.default_rng(2)
    B, d = 64, 6
    x = rng.normal(0, 2.0, (B, d))
    inv, vx, vxp, cx, cxp = vr.terms(x, x)
    assert inv == 0.0 and vx == vxp and cx == cxp            # identical views
    # a collapsed representation pays the whole hinge: gamma - sqrt(eps) per dimension
    col = np.ones((B, d)) * 3.0
    _, v, _, c, _ = vr.terms(col, col)
    assert abs(v - (vr.GAMMA - math.sqrt(vr.EPS))) < 1e-12 and c == 0.0
    # columns that are centred and orthogonal have no covariance; unit-or-larger std, no hinge
    q, _ = np.linalg.qr(rng.normal(size=(B, d)))
    z = q - q.mean(axis=0)
    z, _ = np.linalg.qr(z)
    z = z * np.sqrt(B - 1) * 1.5
    z -= z.mean(axis=0)
    _, v, _, c, _ = vr.terms(z, z)
    assert v == 0.0 and c < 1e-20
    # symmetry in the two views
    y = rng.normal(size=(B, d))
    assert abs(vr.loss(x, y) - vr.loss(y, x)) < 1e-12
    # the covariance term scales with the fourth power of the representation
    _, _, _, c1, _ = vr.terms(x, x)
    _, _, _, c2, _ = vr.terms(2 * x, 2 * x)
    assert abs(c2 - 16 * c1) < 1e-9 * c2

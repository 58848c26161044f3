"""Pins of the ResNet-1D oracle (oracle/resnet.py): convolution against brute force (the
network's direct tap-by-tap form and the im2col helper), the backward by the adjoint
identities, the im2col/col2im adjoint pair, group normalisation's statistics and gradient, max pooling,
and the whole network's gradient against central differences."""
import numpy as np
import pytest

from oracle import resnet as rn
from oracle.flow import exact

SMALL = ((8, 2, 1), (16, 1, 2), (16, 1, 2))


@pytest.mark.parametrize("k,s,p", [(7, 2, 3), (5, 1, 2), (5, 2, 2), (1, 2, 0)])
def test_conv_matches_brute_force(k, s, p):
    rng = np.random.default_rng(k * 10 + s)
    B, T, C, O = 2, 23, 3, 4
    x = rng.normal(size=(B, T, C))
    W = rng.normal(size=(O, k * C))
    y, _ = rn.conv(x, W, k, s, p)
    To = (T + 2 * p - k) // s + 1
    assert y.shape == (B, To, O)
    ref = np.zeros((B, To, O))
    for b in range(B):
        for t in range(To):
            for o in range(O):
                for j in range(k):
                    src = s * t + j - p
                    if 0 <= src < T:
                        ref[b, t, o] += sum(W[o, j * C + c] * x[b, src, c] for c in range(C))
    np.testing.assert_allclose(y, ref, atol=1e-12)


@pytest.mark.parametrize("k,s,p", [(7, 2, 3), (5, 1, 2), (5, 2, 2), (1, 2, 0), (3, 1, 1)])
def test_direct_convolution_and_its_backward(k, s, p):
    """The network's convolution (conv_direct, tap by tap) equals a brute-force sum and the
    im2col product; its backward equals the adjoint identity <dy, conv(x)> = <dx, x> and
    <dy, conv(x, W)> = <dW, W> (linearity in x and in W), and the im2col route; padded
    columns of W (the stem's) neither enter nor get a gradient."""
    rng = np.random.default_rng(100 * k + 10 * s + p)
    B, T, C, O = 2, 21, 3, 4
    K = k * C + 5                      # extra zero-weight columns, as the stem's padding
    x = rng.normal(size=(B, T, C))
    W = rng.normal(size=(O, K))
    W[:, k * C:] = 0.0
    y = rn.conv_direct(x, W, k, s, p)
    To = (T + 2 * p - k) // s + 1
    ref = np.zeros((B, To, O))
    for b in range(B):
        for t in range(To):
            for j in range(k):
                src = s * t + j - p
                if 0 <= src < T:
                    ref[b, t] += W[:, j * C:(j + 1) * C] @ x[b, src]
    np.testing.assert_allclose(y, ref, atol=1e-12)
    np.testing.assert_allclose(y, rn.conv(x, W, k, s, p)[0], atol=1e-12)
    dy = rng.normal(size=(B, To, O))
    dx, dW = rn.conv_backward_direct(dy, x, W, k, s, p)
    assert dW.shape == W.shape and np.all(dW[:, k * C:] == 0.0)
    np.testing.assert_allclose(np.sum(dy * y), np.sum(dx * x), rtol=1e-12)
    np.testing.assert_allclose(np.sum(dy * y), np.sum(dW * W), rtol=1e-12)
    cols = rn.im2col(x, k, s, p, K)
    np.testing.assert_allclose(dx, rn.col2im((dy.reshape(-1, O) @ W).reshape(B, To, K), T, C, k, s, p), atol=1e-12)
    np.testing.assert_allclose(dW, dy.reshape(-1, O).T @ cols.reshape(-1, K), atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(3)
    for (k, s, p) in [(7, 2, 3), (5, 1, 2), (5, 2, 2), (1, 2, 0)]:
        x = rng.normal(size=(2, 19, 3))
        cols = rn.im2col(x, k, s, p)
        Y = rng.normal(size=cols.shape)
        lhs = np.sum(cols * Y)
        rhs = np.sum(x * rn.col2im(Y, 19, 3, k, s, p))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_group_norm_statistics_and_gradient():
    rng = np.random.default_rng(4)
    z = rng.normal(2.0, 3.0, (2, 10, 16))
    y, xh, r = rn.gn(z, np.ones(16), np.zeros(16))
    g = y.reshape(2, 10, rn.GROUPS, 2)
    np.testing.assert_allclose(g.mean(axis=(1, 3)), 0.0, atol=1e-12)
    np.testing.assert_allclose(g.var(axis=(1, 3)), 1.0 / (1.0 + rn.EPS * r ** 2), rtol=1e-9)
    gamma, beta = rng.normal(size=16), rng.normal(size=16)
    dy = rng.normal(size=z.shape)
    _, xh, r = rn.gn(z, gamma, beta)
    dz, dg, db = rn.gn_back(dy, xh, r, gamma)
    h = 1e-6
    for _ in range(10):
        i = tuple(rng.integers(0, n) for n in z.shape)
        zp, zm = z.copy(), z.copy()
        zp[i] += h
        zm[i] -= h
        fd = (np.sum(dy * rn.gn(zp, gamma, beta)[0]) - np.sum(dy * rn.gn(zm, gamma, beta)[0])) / (2 * h)
        assert abs(fd - dz[i]) < 1e-6 * max(1.0, abs(fd))
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1)))
    np.testing.assert_allclose(dg, np.sum(dy * xh, axis=(0, 1)))


def test_maxpool_brute_force():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 11, 3))
    y, arg = rn.maxpool(x)
    assert y.shape == (2, 6, 3)
    for b in range(2):
        for t in range(6):
            for c in range(3):
                win = [x[b, i, c] for i in (2 * t - 1, 2 * t, 2 * t + 1) if 0 <= i < 11]
                assert y[b, t, c] == max(win)


def test_network_gradient_by_central_differences():
    rng = np.random.default_rng(6)
    D, C = 2, 6
    P = rn.init_params(rng, D, C, SMALL)
    y = rng.normal(size=(2, D, 64))
    c, tape = rn.forward(y, P, exact)
    assert c.shape == (2, C)
    dc = rng.normal(size=c.shape)
    G = rn.backward(dc, P, tape, exact)

    def loss(P2):
        return float(np.sum(dc * rn.forward(y, P2, exact)[0]))

    import copy
    h = 1e-6
    checks = [("Wf", None), ("bf", None), ("W0", None), ("g0", None), ("b0", None)]
    for bi in range(len(P["blocks"])):
        for key in P["blocks"][bi]:
            if key != "s":
                checks.append((key, bi))
    for key, bi in checks:
        arr = P[key] if bi is None else P["blocks"][bi][key]
        grad = G[key] if bi is None else G["blocks"][bi][key]
        for _ in range(2):
            i = tuple(rng.integers(0, n) for n in arr.shape)
            if key == "W0" and i[1] >= 7 * D:
                continue
            Pp, Pm = copy.deepcopy(P), copy.deepcopy(P)
            (Pp[key] if bi is None else Pp["blocks"][bi][key])[i] += h
            (Pm[key] if bi is None else Pm["blocks"][bi][key])[i] -= h
            fd = (loss(Pp) - loss(Pm)) / (2 * h)
            assert abs(fd - grad[i]) < 1e-5 * max(1.0, abs(fd)), (key, bi, i, fd, grad[i])

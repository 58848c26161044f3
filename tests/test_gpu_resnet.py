"""ResNet-1D data summary on the GPU (paper_2407_19048_gb300.resnet) against
oracle.resnet (needs a GPU), element by element.

Whole network (representation and every gradient tensor): the oracle rounds to bfloat16
at the same points but sums convolutions and statistics in FP64, so activations next to
a rounding boundary can flip by one bfloat16 ulp and propagate; each element is held to
its own bound from tests/rounding_bounds.py (the oracle's chain re-run with FP32-sized
perturbations at every product and rounding point; SAFETY x the spread plus the FP32
bound of the final product).  That runs on the two-stage network at the training input
length (2 x 2048): at random initialisation the full (5, 3, 3) stack is chaotic (one
flip or moved max-pool argument shifts the stem's gradient by tens of per cent, and an
FP32 emulation of the network on the host leaves such perturbation bounds), so the full
network is checked layer by layer instead: every operation of its forward and backward
pass at the training shape (B = 64 windows of 2 x 2048 samples; the weight gradient's
split-K product over the 262,144 rows of a 512-window batch), each against a bound from
its own arithmetic: FP32 outputs within 2 K 2^-24 sum |a b| (K the summed terms),
bfloat16 outputs exact unless the oracle's value before rounding lies within that FP32
bound of a rounding boundary (then one ulp), copies and pooling bit-exact."""
import numpy as np
import pytest

from oracle import resnet as rn
from oracle.flow import round_bf16

import rounding_bounds as rb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = ((8, 2, 1), (16, 1, 2), (16, 1, 2))


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def _bf16_exact(P):
    """Weights rounded to bfloat16 values, so the GPU copies equal the masters."""
    from oracle.flow import round_bf16
    out = {}
    for k, v in P.items():
        if k == "blocks":
            out[k] = [{kk: (vv if kk == "s" else (round_bf16(vv) if kk.startswith("W") else vv))
                       for kk, vv in b.items()} for b in v]
        else:
            out[k] = round_bf16(v) if k.startswith("W") else v
    return out


@pytest.mark.parametrize("N,B", [(256, 8), (2048, 16)])
def test_forward_and_backward_match_oracle(gwx, N, B):
    from paper_2407_19048_gb300.resnet import ResNet1D
    rng = np.random.default_rng(N + B)
    D, C = 2, 8
    P = _bf16_exact(rn.init_params(rng, D, C, SMALL))
    y = rng.normal(size=(B, D, N)).astype(np.float32)
    net = ResNet1D(D, C, stages=SMALL, params=P)
    c = net.forward(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    c_ref, tape = rn.forward(y.astype(np.float64), P)
    dc = rng.normal(size=c.shape).astype(np.float32)
    G = net.backward(torch.from_numpy(dc).cuda())
    G_ref = rb._flat_grads(rn.backward(dc.astype(np.float64), P, tape))
    cv, cb, Gv, Gb = rb.resnet(y.astype(np.float64), P, dc.astype(np.float64))
    assert np.array_equal(cv, c_ref)                  # the bound's chain reproduces the oracle
    _within(c, c_ref, cb, "representation")
    for k, ref in G_ref.items():
        assert np.array_equal(Gv[k], ref)
        _within(G[k].cpu().numpy().astype(np.float64), ref, Gb[k], "gradient " + k)


def _within(got, ref, bound, what):
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    tol = bound + 1e-12 * np.abs(ref) + 1e-30
    bad = err > tol
    assert not bad.any(), (what, int(bad.sum()), float(err[bad].max()), float(tol[bad].min()),
                           np.argwhere(bad)[:5].tolist())


def test_training_the_summary_lowers_a_regression_loss(gwx):
    """The summary learns to read chirp mass out of simulated whitened strain."""
    import workloads
    from paper_2407_19048_gb300.resnet import ResNet1D
    from paper_2407_19048_gb300.simulator import Simulator
    wl = workloads.workload("small", B=256)
    sim = Simulator(wl)
    net = ResNet1D(2, 8, stages=SMALL, seed=3)
    mom = {name: (torch.zeros_like(p), torch.zeros_like(p)) for name, p, _ in net.tensors()}
    losses = []
    for step in range(150):
        y, th, _ = sim.step(step)
        t = gwx.flow_targets(th, [25.0, 0.6, 1100.0, 0, 3.14, 0, 3.14, 3.14], [8.0, 0.2, 520.0, 1, 1.8, 1, 1.8, 1.8])
        c = net.forward(y)
        diff = c[:, 0] - t[:, 0]
        losses.append(float((diff ** 2).mean()))
        dc = torch.zeros_like(c)
        dc[:, 0] = 2.0 * diff / len(diff)
        G = net.backward(dc)
        for name, p, p16 in net.tensors():
            m, v = mom[name]
            gwx.adamw(p, G[name].contiguous(), m, v, step + 1, 1e-3, param_bf16=p16)
    assert np.mean(losses[-15:]) < 0.7 * np.mean(losses[:15]), (np.mean(losses[:15]), np.mean(losses[-15:]))


# ---------------------------------------------------------------- layer by layer
U32 = 2.0 ** -24


def _rnd_bound(v, e):
    """Largest |rnd(v') - rnd(v)| over |v' - v| <= e, rnd = bfloat16 nearest even: zero
    unless a rounding boundary lies within e of v."""
    r = round_bf16(v)
    return np.maximum(round_bf16(v + e) - r, r - round_bf16(v - e))


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(dtype)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _bf(rng, shape, scale=1.0):
    return round_bf16(rng.normal(0.0, scale, shape))


def _gn_bounds(z, gamma, beta, res, G=8):
    """Oracle group norm (pre-activation y = gamma xhat + beta + res, xhat, rstd, mean) and
    the FP32 bounds of the GPU's y and xhat: statistics from FP32 runs of at most 64
    terms of values shifted by the group's first value (mean within 64 2^-24 of their mean
    absolute deviation, variance within 64 2^-24 relative of the shifted second moment),
    then a few FP32 operations per element."""
    B, T, C = z.shape
    y0, xh, rstd = rn.gn(z, gamma, beta, G)
    zg = z.reshape(B, T, G, C // G)
    mean = zg.mean(axis=(1, 3), keepdims=True)
    # the shift is one of the group's values: bound its distance from the mean by the largest
    spread = np.abs(zg - mean).max(axis=(1, 3), keepdims=True)
    dev1 = np.abs(zg - mean).mean(axis=(1, 3), keepdims=True) + spread
    mom2 = ((zg - mean) ** 2).mean(axis=(1, 3), keepdims=True) + spread ** 2
    r = rstd.reshape(B, 1, G, 1)
    e_mean = 64 * U32 * dev1
    e_rstd_rel = 0.5 * 64 * U32 * mom2 * r * r + 4 * U32
    xhg = xh.reshape(B, T, G, C // G)
    e_xh = (np.abs(xhg) * e_rstd_rel + r * (e_mean + 4 * U32 * (np.abs(zg) + np.abs(mean)))).reshape(B, T, C)
    y = y0 + (0.0 if res is None else res)
    e_y = np.abs(gamma) * e_xh + 4 * U32 * (np.abs(gamma * xh) + np.abs(beta) + (0 if res is None else np.abs(res))
                                            + np.abs(y))
    return y, xh, rstd, e_xh, e_y, np.broadcast_to(e_rstd_rel, zg.shape).reshape(B, T, C)


@pytest.mark.parametrize("B,T,C", [(3, 37, 96), (2, 50, 64), (2, 33, 24), (4, 64, 256), (64, 512, 64),
                                   (64, 128, 256)])
def test_group_norm_kernels(gwx, B, T, C):
    """gwx_group_norm (residual, ReLU, bfloat16 and FP32 outputs) and
    gwx_group_norm_backward against oracle.resnet's gn / gn_back on values with a mean far
    from zero, element by element.  The shapes take each kernel path: C = 96 per group with
    four-channel loads, C = 64 and 256 per sample (the training shapes of the first and
    last stage, B = 64), C = 24 (three channels per group) one channel at a time."""
    from paper_2407_19048_gb300 import _lib
    lib = _lib.load()
    G = 8
    rng = np.random.default_rng(B * 1000 + T + C)
    z = (3.0 + 2.0 * rng.normal(size=(B, T, C))).astype(np.float32).astype(np.float64)
    g = (1.0 + 0.1 * rng.normal(size=C)).astype(np.float32).astype(np.float64)
    b = (0.1 * rng.normal(size=C)).astype(np.float32).astype(np.float64)
    res = rng.normal(size=(B, T, C)).astype(np.float32).astype(np.float64)
    dy = rng.normal(size=(B, T, C)).astype(np.float32).astype(np.float64)
    Z, Gm, Bt, R, DY = (_t(a, torch.float32) for a in (z, g, b, res, dy))
    out32 = torch.empty_like(Z)
    out16 = torch.empty(Z.shape, dtype=torch.bfloat16, device="cuda")
    ms = torch.empty((B, G, 2), dtype=torch.float32, device="cuda")
    gwx._check(lib.gwx_group_norm(gwx._ptr(Z), B, T, C, G, gwx._ptr(Gm), gwx._ptr(Bt), gwx._ptr(R), None, 1,
                                  gwx._ptr(out16), gwx._ptr(out32), gwx._ptr(ms), gwx._stream()))
    y, xh, rstd, e_xh, e_y, e_rstd_rel = _gn_bounds(z, g, b, res, G)
    ref = np.maximum(y, 0.0)
    e_out = np.where(y + e_y <= 0.0, 0.0, e_y)          # surely negative before the ReLU: 0 on both sides
    _within(_np(out32), ref, e_out, "group norm FP32 output")
    _within(_np(out16), round_bf16(ref), _rnd_bound(ref, e_out), "group norm bfloat16 output")
    dz = torch.empty_like(Z)
    dg = torch.empty(C, dtype=torch.float32, device="cuda")
    db = torch.empty(C, dtype=torch.float32, device="cuda")
    nb = lib.gwx_group_norm_backward_scratch(B, C, G)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    gwx._check(lib.gwx_group_norm_backward(gwx._ptr(DY), gwx._ptr(Z), B, T, C, G, gwx._ptr(ms), gwx._ptr(Gm),
                                           gwx._ptr(scratch), gwx._ptr(dz), gwx._ptr(dg), gwx._ptr(db),
                                           gwx._stream()))
    dz_ref, dg_ref, db_ref = rn.gn_back(dy, xh, rstd, g, G)
    # dz = rstd (dxh - m1 - xhat m2), dxh = dy gamma, m1 and m2 group means (FP32 runs of
    # at most 64 terms); each factor's error through the expression, plus its FP32 roundings
    dxh = (dy * g).reshape(B, T, G, C // G)
    xg = xh.reshape(B, T, G, C // G)
    exg = e_xh.reshape(B, T, G, C // G)
    r = rstd.reshape(B, 1, G, 1)
    m1 = dxh.mean(axis=(1, 3), keepdims=True)
    m2 = (dxh * xg).mean(axis=(1, 3), keepdims=True)
    e_m1 = 64 * U32 * np.abs(dxh).mean(axis=(1, 3), keepdims=True)
    e_m2 = 64 * U32 * np.abs(dxh * xg).mean(axis=(1, 3), keepdims=True) + (np.abs(dxh) * exg).mean(axis=(1, 3),
                                                                                                     keepdims=True)
    inner = np.abs(dxh) + np.abs(m1) + np.abs(xg * m2)
    e_in = 4 * U32 * inner + e_m1 + np.abs(xg) * e_m2 + exg * np.abs(m2)
    e_dz = (r * e_in).reshape(B, T, C) + np.abs(dz_ref) * (e_rstd_rel + 4 * U32)
    e_dg = 64 * U32 * np.sum(np.abs(dy * xh), axis=(0, 1)) + np.sum(np.abs(dy) * e_xh, axis=(0, 1))
    e_db = 64 * U32 * np.sum(np.abs(dy), axis=(0, 1))
    _within(_np(dz), dz_ref, e_dz, "group norm dz")
    _within(_np(dg), dg_ref, e_dg, "group norm dgamma")
    _within(_np(db), db_ref, e_db, "group norm dbeta")


@pytest.mark.parametrize("name,T,C,Co,k,s,p", [("stem", 2048, 2, 64, 7, 2, 3), ("stage 1", 512, 64, 64, 5, 1, 2),
                                               ("stage 2 entry", 512, 64, 128, 5, 2, 2),
                                               ("stage 3", 128, 256, 256, 5, 1, 2),
                                               ("stage 3 shortcut", 256, 128, 256, 1, 2, 0)])
def test_convolution_layers_at_training_shape(gwx, name, T, C, Co, k, s, p):
    """One convolution of the network at its training shape (B = 64 windows of 2 x 2048
    samples): im2col rows bit-exact (the stem's from the FP32 strain, rounded), the
    product within 2 K 2^-24 sum |cols| |W| of the oracle, element by element; then the
    backward: dX rows through col2im (FP32, at most k terms per element) and dW."""
    from paper_2407_19048_gb300 import _lib
    lib = _lib.load()
    B = 64
    rng = np.random.default_rng(T + C + Co + k)
    K = rn.stem_k(C) if name == "stem" else k * C
    W = np.zeros((Co, K))
    W[:, :k * C] = _bf(rng, (Co, k * C), np.sqrt(2.0 / (k * C)))
    To = (T + 2 * p - k) // s + 1
    if name == "stem":
        y = rng.normal(size=(B, C, T)).astype(np.float32).astype(np.float64)
        x = round_bf16(np.transpose(y, (0, 2, 1)))
        cols = torch.empty((B * To, K), dtype=torch.bfloat16, device="cuda")
        gwx._check(lib.gwx_im2col_cf(gwx._ptr(_t(y, torch.float32)), B, C, T, k, s, p, K, gwx._ptr(cols),
                                     gwx._stream()))
    else:
        x = _bf(rng, (B, T, C))
        cols = torch.empty((B * To, K), dtype=torch.bfloat16, device="cuda")
        gwx._check(lib.gwx_im2col(gwx._ptr(_t(x, torch.bfloat16)), B, T, C, k, s, p, K, gwx._ptr(cols),
                                  gwx._stream()))
    cref = rn.im2col(x, k, s, p, K).reshape(B * To, K)
    assert np.array_equal(_np(cols), cref), name
    W16 = _t(W, torch.bfloat16)
    z = gwx.dense_bf16(cols, W16, None, act=gwx.ACT_NONE, out_dtype=torch.float32)
    zref = cref @ W.T
    _within(_np(z), zref, 2 * K * U32 * (np.abs(cref) @ np.abs(W.T)), name + " forward")
    dz = rng.normal(size=(B * To, Co)).astype(np.float32).astype(np.float64)
    dcols, dW, _ = gwx.dense_bf16_backward(cols, W16, None, _t(dz, torch.float32), act=gwx.ACT_NONE)
    dzp = round_bf16(dz)
    _within(_np(dW), dzp.T @ cref, 2 * B * To * U32 * (np.abs(dzp).T @ np.abs(cref)), name + " dW")
    if name == "stem":
        return
    dcref = dzp @ W
    _within(_np(dcols), dcref, 2 * Co * U32 * (np.abs(dzp) @ np.abs(W)), name + " dcols")
    dx = torch.empty((B, T, C), dtype=torch.float32, device="cuda")
    gwx._check(lib.gwx_col2im(gwx._ptr(dcols), B, T, C, k, s, p, K, None, gwx._ptr(dx), gwx._stream()))
    # col2im of the GPU's own dcols: the sum of at most k of its terms, FP32
    dcg = _np(dcols).reshape(B, To, K)
    _within(_np(dx), rn.col2im(dcg, T, C, k, s, p), k * U32 * rn.col2im(np.abs(dcg), T, C, k, s, p) + 1e-38,
            name + " col2im")


def test_weight_gradient_over_a_512_window_batch(gwx):
    """The first stage's weight gradient at the training batch of 512 windows: dW = dZ^T
    cols over B T = 262,144 rows (the split-K path: FP32 slice products summed in order),
    every element within 2 (B T) 2^-24 sum |dZ| |cols| of the oracle; dX on sampled rows."""
    M, N, K = 512 * 512, 64, 320
    rng = np.random.default_rng(262144)
    X = _bf(rng, (M, K))
    W = _bf(rng, (N, K), np.sqrt(2.0 / K))
    dY = rng.normal(size=(M, N)).astype(np.float32).astype(np.float64)
    dX, dW, _ = gwx.dense_bf16_backward(_t(X, torch.bfloat16), _t(W, torch.bfloat16), None, _t(dY, torch.float32),
                                        act=gwx.ACT_NONE)
    dzp = round_bf16(dY)
    _within(_np(dW), dzp.T @ X, 2 * M * U32 * (np.abs(dzp).T @ np.abs(X)), "dW over 262,144 rows")
    rows = np.unique(np.concatenate([[0, 1, M - 1], rng.integers(0, M, 200)]))
    _within(_np(dX[torch.from_numpy(rows).cuda()]), dzp[rows] @ W, 2 * N * U32 * (np.abs(dzp[rows]) @ np.abs(W)),
            "dX rows")


def test_pooling_and_mean_at_training_shape(gwx):
    """Max pooling of the stem's output (B = 64, 1024 steps, 64 channels) bit-exact with
    its argument; its backward and the mean over time (and back) of the last stage's
    output (128 steps, 256 channels): FP32 sums within their bounds, the bfloat16 mean
    exact unless its pre-rounding value sits within that bound of a rounding boundary."""
    from paper_2407_19048_gb300 import _lib
    lib = _lib.load()
    B, T, C = 64, 1024, 64
    rng = np.random.default_rng(1024)
    a0 = np.maximum(_bf(rng, (B, T, C)), 0.0)
    To = (T + 2 - 3) // 2 + 1
    h = torch.empty((B, To, C), dtype=torch.bfloat16, device="cuda")
    arg = torch.empty((B, To, C), dtype=torch.uint8, device="cuda")
    gwx._check(lib.gwx_maxpool(gwx._ptr(_t(a0, torch.bfloat16)), B, T, C, gwx._ptr(h), gwx._ptr(arg), gwx._stream()))
    href, aref = rn.maxpool(a0)
    assert np.array_equal(_np(h), href)
    assert np.array_equal(arg.cpu().numpy().astype(np.int64), aref)
    dh = rng.normal(size=(B, To, C)).astype(np.float32).astype(np.float64)
    da = torch.empty((B, T, C), dtype=torch.float32, device="cuda")
    gwx._check(lib.gwx_maxpool_backward(gwx._ptr(_t(dh, torch.float32)), gwx._ptr(arg), B, T, C, gwx._ptr(da),
                                        gwx._stream()))
    _within(_np(da), rn.maxpool_back(dh, aref, T), 2 * U32 * rn.maxpool_back(np.abs(dh), aref, T) + 1e-38,
            "max pool backward")
    B, T, C = 64, 128, 256
    hT = _bf(rng, (B, T, C))
    m = torch.empty((B, C), dtype=torch.bfloat16, device="cuda")
    gwx._check(lib.gwx_mean_time(gwx._ptr(_t(hT, torch.bfloat16)), B, T, C, gwx._ptr(m), gwx._stream()))
    mv = hT.mean(axis=1)
    _within(_np(m), round_bf16(mv), _rnd_bound(mv, 2 * T * U32 * np.abs(hT).mean(axis=1)), "mean over time")
    dm = rng.normal(size=(B, C)).astype(np.float32).astype(np.float64)
    dht = torch.empty((B, T, C), dtype=torch.float32, device="cuda")
    gwx._check(lib.gwx_mean_time_backward(gwx._ptr(_t(dm, torch.float32)), B, T, C, gwx._ptr(dht), gwx._stream()))
    ref = np.repeat(dm[:, None, :], T, axis=1) / T
    _within(_np(dht), ref, 2 * U32 * np.abs(ref), "mean over time backward")

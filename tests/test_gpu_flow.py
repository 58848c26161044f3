"""Parity of the conditional coupling flow (csrc/k_flow.cu, the orchestrated training
step, density and posterior sampler) with oracle.flow (needs a GPU).

Tolerances.  Stage kernels: FP32 arithmetic on the same FP32 inputs (1e-5 relative;
the conditioner input rows are bfloat16 roundings of FP32 values, bit-exact; the
proposal map works in FP64 from the same FP32 draws, 1e-9).  Whole-flow results
(densities, draws, the loss and every element of every gradient tensor) are compared
element by element against bounds propagated through the oracle's own chain from the
FP32 rounding model (tests/rounding_bounds.py): the oracle rounds to bfloat16 at the
same points as the GPU but accumulates in FP64, and each rounding either absorbs the
accumulated difference (no rounding boundary within it: the two sides agree exactly)
or carries it plus one bfloat16 ulp, so an element fails only if it differs by more
than its own propagated bound.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import flow as fl
from oracle import learn

import rounding_bounds as rb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bf16_bits(t):
    return host(t.view(torch.int16)).view(np.uint16)


WL = workloads.workload("small")
GROUP = 16


def _std():
    th = workloads.random_theta(300, 5000, WL["prior"])
    r = fl.coords(th)
    return [float(v) for v in r.mean(axis=0)], [float(v) for v in r.std(axis=0)]


MEAN, SCALE = _std()


def _make_model(hidden, layers=4):
    from paper_2407_19048_gb300.flow import FlowPosterior
    fp = FlowPosterior(WL, layers=layers, hidden=hidden, context=32, embed_hidden=64, group=GROUP, seed=1)
    assert fp.shape["extra"] == 3          # cross spectra and lag-one products
    shape = workloads.flow_shape(features=fp.shape["features"], group=GROUP, embed_hidden=64, context=32,
                                 layers=layers, hidden=hidden)
    params = workloads.random_flow_params(301, shape, gain=1.0, last_gain=0.5)
    fp.set_tensors(params)
    fp.mean, fp.scale = list(MEAN), list(SCALE)
    return fp, params


@pytest.fixture(scope="module")
def model(gwx):
    return _make_model(64)


# hidden width 128 or 256 takes the fused sampling kernel (k_flow_fused.cu); 64 the
# per-layer path
@pytest.fixture(scope="module", params=[64, 128, 256])
def sampler(gwx, request):
    return _make_model(request.param, layers=5)


def oracle_features(y, F, cross=True, lag=True, rounded=True):
    """bfloat16-rounded (or, with rounded False, the unrounded FP64) features of windows y
    from the oracle's FP64 spectrum: log group powers, then the cross-spectral columns,
    then the lag-one columns."""
    y = np.asarray(y, dtype=np.float64)
    k_lo = int(math.ceil(WL["f_lo"] * WL["N"] / WL["fs"] - 1e-9))
    f = learn.features(y, k_lo, GROUP, F)
    D, ng = y.shape[1], (WL["N"] // 2 - k_lo) // GROUP
    col = D * ng
    for on, fn in ((cross, learn.cross_features), (lag, learn.lag_features)):
        if on:
            c = fn(y, k_lo, GROUP)
            f[:, col:col + c.shape[1]] = c
            col += c.shape[1]
    return fl.round_bf16(f) if rounded else f


# ---------------------------------------------------------------- stage kernels

def test_layout(gwx, model):
    fp, params = model
    n, off = gwx.flow_layout(fp.shape)
    assert all(o % 64 == 0 for o in off)
    sizes = [int(np.prod(p.shape)) for p in params]
    for t in range(len(off) - 1):
        assert off[t] + sizes[t] <= off[t + 1]
    assert off[-1] + sizes[-1] <= n


def test_targets(gwx):
    th = workloads.random_theta(302, 500, WL["prior"])
    got = host(gwx.flow_targets(cuda(th), MEAN, SCALE)).astype(np.float64)
    ref = fl.standardise(fl.coords(th), MEAN, SCALE)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("with_events", [False, True])
def test_conditioner_input_bit_exact(gwx, with_events):
    rng = np.random.default_rng(303)
    B, C = 37, 32
    v = rng.normal(0, 2, (B, 8)).astype(np.float32)
    if with_events:
        E = 5
        ctx_bits = workloads.random_bf16_bits(304, (E, C))
        offsets = np.array([0, 3, 3, 20, 30, B], dtype=np.int64)
    else:
        ctx_bits = workloads.random_bf16_bits(304, (B, C))
        offsets = None
    from oracle.gemm import bf16_to_f64, f64_to_bf16
    c_rows = bf16_to_f64(ctx_bits)
    if with_events:
        c_rows = c_rows[fl.event_of(offsets, B)]
    ctx = cuda(ctx_bits.view(np.int16)).view(torch.bfloat16)
    for l in range(4):
        X = gwx.flow_conditioner_input(l, cuda(v), ctx, None if offsets is None else cuda(offsets))
        ref = f64_to_bf16(fl.conditioner_input(v.astype(np.float64), c_rows, l, fl.round_bf16))
        assert np.array_equal(bf16_bits(X), ref)


def test_coupling_both_directions(gwx):
    rng = np.random.default_rng(305)
    B = 1000
    v = rng.normal(0, 1.5, (B, 8)).astype(np.float32)
    o = rng.normal(0, 2.0, (B, 8)).astype(np.float32)
    for l in range(4):
        for direction in (+1, -1):
            sum_s = cuda(np.full(B, 0.25, dtype=np.float32))
            out = gwx.flow_coupling(l, direction, cuda(v), cuda(o), sum_s, init=False)
            w_ref, ss_ref = fl.coupling(v.astype(np.float64), o.astype(np.float64), l, direction)
            np.testing.assert_allclose(host(out), w_ref, rtol=2e-6, atol=2e-6)
            np.testing.assert_allclose(host(sum_s), ss_ref + 0.25, rtol=1e-5, atol=1e-5)
    # in place, init
    vv = cuda(v)
    sum_s = cuda(np.zeros(B, dtype=np.float32))
    gwx.flow_coupling(2, -1, vv, cuda(o), sum_s, init=True, v_out=vv)
    w_ref, ss_ref = fl.coupling(v.astype(np.float64), o.astype(np.float64), 2, -1)
    np.testing.assert_allclose(host(vv), w_ref, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(host(sum_s), ss_ref, rtol=1e-5, atol=1e-5)


def test_nll_and_backward_stages(gwx):
    rng = np.random.default_rng(306)
    B, C = 200, 16
    z = rng.normal(0, 1, (B, 8)).astype(np.float32)
    ss = rng.normal(0, 1, B).astype(np.float32)
    rows, mean, grad = gwx.flow_nll(cuda(z), cuda(ss))
    r_ref, m_ref = fl.nll(z.astype(np.float64), ss.astype(np.float64))
    np.testing.assert_allclose(host(rows), r_ref, rtol=1e-5, atol=1e-5)
    assert abs(host(mean)[0] - m_ref) <= 1e-6 * abs(m_ref) + 1e-6
    np.testing.assert_allclose(host(grad), z / B, rtol=1e-6, atol=1e-9)
    w = rng.normal(0, 1, (B, 8)).astype(np.float32)
    o = rng.normal(0, 2, (B, 8)).astype(np.float32)
    g = rng.normal(0, 1, (B, 8)).astype(np.float32)
    dX = rng.normal(0, 1, (B, 8 + C)).astype(np.float32)
    for l in range(4):
        d_o, g_u = gwx.flow_coupling_backward(l, cuda(w), cuda(o), cuda(g), 1.0 / B)
        do_ref, gu_ref = fl.coupling_backward(l, w.astype(np.float64), o.astype(np.float64), g.astype(np.float64),
                                              np.float32(1.0 / B).astype(np.float64))
        np.testing.assert_allclose(host(d_o), do_ref, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(host(g_u), gu_ref, rtol=1e-5, atol=1e-6)
        dc0 = rng.normal(0, 1, (B, C)).astype(np.float32)
        gu_t, dc_t = cuda(host(g_u).copy()), cuda(dc0)
        gwx.flow_input_backward(l, cuda(dX), gu_t, dc_t, init=(l == 0))
        gu2, dc2 = fl.input_backward(l, dX.astype(np.float64), host(g_u).astype(np.float64),
                                     np.zeros((B, C)) if l == 0 else dc0.astype(np.float64))
        np.testing.assert_allclose(host(gu_t), gu2, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(host(dc_t), dc2, rtol=1e-6, atol=1e-6)


def test_base_normals(gwx):
    z = host(gwx.flow_base(77, 5, 1000, 3000)).astype(np.float64)
    ref, _ = fl.base_normals(77, 5, np.arange(1000, 4000))
    np.testing.assert_allclose(z, ref, rtol=1e-6, atol=1e-6)


def test_proposal_stage(gwx):
    rng = np.random.default_rng(307)
    S = 600
    x = rng.normal(0, 1.2, (S, 8)).astype(np.float32)
    z = rng.normal(0, 1, (S, 8)).astype(np.float32)
    ss = rng.normal(0, 1, S).astype(np.float32)
    th, lq, lr = gwx.flow_proposal(cuda(x), cuda(z), cuda(ss), MEAN, SCALE, WL["prior"], 91, 3)
    _, coin = fl.base_normals(91, 3, np.arange(S))
    th_ref, lq_ref, lr_ref = fl.proposal_params(x.astype(np.float64), z.astype(np.float64), ss.astype(np.float64),
                                                MEAN, SCALE, WL["prior"], coin, fl.nuisance_uniforms(91, 3, np.arange(S)))
    th, lq, lr = host(th), host(lq), host(lr)
    assert np.array_equal(np.isfinite(lr), np.isfinite(lr_ref))
    assert 50 < np.isfinite(lr).sum() < S          # both branches exercised
    np.testing.assert_allclose(th, th_ref, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(lq, lq_ref, rtol=1e-9, atol=1e-9)
    ok = np.isfinite(lr)
    np.testing.assert_allclose(lr[ok], lr_ref[ok], rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------- whole flow

def _batch(seed, B):
    y = workloads.random_strain(seed, (B, len(WL["dets"]), WL["N"]), 1.0).astype(np.float32)
    th = workloads.random_theta(seed + 1, B, WL["prior"])
    return y, th


def test_log_prob(gwx, model):
    fp, params = model
    y, th = _batch(310, 48)
    got = host(fp.log_prob(cuda(y), cuda(th)))
    feat = oracle_features(y, fp.shape["features"])
    ref = fl.log_prob(feat, th, params, 4, MEAN, SCALE)
    x = fl.standardise(fl.coords(th), MEAN, SCALE)
    v, bound = rb.log_prob(oracle_features(y, fp.shape["features"], rounded=False), x, params, 4,
                           np.sum(np.log(SCALE)))
    assert np.allclose(v, ref, rtol=1e-12, atol=1e-12)        # the bound's chain reproduces the oracle
    _within(got, ref, bound, "ln q")


def _within(got, ref, bound, what):
    """Every element within its propagated bound (plus FP64 noise of the oracle)."""
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    tol = bound + 1e-12 * np.abs(ref) + 1e-30
    bad = err > tol
    assert not bad.any(), (what, int(bad.sum()), float(err[bad].max()), float(tol[bad].min()),
                           np.argwhere(bad)[:5].tolist())
    return float(np.max(err / tol))


def _lognormal_bound(z):
    """|d ln N(z)| for base normals held in FP32 (Box-Muller radius in FP64, angle in FP32:
    each within 8 x 2^-24 (|z| + 4))."""
    e = 8.0 * 2.0 ** -24 * (np.abs(z) + 4.0)
    return np.sum(np.abs(z) * e + 0.5 * e * e, axis=1)


def test_train_step_loss_and_gradients(gwx, model):
    """The training step's loss and every element of every gradient tensor against the
    oracle's chain rule, each within its own propagated bound; the bounds themselves are
    a small multiple of the FP32 accumulation error nearly everywhere."""
    fp, params = model
    y, th = _batch(320, 64)
    loss = host(fp.train_step(cuda(y), cuda(th), update=False))[0]
    feat = oracle_features(y, fp.shape["features"])
    x = fl.standardise(fl.coords(th), MEAN, SCALE)
    m_ref, _, g_ref = fl.loss_and_grads(feat, x, params, 4)
    m, mb, gv, gb = rb.loss_and_grads(oracle_features(y, fp.shape["features"], rounded=False), x, params, 4)
    assert abs(m - m_ref) <= 1e-12 * abs(m_ref)
    _within(loss, m_ref, mb, "loss")
    for t in range(len(params)):
        g = host(fp.grads[fp.offsets[t]:fp.offsets[t] + params[t].size]).reshape(params[t].shape)
        np.testing.assert_allclose(gv[t], g_ref[t], rtol=1e-12, atol=1e-14 * np.abs(g_ref[t]).max())
        _within(g, g_ref[t], gb[t], "gradient tensor %d" % t)
        # the bound stays informative: a fraction of the tensor's typical element
        assert np.median(gb[t]) <= 0.25 * np.median(np.abs(g_ref[t])) + 1e-30, (t, np.median(gb[t]))


def test_sample_posterior(gwx, sampler):
    fp, params = sampler
    K = fp.shape["layers"]
    E = 4
    y, _ = _batch(330, E)
    offsets = np.array([0, 150, 150, 400, 700], dtype=np.int64)
    th, lq, lr = fp.sample(cuda(y), cuda(offsets), 2024, 9)
    th, lq, lr = host(th), host(lq), host(lr)
    feat = oracle_features(y, fp.shape["features"])
    th_ref, lq_ref, lr_ref = fl.sample_posterior(feat, params, K, MEAN, SCALE, WL["prior"], offsets, 2024, 9)
    both = np.isfinite(lr) & np.isfinite(lr_ref)
    assert both.sum() >= 0.95 * min(np.isfinite(lr).sum(), np.isfinite(lr_ref).sum())
    assert np.mean(np.isfinite(lr) != np.isfinite(lr_ref)) < 0.01
    S = int(offsets[-1])
    ev = fl.event_of(offsets, S)
    z, _ = fl.base_normals(2024, 9, np.arange(S))
    (xb, ssb), (xe, sse) = rb.draws(oracle_features(y, fp.shape["features"], rounded=False), z, ev, params, K)
    _within(lq, lq_ref, sse + _lognormal_bound(z), "ln q of the draws")
    x = fl.standardise(fl.coords(th[:, both]), MEAN, SCALE)
    x_ref = fl.standardise(fl.coords(th_ref[:, both]), MEAN, SCALE)
    np.testing.assert_allclose(xb[both], x_ref, rtol=1e-9, atol=1e-9)
    _within(x, x_ref, xe[both] + 1e-9 * np.abs(x_ref), "draws")
    for r in (2, 3, 5):                     # spins and t_c from the prior: FP64 on both sides
        np.testing.assert_allclose(th[r], th_ref[r], rtol=0, atol=1e-14 * max(1.0, np.abs(th_ref[r]).max()))


def test_sample_then_density_round_trip(gwx, sampler):
    fp, _ = sampler
    E = 3
    y, _ = _batch(340, E)
    offsets = np.array([0, 300, 600, 900], dtype=np.int64)
    th, lq, lr = fp.sample(cuda(y), cuda(offsets), 5, 1)
    ev = fl.event_of(offsets, 900)
    ok = np.isfinite(host(lr))
    lp = host(fp.log_prob(cuda(y[ev][ok]), th[:, torch.from_numpy(ok).cuda()].contiguous()))
    assert np.all(np.abs(lp - host(lq)[ok]) <= 1e-2 + 1e-3 * np.abs(lp))


def test_sample_posterior_across_chunks(gwx, sampler):
    fp, params = sampler
    K = fp.shape["layers"]
    E = 2
    y, _ = _batch(350, E)
    S = (1 << 17) + 3000
    offsets = np.array([0, 70000, S], dtype=np.int64)
    th, lq, lr = fp.sample(cuda(y), cuda(offsets), 8, 2)
    pick = np.r_[0:5, 69998:70003, (1 << 17) - 3:(1 << 17) + 3, S - 4:S]
    feat = oracle_features(y, fp.shape["features"])
    emb, layers = fl.split_params(params, K)
    c, _ = fl.embed(feat, emb)
    ev = fl.event_of(offsets, S)[pick]
    z, coin = fl.base_normals(8, 2, pick)
    x, ss = fl.sample(z, c[ev], layers)
    _, lq_ref, _ = fl.proposal_params(x, z, ss, MEAN, SCALE, WL["prior"], coin, fl.nuisance_uniforms(8, 2, pick))
    _, (_, sse) = rb.draws(oracle_features(y, fp.shape["features"], rounded=False), z, ev, params, K)
    _within(host(lq)[pick], lq_ref, sse + _lognormal_bound(z), "ln q across chunks")


def test_training_lowers_the_loss(gwx):
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    sim = Simulator(WL)
    fp = FlowPosterior(WL, layers=4, hidden=64, context=32, embed_hidden=64, group=GROUP, seed=3, lr=2e-3)
    first, last = [], []
    for step in range(300):
        y, theta, _ = sim.step(step)
        loss = fp.train_step(y, theta)
        if step < 20:
            first.append(float(host(loss)[0]))
        if step >= 280:
            last.append(float(host(loss)[0]))
    assert np.mean(last) < np.mean(first) - 0.5, (np.mean(first), np.mean(last))


def test_checkpoint_resume_is_bit_exact(gwx, tmp_path):
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    sim = Simulator(WL)
    kw = dict(layers=2, hidden=32, context=16, embed_hidden=32, group=GROUP)
    a = FlowPosterior(WL, seed=4, **kw)
    for step in range(5):
        y, theta, _ = sim.step(step)
        a.train_step(y, theta)
    path = str(tmp_path / "flow.ckpt")
    a.save(path, next_step=5)
    for step in range(5, 10):
        y, theta, _ = sim.step(step)
        a.train_step(y, theta)
    b = FlowPosterior(WL, seed=99, **kw)
    nxt = b.load(path)
    assert nxt == 5
    for step in range(nxt, 10):
        y, theta, _ = sim.step(step)
        b.train_step(y, theta)
    assert torch.equal(a.params, b.params) and torch.equal(a.m, b.m) and b.steps == a.steps


def test_scorer_with_the_flow_matches_the_separate_calls(gwx, sampler):
    from paper_2407_19048_gb300.scorer import Scorer
    from paper_2407_19048_gb300.simulator import Simulator
    fp, _ = sampler
    wl = dict(WL, B=4)
    sim = Simulator(wl)
    y, th, _ = sim.step(7)
    sc = Scorer(wl, 3000, sim.psd, flow=fp)
    for e, S in ((0, 3000), (2, 1234)):
        got = sc.score(y[e:e + 1], S, 11)
        offs = torch.tensor([0, S], dtype=torch.int64, device="cuda")
        theta, _, lr = gwx.sample_posterior(fp.shape, fp.params, fp.params16, fp.mean, fp.scale, wl["prior"],
                                            y[e:e + 1].contiguous(), wl["fs"], wl["f_lo"], offs, 55, 11)
        lnl = gwx.log_likelihood(y[e:e + 1].contiguous(), sim.psd, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"],
                                 0.0, theta, offs)
        _, ess, eff, lnz = gwx.importance_weights(lnl, offs, lr)
        ref = (float(ess[0]), float(eff[0]), float(lnz[0]))
        assert got == ref or np.allclose(got, ref, rtol=1e-12, atol=0), (got, ref)


def test_captured_training_step_replays_like_eager_steps(gwx):
    """A CUDA graph of one training step (AdamW step count on the device) replayed on
    successive batches matches the eager steps on the same batches."""
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    kw = dict(layers=3, hidden=64, context=16, embed_hidden=32, group=GROUP, clip=0.5)
    sim = Simulator(WL)
    a = FlowPosterior(WL, seed=6, **kw)
    b = FlowPosterior(WL, seed=6, **kw)
    y0, th0, _ = sim.step(0)
    yb, thb = y0.clone(), th0.clone()          # the graph's fixed input buffers
    graph = b.capture_train_step(yb, thb)
    for step in range(4):
        y, th, _ = sim.step(step)
        a.train_step(y, th)
        yb.copy_(y)
        thb.copy_(th)
        graph.replay()
        b.note_replay()
    torch.cuda.synchronize()
    assert int(b.step_dev.item()) == 4 and b.steps == 4
    assert torch.allclose(a.params, b.params, rtol=1e-5, atol=1e-7)
    assert torch.allclose(a.m, b.m, rtol=1e-5, atol=1e-9)


def test_captured_resnet_training_step_replays_like_eager_steps(gwx):
    """The same with the ResNet-1D summary inside the graph: its forward, the flow's step
    (which advances the device step counter), its backward and AdamW on every summary
    tensor at that step (gwx_adamw_at).  64-window batches of the two-detector workload;
    the stride-1 convolutions of the 64-channel stage run as implicit GEMMs."""
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    wl = dict(WL, B=64)
    kw = dict(layers=2, hidden=64, context=16, embed_hidden=32, group=GROUP, embedding="resnet",
              resnet_stages=((64, 1, 1), (128, 1, 2)))
    sim = Simulator(wl)
    a = FlowPosterior(wl, seed=7, **kw)
    b = FlowPosterior(wl, seed=7, **kw)
    y0, th0, _ = sim.step(0)
    yb, thb = y0.clone(), th0.clone()
    graph = b.capture_train_step(yb, thb)
    for step in range(4):
        y, th, _ = sim.step(step)
        a.train_step(y, th)
        yb.copy_(y)
        thb.copy_(th)
        graph.replay()
        b.note_replay()
    torch.cuda.synchronize()
    assert int(b.step_dev.item()) == 4 and b.steps == 4
    assert torch.allclose(a.params, b.params, rtol=1e-5, atol=1e-7)
    for (name, pa, _), (_, pb, _) in zip(a.resnet.tensors(), b.resnet.tensors()):
        assert torch.allclose(pa, pb, rtol=1e-5, atol=1e-7), name
        assert torch.allclose(a.rmom[name][0], b.rmom[name][0], rtol=1e-5, atol=1e-9), name
    assert gwx._lib.load().gwx_device_status() == 0


def test_external_context_matches_oracle_and_resnet_summary_trains(gwx, model):
    """The flow with the caller's context (the ResNet-1D path) against the oracle's flow
    with that context, and a short training run of flow + ResNet-1D summary."""
    from oracle.gemm import bf16_to_f64
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    fp, params = model
    B = 32
    y, th = _batch(360, B)
    bits = workloads.random_bf16_bits(361, (B, 32), exp_lo=-3, exp_hi=0)
    ctx = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    got = host(fp.gwx.flow_log_prob(fp.shape, fp.params, fp.params16, MEAN, SCALE, cuda(y), cuda(th), WL["fs"],
                                    WL["f_lo"], ctx=ctx))
    _, layers = fl.split_params(params, 4)
    x = fl.standardise(fl.coords(th), MEAN, SCALE)
    z, ss, _ = fl.density(x, bf16_to_f64(bits), layers)
    ref = fl.log_normal(z) - ss - np.sum(np.log(SCALE))
    v, bound = rb.log_prob(None, x, params, 4, np.sum(np.log(SCALE)), ctx=bf16_to_f64(bits))
    assert np.allclose(v, ref, rtol=1e-12, atol=1e-12)
    _within(got, ref, bound, "ln q with an external context")
    # flow + ResNet-1D summary: the loss falls
    sim = Simulator(dict(WL, B=64))
    net = FlowPosterior(dict(WL, B=64), layers=2, hidden=64, context=32, group=GROUP, seed=8, lr=1e-3,
                        embedding="resnet", resnet_stages=((8, 1, 1), (16, 1, 2), (16, 1, 2)))
    losses = []
    for step in range(120):
        yb, tb, _ = sim.step(step)
        losses.append(float(host(net.train_step(yb, tb))[0]))
    assert np.mean(losses[-15:]) < np.mean(losses[:15]) - 0.3, (np.mean(losses[:15]), np.mean(losses[-15:]))
    offs = torch.tensor([0, 100, 250], dtype=torch.int64, device="cuda")
    theta_s, lq, lr = net.sample(yb[:2].contiguous(), offs, 3, 0)
    ok = torch.isfinite(lr)
    lp = net.log_prob(yb[torch.tensor([0] * 100 + [1] * 150, device="cuda")][ok].contiguous(),
                      theta_s[:, ok].contiguous())
    assert torch.allclose(lp, lq[ok], atol=1e-2, rtol=1e-3)

"""ResNet-1D data summary on the GPU (paper_2407_19048_gb300.resnet) against
oracle.resnet (needs a GPU).  Tolerances: the oracle rounds to bfloat16 at the same
points but sums convolutions and statistics in FP64, so activations next to a rounding
boundary can flip by one bfloat16 ulp and propagate through the residual stack.  The
representation is compared within 2 % of its scale.  A gradient's sensitivity to those
roundings grows with its depth below the output: the oracle itself, run exactly and
with the bfloat16 roundings, differs by up to ~20 % at the stem of the full network
(0.2 % for the small one).  So each gradient must lie within max(5 %, 1.5 x that
measured sensitivity) of the oracle's, in norm; a wrong tap, stride, group or sign moves
a gradient by O(1)."""
import numpy as np
import pytest

from oracle import resnet as rn

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


@pytest.mark.parametrize("stages,N,B", [(SMALL, 256, 8), (rn.STAGES, 512, 8)])
def test_forward_and_backward_match_oracle(gwx, stages, N, B):
    from paper_2407_19048_gb300.resnet import ResNet1D
    rng = np.random.default_rng(N + B)
    D, C = 2, 8
    P = _bf16_exact(rn.init_params(rng, D, C, stages))
    y = rng.normal(size=(B, D, N)).astype(np.float32)
    net = ResNet1D(D, C, stages=stages, params=P)
    c = net.forward(torch.from_numpy(y).cuda()).cpu().numpy()
    c_ref, tape = rn.forward(y.astype(np.float64), P)
    scale = np.abs(c_ref).max()
    assert np.max(np.abs(c - c_ref)) <= 0.02 * scale, (np.max(np.abs(c - c_ref)), scale)
    dc = rng.normal(size=c.shape).astype(np.float32)
    G = net.backward(torch.from_numpy(dc).cuda())
    G_ref = rn.backward(dc.astype(np.float64), P, tape)
    names = {"W0": G_ref["W0"], "g0": G_ref["g0"], "b0": G_ref["b0"], "Wf": G_ref["Wf"], "bf": G_ref["bf"]}
    for i, g in enumerate(G_ref["blocks"]):
        for k, v in g.items():
            names["%d.%s" % (i, k)] = v
    from oracle.flow import exact
    _, tape_ex = rn.forward(y.astype(np.float64), P, exact)
    G_ex = rn.backward(dc.astype(np.float64), P, tape_ex, exact)
    sens = {"W0": G_ex["W0"], "g0": G_ex["g0"], "b0": G_ex["b0"], "Wf": G_ex["Wf"], "bf": G_ex["bf"]}
    for i, g in enumerate(G_ex["blocks"]):
        for k, v in g.items():
            sens["%d.%s" % (i, k)] = v
    for k, ref in names.items():
        got = G[k].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(got - ref)
        tol = max(0.05, 1.5 * np.linalg.norm(sens[k] - ref) / (np.linalg.norm(ref) + 1e-30))
        assert err <= tol * np.linalg.norm(ref) + 1e-6, (k, err / np.linalg.norm(ref), tol)


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


@pytest.mark.parametrize("B,T,C", [(3, 37, 96), (2, 50, 64), (2, 33, 24), (4, 64, 256)])
def test_group_norm_kernels(gwx, B, T, C):
    """gwx_group_norm (residual, ReLU) and gwx_group_norm_backward against oracle.resnet's
    gn / gn_back on values with a mean far from zero.  The shapes take each kernel path:
    C = 96 per group with four-channel loads, C = 64 and 256 per sample, C = 24 (three
    channels per group) one channel at a time.  FP32 arithmetic against FP64: 2e-5 of the
    output scale forward, 1e-4 of each gradient's norm backward."""
    from paper_2407_19048_gb300 import _lib
    lib = _lib.load()
    G = 8
    rng = np.random.default_rng(B * 1000 + T + C)
    z = (3.0 + 2.0 * rng.normal(size=(B, T, C))).astype(np.float32)
    g = (1.0 + 0.1 * rng.normal(size=C)).astype(np.float32)
    b = (0.1 * rng.normal(size=C)).astype(np.float32)
    res = rng.normal(size=(B, T, C)).astype(np.float32)
    dy = rng.normal(size=(B, T, C)).astype(np.float32)
    Z, Gm, Bt, R, DY = (torch.from_numpy(a).cuda() for a in (z, g, b, res, dy))
    out = torch.empty_like(Z)
    ms = torch.empty((B, G, 2), dtype=torch.float32, device="cuda")
    gwx._check(lib.gwx_group_norm(gwx._ptr(Z), B, T, C, G, gwx._ptr(Gm), gwx._ptr(Bt), gwx._ptr(R), None, 1, None,
                                  gwx._ptr(out), gwx._ptr(ms), gwx._stream()))
    y, xh, rstd = rn.gn(z.astype(np.float64), g.astype(np.float64), b.astype(np.float64), G)
    ref = np.maximum(y + res, 0.0)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 2e-5 * np.abs(ref).max()
    dz = torch.empty_like(Z)
    dg = torch.empty(C, dtype=torch.float32, device="cuda")
    db = torch.empty(C, dtype=torch.float32, device="cuda")
    nb = lib.gwx_group_norm_backward_scratch(B, C, G)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    gwx._check(lib.gwx_group_norm_backward(gwx._ptr(DY), gwx._ptr(Z), B, T, C, G, gwx._ptr(ms), gwx._ptr(Gm),
                                           gwx._ptr(scratch), gwx._ptr(dz), gwx._ptr(dg), gwx._ptr(db),
                                           gwx._stream()))
    dz_ref, dg_ref, db_ref = rn.gn_back(dy.astype(np.float64), xh, rstd, g.astype(np.float64), G)
    for got, want in ((dz, dz_ref), (dg, dg_ref), (db, db_ref)):
        err = np.linalg.norm(got.cpu().numpy().astype(np.float64) - want)
        assert err <= 1e-4 * np.linalg.norm(want), (err, np.linalg.norm(want))

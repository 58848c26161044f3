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

"""VICReg pre-training pieces on the GPU against oracle.vicreg (needs a GPU): the loss,
its terms and gradient (FP32 inputs, FP64 sums: 1e-5 relative), the second view's
parameters (bit-exact), rendering given parameters (bit-exact against the batch call),
and a short pre-training run that lowers the loss."""
import numpy as np
import pytest

import workloads
from oracle import vicreg as vr

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


@pytest.mark.parametrize("B,d", [(2, 1), (100, 24), (4096, 24), (300, 32)])
def test_vicreg_matches_oracle(gwx, B, d):
    rng = np.random.default_rng(B + d)
    x = rng.normal(0, 0.8, (B, d)).astype(np.float32)
    xp = (x + rng.normal(0, 0.3, (B, d))).astype(np.float32)
    xp[:, 0] *= 2.5
    loss, terms, gx, gxp = gwx.vicreg(torch.from_numpy(x).cuda(), torch.from_numpy(xp).cuda())
    x64, xp64 = x.astype(np.float64), xp.astype(np.float64)
    np.testing.assert_allclose(terms.cpu().numpy(), vr.terms(x64, xp64), rtol=1e-9, atol=1e-12)
    assert abs(loss.item() - vr.loss(x64, xp64)) <= 1e-9 * abs(vr.loss(x64, xp64)) + 1e-12
    rx, rxp = vr.grad(x64, xp64)
    scale = max(np.abs(rx).max(), np.abs(rxp).max())
    np.testing.assert_allclose(gx.cpu().numpy(), rx, rtol=1e-5, atol=1e-6 * scale)
    np.testing.assert_allclose(gxp.cpu().numpy(), rxp, rtol=1e-5, atol=1e-6 * scale)


def test_retime_matches_oracle(gwx):
    prior = workloads.workload("small")["prior"]
    th = workloads.random_theta(500, 777, prior)
    got = gwx.retime(torch.from_numpy(th).cuda(), prior["tc_lo"], prior["tc_hi"], 31, 4).cpu().numpy()
    ref = vr.retime(th, prior["tc_lo"], prior["tc_hi"], 31, 4)
    assert np.array_equal(got, ref)
    assert np.array_equal(np.delete(got, 5, axis=0), np.delete(th, 5, axis=0))
    assert np.all((got[5] >= prior["tc_lo"]) & (got[5] <= prior["tc_hi"]))


def test_rendering_given_parameters_equals_the_batch_call(gwx):
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.pretrain import VICRegPretrainer
    wl = workloads.workload("small", B=64)
    fp = FlowPosterior(wl, layers=2, hidden=64, context=32, embed_hidden=64, group=16)
    pt = VICRegPretrainer(fp, batch=64)
    pt._background(0)
    y, th, off = gwx.simulate_batch(wl["prior"], pt.seed, 3, pt.noise, pt.psd, wl["seg_len"], wl["fs"], wl["f_lo"],
                                    wl["dets"], 0.0, 64, wl["N"])
    out = torch.empty_like(y)
    pt._render(th, off, out)
    assert torch.equal(out, y)


def test_pretraining_lowers_the_loss_and_pulls_views_together(gwx):
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.pretrain import VICRegPretrainer
    wl = workloads.workload("small", B=512)
    fp = FlowPosterior(wl, layers=2, hidden=64, context=32, embed_hidden=128, group=16)
    pt = VICRegPretrainer(fp, batch=512, lr=1e-3)
    first, last = [], []
    for k in range(120):
        loss, _ = pt.step(k)
        if k < 10:
            first.append(loss.item())
        if k >= 110:
            last.append(loss.item())
    assert np.mean(last) < 0.8 * np.mean(first), (np.mean(first), np.mean(last))


def test_pretraining_the_resnet_summary_on_raw_strain_lowers_the_loss(gwx):
    """VICReg on the ResNet-1D over the raw whitened strain (the paper's case): both views
    run through the ResNet, the expander and the loss; the gradient flows back through the
    ResNet's implicit-GEMM convolutions and group norms and AdamW updates its tensors in
    place.  A two-stage ResNet on one fixed batch of 256 view pairs (every call renders the
    views of step 0): the first update lowers the loss, 25 of them lower it by more than 7 %
    (measured: 1.95 -> 1.73; the hinged variance terms keep it well above zero this early),
    and every ResNet tensor moves."""
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.pretrain import VICRegPretrainer
    wl = workloads.workload("small", B=256)
    fp = FlowPosterior(wl, layers=2, hidden=64, context=32, embedding="resnet",
                       resnet_stages=((64, 1, 1), (128, 1, 2)))
    before = {name: p.clone() for name, p, _ in fp.resnet.tensors()}
    pt = VICRegPretrainer(fp, batch=256, lr=1e-3)
    losses = []
    for _ in range(25):
        loss, terms = pt.step(0)
        assert torch.isfinite(loss).all() and torch.isfinite(terms).all()
        losses.append(loss.item())
    assert losses[1] < losses[0], losses[:3]
    assert losses[-1] < 0.93 * losses[0], (losses[0], losses[-1])
    moved = [name for name, p, _ in fp.resnet.tensors() if not torch.equal(p, before[name])]
    assert len(moved) == len(before)
    assert gwx._lib.load().gwx_device_status() == 0

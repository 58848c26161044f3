"""Parity of the learned-proposal kernels with oracle.learn (needs a GPU).

Tolerances: features are bfloat16 (2^-8 relative) of an FP32 spectrum; targets FP32
(1e-6 relative); the Gaussian loss and its gradient FP32 (1e-5 relative); AdamW FP32
(1e-5 relative after three steps); proposal draws FP64 from identical Philox integers
(1e-12 relative; -inf log ratios at the same samples).
"""
import numpy as np
import pytest

import workloads
from oracle import learn

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


MEAN, SCALE = [22.0, 60.0, 1100.0], [6.0, 16.0, 520.0]


def test_spectral_features(gwx):
    wl = workloads.workload("small")
    y = workloads.random_strain(200, (16, 2, wl["N"]), 1.0).astype(np.float32)
    k_lo = int(np.ceil(wl["f_lo"] * wl["N"] / wl["fs"]))
    got = host(gwx.spectral_features(cuda(y), wl["fs"], wl["f_lo"], 4, 512).float()).astype(np.float64)
    ref = learn.features(y.astype(np.float64), k_lo, 4, 512)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-4)


def test_cross_and_lag_features(gwx):
    wl = workloads.workload("hl3")
    y = workloads.random_strain(206, (8, 3, wl["N"]), 1.0)
    # a common chirp-like tone in all three detectors with different delays and gains
    n = np.arange(wl["N"])
    tone = np.cos(2 * np.pi * (60.0 + 20.0 * n / wl["N"]) * n / wl["fs"])
    for d, (lag, gain) in enumerate(((0, 3.0), (9, 2.0), (-14, 1.5))):
        y[:, d] += gain * np.roll(tone, lag)[None]
    y = y.astype(np.float32)
    k_lo = int(np.ceil(wl["f_lo"] * wl["N"] / wl["fs"]))
    G = 8
    ng = (wl["N"] // 2 - k_lo) // G
    F = ((3 * ng + 6 * ng + 6 * ng + 7) // 8) * 8
    out = gwx.spectral_features(cuda(y), wl["fs"], wl["f_lo"], G, F)
    gwx.cross_features(cuda(y), wl["fs"], wl["f_lo"], G, F, 3 * ng, out)
    gwx.lag_features(cuda(y), wl["fs"], wl["f_lo"], G, F, 9 * ng, out)
    got = host(out.float()).astype(np.float64)
    ref = np.zeros_like(got)
    ref[:, :3 * ng] = learn.features(y.astype(np.float64), k_lo, G, F)[:, :3 * ng]
    ref[:, 3 * ng:9 * ng] = learn.cross_features(y.astype(np.float64), k_lo, G)
    ref[:, 9 * ng:15 * ng] = learn.lag_features(y.astype(np.float64), k_lo, G)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-4)
    assert np.all(got[:, 15 * ng:] == 0.0)


def test_adamw_clip(gwx):
    rng = np.random.default_rng(207)
    n = 100003
    p = rng.normal(0, 1, n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    pt, mt, vt = cuda(p), cuda(m), cuda(v)
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step, gain in ((1, 3.0), (2, 0.01), (3, 5.0)):          # clipped, not clipped, clipped
        g = (rng.normal(0, 1, n) * gain / np.sqrt(n)).astype(np.float32)
        gwx.adamw_clip(pt, cuda(g), mt, vt, step, 1e-3, 0.5, weight_decay=1e-2)
        pr, mr, vr = learn.adamw(pr, g.astype(np.float64), mr, vr, 1e-3, 0.9, 0.999, 1e-8, 1e-2, step, clip=0.5)
    np.testing.assert_allclose(host(pt), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(host(mt), mr, rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(host(vt), vr, rtol=1e-4, atol=1e-12)


def test_targets_and_gauss_nll(gwx):
    wl = workloads.workload("small")
    th = workloads.random_theta(201, 300, wl["prior"])
    t = host(gwx.proposal_targets(cuda(th), MEAN, SCALE)).astype(np.float64)
    t_ref = learn.targets(th, MEAN, SCALE)
    np.testing.assert_allclose(t, t_ref, rtol=1e-6, atol=1e-6)
    out = np.random.default_rng(202).normal(0.0, 0.7, (300, 8)).astype(np.float32)
    loss, mean, grad = gwx.gauss_nll(cuda(out), cuda(t.astype(np.float32)))
    l_ref, m_ref, g_ref = learn.gauss_nll(out.astype(np.float64), t.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(host(loss), l_ref, rtol=1e-5, atol=1e-5)
    assert abs(host(mean)[0] - m_ref) <= 1e-5 * abs(m_ref) + 1e-6
    np.testing.assert_allclose(host(grad), g_ref, rtol=1e-5, atol=1e-8)


def test_adamw_three_steps(gwx):
    rng = np.random.default_rng(203)
    n = 1000
    p = rng.normal(0.0, 1.0, n).astype(np.float32)
    P, M, V = cuda(p.copy()), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    P16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    pr, mr, vr = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.normal(0.0, 0.1, n).astype(np.float32)
        gwx.adamw(P, cuda(g), M, V, step, lr=1e-2, weight_decay=0.01, param_bf16=P16)
        pr, mr, vr = learn.adamw(pr, g.astype(np.float64), mr, vr, 1e-2, 0.9, 0.999, 1e-8, 0.01, step)
    np.testing.assert_allclose(host(P), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(host(P16.float()), pr, rtol=2.0 ** -8, atol=1e-6)


@pytest.mark.parametrize("learned,fix", [(False, False), (True, False), (True, True)])
def test_sample_proposal(gwx, learned, fix):
    wl = workloads.workload("small")
    prior = wl["prior"]
    E = 7
    truth = workloads.random_theta(204, E, prior)
    counts = workloads.ragged_counts(205, E, 50, 400, zeros=1)
    offs = np.concatenate([[0], np.cumsum(counts)])
    net = np.random.default_rng(206).normal(0.0, 0.4, (E, 8)).astype(np.float32) if learned else None
    if learned:
        net[:, 3:6] -= 1.0
    th, lr = gwx.sample_proposal(prior, cuda(truth), cuda(offs), seed=11, counter=5,
                                 net_out=cuda(net) if learned else None, mean=MEAN, scale=SCALE, fix_angles=fix)
    th_ref, lr_ref = learn.sample_proposal(net, MEAN, SCALE, prior, truth, offs, seed=11, counter=5, fix_angles=fix)
    np.testing.assert_allclose(host(th), th_ref, rtol=1e-12, atol=1e-12)
    got = host(lr)
    fin = np.isfinite(lr_ref)
    np.testing.assert_array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], lr_ref[fin], rtol=0, atol=1e-9)
    if learned:
        assert fin.sum() > 0.3 * len(fin)


def test_training_lowers_the_loss(gwx):
    """300 AdamW steps of the learned proposal on simulated batches (512 draws of the
    two-detector workload) lower the batch Gaussian loss from its start."""
    import paper_2407_19048_gb300.simulator as S
    from paper_2407_19048_gb300.proposal import LearnedProposal
    wl = workloads.workload("small", B=512)
    sim = S.Simulator(wl, pipeline=True, background_every=16)
    net = LearnedProposal(wl, hidden=256)
    first, last = [], []
    for i in range(300):
        y, th, _ = sim.step(i)
        loss = net.train_step(y, th)
        if i < 10:
            first.append(float(loss.item()))
        if i >= 290:
            last.append(float(loss.item()))
    gwx.device_status()
    assert np.mean(last) < np.mean(first) - 0.5, (np.mean(first), np.mean(last))


def test_checkpoint_resume_is_bit_exact(gwx, tmp_path):
    """Training resumed from a checkpoint (weights, AdamW moments, step count, data-stream
    counter) follows the uninterrupted run bit for bit: the batches come from Philox
    counters, so the data stream resumes exactly too."""
    import paper_2407_19048_gb300.simulator as S
    from paper_2407_19048_gb300.proposal import LearnedProposal
    wl = workloads.workload("small", B=128)

    def run(net, sim, first, n):
        for i in range(first, first + n):
            y, th, _ = sim.step(i)
            net.train_step(y, th)

    a = LearnedProposal(wl, hidden=128, seed=3)
    sim_a = S.Simulator(wl)
    run(a, sim_a, 0, 15)
    path = str(tmp_path / "prop.ckpt")
    a.save(path, next_step=15)
    run(a, sim_a, 15, 10)
    b = LearnedProposal(wl, hidden=128, seed=99)      # different initial weights
    nxt = b.load(path)
    assert nxt == 15 and b.steps == 15
    run(b, S.Simulator(wl), nxt, 10)
    torch.cuda.synchronize()
    for i in range(3):
        np.testing.assert_array_equal(host(a.W[i]), host(b.W[i]))
        np.testing.assert_array_equal(host(a.vb[i]), host(b.vb[i]))

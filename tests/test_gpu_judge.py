"""The likelihood judge of the learned part (needs a GPU): a flow trained on the
non-spinning two-detector generator must beat the prior as an importance-sampling
proposal, with every draw scored by the likelihood that integrates the merger time out
(neither proposal is given anything about the event but its whitened strain)."""
import numpy as np
import pytest

import workloads

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


def test_trained_flow_beats_the_prior_on_eight_events(gwx):
    from paper_2407_19048_gb300.flow import FlowPosterior
    from paper_2407_19048_gb300.simulator import Simulator
    wl = workloads.workload("small_nonspinning", B=4096)
    sim = Simulator(wl, pipeline=True, background_every=16)
    fp = FlowPosterior(wl, layers=16, hidden=256, context=64, embed_hidden=512, group=4, seed=0, lr=1e-3,
                       weight_decay=2e-3, clip=1.0)
    sv = Simulator(dict(wl, B=8192, param_seed=911))
    yv, thv, _ = sv.step(7)
    hist = fp.fit(sim, 2000, 40000, (yv.clone(), thv.clone()))
    assert hist["best_val_loss"] < hist["epochs"][0][1] - 1.0       # it learned something
    E, S = 8, 20000
    wl_ev = dict(workloads.workload("small_nonspinning", B=E), param_seed=4321)
    se = Simulator(wl_ev)
    y, _, _ = se.step(3)
    offs = torch.arange(E + 1, dtype=torch.int64, device="cuda") * S
    tc_lo, n_tc, u = workloads.tc_grid(wl_ev)
    eff = {}
    for arm in ("prior", "flow"):
        if arm == "flow":
            theta, _, lrat = fp.sample(y, offs, 9, 0, S=E * S)
        else:
            theta, _ = gwx.sample_prior(wl_ev["prior"], 9, 0, E * S, wl_ev["L"], wl_ev["N"])
            lrat = None
        lnl = gwx.log_likelihood_tmarg(y, se.psd, wl_ev["seg_len"], wl_ev["fs"], wl_ev["f_lo"], wl_ev["dets"], 0.0,
                                       tc_lo, n_tc, u, theta, offs)
        _, ess, e, _ = gwx.importance_weights(lnl, offs, lrat)
        eff[arm] = e.cpu().numpy()
        assert np.all(np.isfinite(eff[arm])) and np.all(ess.cpu().numpy() >= 1.0 - 1e-9)
    assert np.median(eff["flow"]) > np.median(eff["prior"]), (eff["flow"], eff["prior"])

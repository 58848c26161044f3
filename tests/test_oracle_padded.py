"""Pins of Definition B (the padded-grid waveform, oracle.pipeline.simulate_batch_padded):
it is Definition A when the padded segment is the window itself, and the injected window
stops changing once the padded segment holds the whole inspiral, while Definition A
carries the wrapped early inspiral."""
import numpy as np

import workloads
from oracle import pipeline


def _wl():
    return workloads.workload("small", B=6)


def test_no_padding_is_definition_a():
    wl = _wl()
    bg = pipeline.background(wl, 0)
    a = pipeline.simulate_batch(wl, 0, bg=bg)
    b = pipeline.simulate_batch_padded(wl, 0, wl["N"], bg=bg)
    np.testing.assert_allclose(b["y"], a["y"], rtol=0, atol=1e-12 * np.abs(a["y"]).max())




def test_padding_converges_and_removes_the_wrap():
    wl = _wl()
    bg = pipeline.background(wl, 0)
    zero = (np.zeros_like(bg[0]), bg[1])
    from oracle.prior import sample_prior
    th, _ = sample_prior(wl["prior"], wl["param_seed"], 0, wl["B"], wl["L"], wl["N"])
    m_tot = th[0] + th[1]
    light = int(np.argmin(m_tot))                 # the longest signal of the batch
    assert m_tot[light] < 50.0                    # tau(20 Hz) well above the 2 s window
    ys = {n: pipeline.simulate_batch_padded(wl, 0, n, draws=[light], bg=zero)["y"][0]
          for n in (wl["N"], 4 * wl["N"], 8 * wl["N"], 16 * wl["N"])}
    norm = np.linalg.norm(ys[16 * wl["N"]])
    assert norm > 0
    # 8N and 16N (16 s and 32 s) both hold the whole inspiral: the window agrees
    assert np.linalg.norm(ys[8 * wl["N"]] - ys[16 * wl["N"]]) < 0.02 * norm
    # Definition A (no padding) differs: the early inspiral wraps into the window
    assert np.linalg.norm(ys[wl["N"]] - ys[16 * wl["N"]]) > 0.1 * norm

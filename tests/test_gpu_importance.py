"""Parity of gwx_importance_weights with oracle.importance (needs a GPU).

Tolerances: exp is evaluated in FP32 on an exactly split FP64 argument, so weights,
effective sample sizes and efficiencies agree to a relative 2e-6 and ln Z to 2e-6
absolute; weights the FP32 exponential flushes to zero (below ~1e-44 of the largest)
are compared with an absolute 1e-30.  Chained after the likelihood, where each ln L
may differ from the oracle's by up to 1e-3, weights agree to a relative 5e-3.
"""
import numpy as np
import pytest

import workloads
from oracle import importance, likelihood

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


def _compare(got, ref, rtol=2e-6, z_atol=2e-6):
    w, ess, eff, lnz = (host(t) for t in got)
    rw, ress, reff, rlnz = ref
    np.testing.assert_allclose(w, rw, rtol=rtol, atol=1e-30)
    np.testing.assert_allclose(ess, ress, rtol=rtol, atol=0)
    np.testing.assert_allclose(eff, reff, rtol=rtol, atol=0)
    fin = np.isfinite(rlnz)
    np.testing.assert_array_equal(np.isfinite(lnz), fin)
    np.testing.assert_allclose(lnz[fin], rlnz[fin], rtol=0, atol=z_atol)


@pytest.mark.parametrize("with_ratio", [False, True])
def test_importance_weights_ragged_edge_cases(gwx, with_ratio):
    rng = np.random.default_rng(50 + with_ratio)
    counts = workloads.ragged_counts(51, 40, 1, 3000, zeros=4)
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    lnl = rng.normal(-2.0e4, 30.0, S)
    nz = np.flatnonzero(counts)
    lnl[offs[nz[0]]:offs[nz[0] + 1]] = -np.inf                   # an event with no support
    lnl[offs[nz[1]]] = -np.inf                                   # a single impossible sample
    lnl[offs[nz[2]]] += 500.0                                    # one sample dominates its event
    lnl[offs[nz[3]]:offs[nz[3] + 1]] = -7.5                      # flat: uniform weights
    ratio = rng.normal(0.0, 2.0, S) if with_ratio else None
    got = gwx.importance_weights(cuda(lnl), cuda(offs), None if ratio is None else cuda(ratio))
    _compare(got, importance.importance_weights(lnl, offs, ratio))


def test_importance_weights_full_scale(gwx):
    """64 events with U{2000..50000} samples (~1.7 million), every output compared."""
    counts = workloads.ragged_counts(52, 64, 2000, 50000)
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    rng = np.random.default_rng(53)
    lnl = rng.normal(-5.0e4, 60.0, S)
    ratio = rng.normal(0.0, 3.0, S)
    got = gwx.importance_weights(cuda(lnl), cuda(offs), cuda(ratio))
    _compare(got, importance.importance_weights(lnl, offs, ratio))


def test_importance_weights_empty_and_errors(gwx):
    w, ess, eff, lnz = gwx.importance_weights(cuda(np.zeros(0)), cuda(np.array([0, 0, 0])))
    assert w.shape == (0,)
    np.testing.assert_array_equal(host(ess), [0.0, 0.0])
    assert np.all(np.isneginf(host(lnz)))
    with pytest.raises(gwx.GwxError):
        gwx.importance_weights(cuda(np.zeros(3)), cuda(np.array([0])))


def test_importance_weights_after_log_likelihood(gwx):
    """Prior samples scored by the likelihood, then weighted: the plain prior-proposal path."""
    from test_gpu_parity import _events
    wl = workloads.workload("small")
    E = 4
    th_true, y, psd = _events(wl, E, 54)
    counts = workloads.ragged_counts(55, E, 20, 60)
    offs = np.concatenate([[0], np.cumsum(counts)])
    S = int(offs[-1])
    samples = workloads.random_theta(56, S, wl["prior"])
    samples[:, offs[:-1]] = th_true
    lnl_ref = likelihood.log_likelihood(y.astype(np.float64), psd, wl["seg_len"], wl["fs"], wl["f_lo"], samples,
                                        offs, wl["dets"])
    lnl = gwx.log_likelihood(cuda(y), cuda(psd), wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                             cuda(samples), cuda(offs))
    got = gwx.importance_weights(lnl, cuda(offs))
    _compare(got, importance.importance_weights(lnl_ref, offs), rtol=5e-3, z_atol=2e-3)


def test_scorer_matches_the_separate_calls(gwx):
    """The serving Scorer (preallocated, one stream) gives the same ESS, efficiency and
    evidence as sample_prior + log_likelihood + importance_weights called separately."""
    import paper_2407_19048_gb300.simulator as S
    from paper_2407_19048_gb300.scorer import Scorer
    wl = workloads.workload("small", B=3)
    sim = S.Simulator(wl)
    y, _, _ = sim.step(4)
    sc = Scorer(wl, 3000, sim.psd)
    for e, n in enumerate((3000, 1234, 57)):
        ess, eff, lnz = sc.score(y[e], n, 40 + e)
        th, _ = gwx.sample_prior(wl["prior"], 55, 40 + e, n, wl["L"], wl["N"])
        offs = cuda(np.array([0, n]))
        lnl = gwx.log_likelihood(y[e:e + 1].contiguous(), sim.psd, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"],
                                 0.0, th, offs)
        _, ess2, eff2, lnz2 = gwx.importance_weights(lnl, offs)
        assert ess == host(ess2)[0] and eff == host(eff2)[0] and lnz == host(lnz2)[0]

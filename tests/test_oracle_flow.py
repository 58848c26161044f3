"""Pins of the coupling-flow oracle (oracle/flow.py) against what the mathematics fixes:
invertibility, the change-of-variables log-determinant by brute force, normalisation by
Monte Carlo, the coupling structure, gradients by central differences, the mass-ratio
Jacobian, the prior's normalisation in the flow's coordinates, the identity flow's
standard normal, and the base draws' distribution."""
import math

import numpy as np
import pytest

import workloads
from oracle import flow as fl
from oracle.philox import uniform52  # noqa: F401  (the base draws use it through oracle.flow)

SHAPE = workloads.flow_shape(features=16, group=4, embed_hidden=16, context=8, layers=4, hidden=16)
K = SHAPE["layers"]


def _params(seed=3, **kw):
    return workloads.random_flow_params(seed, SHAPE, **kw)


def _context(seed, B):
    return np.random.default_rng(seed).normal(0.0, 1.0, (B, SHAPE["context"]))


def test_round_trip_sample_then_density():
    _, layers = fl.split_params(_params(), K)
    rng = np.random.default_rng(0)
    z = rng.normal(size=(64, 8))
    c = _context(1, 64)
    x, ss = fl.sample(z, c, layers, fl.exact)
    z2, ss2, _ = fl.density(x, c, layers, fl.exact)
    assert np.max(np.abs(z2 - z)) < 1e-11
    assert np.max(np.abs(ss2 - ss)) < 1e-11
    assert np.max(np.abs(x - z)) > 0.1          # the flow is not the identity


def test_log_determinant_by_finite_differences():
    _, layers = fl.split_params(_params(gain=1.5, last_gain=1.0), K)
    rng = np.random.default_rng(5)
    c = _context(2, 1)
    for _ in range(4):
        z0 = rng.normal(size=(1, 8))
        _, ss = fl.sample(z0, c, layers, fl.exact)
        h = 1e-6
        J = np.zeros((8, 8))
        for j in range(8):
            zp, zm = z0.copy(), z0.copy()
            zp[0, j] += h
            zm[0, j] -= h
            J[:, j] = (fl.sample(zp, c, layers, fl.exact)[0][0] - fl.sample(zm, c, layers, fl.exact)[0][0]) / (2 * h)
        sign, logdet = np.linalg.slogdet(J)
        assert sign > 0
        assert abs(logdet - ss[0]) < 1e-6 * max(1.0, abs(ss[0]))


def test_density_integrates_to_one():
    _, layers = fl.split_params(_params(seed=7), K)
    rng = np.random.default_rng(11)
    n, sig = 40000, 2.0
    x = rng.normal(0.0, sig, (n, 8))
    c = np.repeat(_context(3, 1), n, axis=0)
    z, ss, _ = fl.density(x, c, layers, fl.exact)
    log_q = fl.log_normal(z) - ss
    log_g = -0.5 * np.sum(x * x, axis=1) / sig ** 2 - 8 * math.log(sig) - 4 * math.log(2 * math.pi)
    w = np.exp(log_q - log_g)
    est, err = w.mean(), w.std() / math.sqrt(n)
    assert abs(est - 1.0) < 4 * err + 1e-3, (est, err)


def test_conditioner_sees_only_the_conditioning_half():
    _, layers = fl.split_params(_params(seed=9), K)
    rng = np.random.default_rng(13)
    v = rng.normal(size=(8, 8))
    c = _context(4, 8)
    for l in range(K):
        a, b = fl.SPLITS[l % 4]
        assert sorted(a + b) == list(range(8))
        o, _ = fl.conditioner(fl.conditioner_input(v, c, l, fl.exact), layers[l], fl.exact)
        vb = v.copy()
        vb[:, list(b)] += 1.0
        ob, _ = fl.conditioner(fl.conditioner_input(vb, c, l, fl.exact), layers[l], fl.exact)
        assert np.array_equal(o, ob)
        va = v.copy()
        va[:, list(a)] += 0.5
        oa, _ = fl.conditioner(fl.conditioner_input(va, c, l, fl.exact), layers[l], fl.exact)
        assert np.max(np.abs(oa - o)) > 1e-3
        # the step leaves the conditioning half alone and moves the other
        w, _ = fl.coupling(v, o, l, +1)
        assert np.array_equal(w[:, list(a)], v[:, list(a)])


def test_gradients_by_central_differences():
    params = _params(seed=21, gain=1.2, last_gain=1.0)
    rng = np.random.default_rng(17)
    B = 6
    feat = rng.normal(size=(B, SHAPE["features"]))
    x = rng.normal(size=(B, 8))
    mean, _, grads = fl.loss_and_grads(feat, x, params, K, fl.exact)
    picks = []
    for t in range(len(params)):
        for _ in range(2):
            picks.append((t, tuple(rng.integers(0, n) for n in params[t].shape)))
    h = 1e-6
    for t, idx in picks:
        pp = [p.astype(np.float64).copy() for p in params]
        pm = [p.astype(np.float64).copy() for p in params]
        pp[t][idx] += h
        pm[t][idx] -= h
        fd = (fl.loss_and_grads(feat, x, pp, K, fl.exact)[0] - fl.loss_and_grads(feat, x, pm, K, fl.exact)[0]) / (2 * h)
        g = grads[t][idx]
        assert abs(fd - g) < 1e-6 + 1e-5 * abs(g), (t, idx, fd, g)


def test_mass_ratio_jacobian():
    rng = np.random.default_rng(23)
    for _ in range(5):
        Mc, q = rng.uniform(5, 40), rng.uniform(0.2, 0.95)
        h = 1e-7
        J = np.zeros((2, 2))
        for j, (dm, dq) in enumerate(((h, 0.0), (0.0, h))):
            p = np.array(fl.masses(Mc + dm, q + dq))
            m = np.array(fl.masses(Mc - dm, q - dq))
            J[:, j] = (p - m) / (2 * h)
        big, small = fl.masses(Mc, q)
        assert abs(abs(np.linalg.det(J)) - big * big / Mc) < 1e-6 * big * big / Mc
        # and the masses give back (Mc, q)
        assert abs((big * small) ** 0.6 / (big + small) ** 0.2 - Mc) < 1e-12 * Mc
        assert abs(small / big - q) < 1e-14


def test_prior_density_integrates_to_one():
    prior = workloads.workload("small")["prior"]
    rng = np.random.default_rng(29)
    n = 400000
    # a box covering the support of (Mc, q); the other six coordinates sample their own ranges
    lo_mc = prior["m_lo"] * 2 ** -0.2
    hi_mc = prior["m_hi"] * 2 ** -0.2
    q_lo = prior["m_lo"] / prior["m_hi"]
    r = np.zeros((n, 8))
    r[:, 0] = rng.uniform(lo_mc, hi_mc, n)
    r[:, 1] = rng.uniform(q_lo, 1.0, n)
    r[:, 2] = rng.uniform(prior["d_lo"], prior["d_hi"], n)
    r[:, 3] = rng.uniform(-1, 1, n)
    r[:, 4] = rng.uniform(0, 2 * math.pi, n)
    r[:, 5] = rng.uniform(-1, 1, n)
    r[:, 6] = rng.uniform(prior["psi_lo"], prior["psi_hi"], n)
    r[:, 7] = rng.uniform(prior["phi_lo"], prior["phi_hi"], n)
    vol = ((hi_mc - lo_mc) * (1.0 - q_lo) * (prior["d_hi"] - prior["d_lo"]) * 2 * 2 * math.pi * 2
           * (prior["psi_hi"] - prior["psi_lo"]) * (prior["phi_hi"] - prior["phi_lo"]))
    w = np.exp(fl.log_prior_r(r, prior)) * vol
    est, err = w.mean(), w.std() / math.sqrt(n)
    assert abs(est - 1.0) < 4 * err, (est, err)
    # the support check rejects a point outside the mass box
    bad = r[:1].copy()
    bad[0, 0] = hi_mc * 1.5
    assert np.isneginf(fl.log_prior_r(bad, prior)[0])


def test_coordinates_round_trip_through_the_proposal_map():
    prior = workloads.workload("small")["prior"]
    th = workloads.random_theta(31, 50, prior)
    r = fl.coords(th)
    mean, scale = r.mean(axis=0), r.std(axis=0)
    x = fl.standardise(r, mean, scale)
    coin = np.where(th[0] < th[1], 0.25, 0.75)     # the coin that reproduces each draw's order
    # the uniforms that reproduce each draw's merger time and spins
    nuis = np.stack([(th[5] - prior["tc_lo"]) / (prior["tc_hi"] - prior["tc_lo"]),
                     (th[2] - prior["chi_lo"]) / (prior["chi_hi"] - prior["chi_lo"]),
                     (th[3] - prior["chi_lo"]) / (prior["chi_hi"] - prior["chi_lo"])], axis=1)
    out, log_q, lr = fl.proposal_params(x, np.zeros((50, 8)), np.zeros(50), mean, scale, prior, coin, nuis)
    assert np.all(np.isfinite(lr))
    assert np.max(np.abs(out - th)) < 1e-9 * np.max(np.abs(th))
    # identity flow at z = 0: ln q_r = -4 ln 2 pi - sum ln scale
    assert np.allclose(log_q, -4 * math.log(2 * math.pi) - np.sum(np.log(scale)))


def test_identity_flow_is_the_standard_normal():
    from scipy.stats import multivariate_normal
    params = _params(seed=37)
    emb, layers = fl.split_params(params, K)
    for l in range(K):
        layers[l][4][:] = 0.0          # V3
        layers[l][5][:] = 0.0          # e3
    rng = np.random.default_rng(41)
    x = rng.normal(size=(20, 8))
    c = _context(5, 20)
    z, ss, _ = fl.density(x, c, layers, fl.exact)
    assert np.array_equal(z, x) and np.all(ss == 0.0)
    assert np.allclose(fl.log_normal(x), multivariate_normal(np.zeros(8), np.eye(8)).logpdf(x), atol=1e-12)
    rows, mean = fl.nll(z, ss)
    assert np.allclose(rows, 0.5 * np.sum(x * x, axis=1) + 4 * math.log(2 * math.pi))


def test_base_normals_distribution():
    from scipy.stats import kstest
    z, coin = fl.base_normals(123, 7, np.arange(20000))
    for j in range(8):
        assert kstest(z[:, j], "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.03
    assert kstest(coin, "uniform").pvalue > 1e-3
    z2, _ = fl.base_normals(123, 8, np.arange(100))
    assert not np.allclose(z2, z[:100])             # the counter changes the stream
    z3, _ = fl.base_normals(123, 7, np.arange(50, 60))
    assert np.array_equal(z3, z[50:60])              # draws depend on their own index only


def test_sample_and_density_agree_on_the_proposal_density():
    prior = workloads.workload("small")["prior"]
    params = _params(seed=43)
    rng = np.random.default_rng(47)
    E = 3
    feat = rng.normal(size=(E, SHAPE["features"]))
    th = workloads.random_theta(48, 4000, prior)
    r = fl.coords(th)
    mean, scale = r.mean(axis=0), r.std(axis=0)
    offsets = np.array([0, 5, 5, 40])
    theta, log_q, lr = fl.sample_posterior(feat, params, K, mean, scale, prior, offsets, 99, 1, fl.exact)
    ev = fl.event_of(offsets, 40)
    ok = np.isfinite(lr)
    assert ok.sum() > 5
    lp = fl.log_prob(feat[ev], theta, params, K, mean, scale, fl.exact)
    assert np.max(np.abs(lp[ok] - log_q[ok])) < 1e-7


def test_parameters_the_flow_does_not_model_follow_their_prior():
    """Spins and t_c of flow draws are uniform over the prior's box, independent of the
    flow's coordinates (so their prior-to-proposal ratio is one)."""
    from scipy.stats import kstest
    prior = dict(workloads.workload("small")["prior"], chi_lo=-0.5, chi_hi=0.5)
    S = 20000
    nuis = fl.nuisance_uniforms(5, 3, np.arange(S))
    x = np.zeros((S, 8))
    th = workloads.random_theta(6, 1, prior)
    r = fl.coords(np.repeat(th, S, axis=1))
    out, _, _ = fl.proposal_params(x, np.zeros((S, 8)), np.zeros(S), r[0], np.ones(8), prior, np.full(S, 0.75), nuis)
    for row, lo, hi in ((5, prior["tc_lo"], prior["tc_hi"]), (2, prior["chi_lo"], prior["chi_hi"]),
                        (3, prior["chi_lo"], prior["chi_hi"])):
        assert kstest((out[row] - lo) / (hi - lo), "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(out[2], out[3])[0, 1]) < 0.03
    assert abs(np.corrcoef(out[5], out[2])[0, 1]) < 0.03
    _, coin = fl.base_normals(5, 3, np.arange(S))
    assert abs(np.corrcoef(coin, nuis[:, 0])[0, 1]) < 0.03


@pytest.mark.parametrize("rnd", ["exact", "bf16"])
def test_loss_is_the_mean_negative_log_density(rnd):
    f = fl.exact if rnd == "exact" else fl.round_bf16
    params = _params(seed=51)
    rng = np.random.default_rng(53)
    B = 10
    feat = fl.round_bf16(rng.normal(size=(B, SHAPE["features"])))
    prior = workloads.workload("small")["prior"]
    th = workloads.random_theta(54, B, prior)
    r = fl.coords(th)
    mean, scale = r.mean(axis=0), r.std(axis=0) + 1.0
    x = fl.standardise(r, mean, scale)
    m, rows, _ = fl.loss_and_grads(feat, x, params, K, f)
    lp = fl.log_prob(feat, th, params, K, mean, scale, f)
    assert np.allclose(rows, -(lp + np.sum(np.log(scale))), atol=1e-9)
    assert abs(m - rows.mean()) < 1e-12

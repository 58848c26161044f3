"""HEALPix sky maps on the GPU (gwx_skymap) against oracle.skymap (needs a GPU).
Pixel indices are integer decisions taken in FP64 on both sides, so each sample lands in
the same pixel; the map values differ only by the order of the FP64 additions."""
import math

import numpy as np
import pytest

import workloads
from oracle import skymap as sk

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


@pytest.mark.parametrize("nside", [1, 8, 64, 128])
def test_skymap_matches_oracle(gwx, nside):
    prior = workloads.workload("small")["prior"]
    th = workloads.random_theta(400 + nside, 5000, prior)
    w = np.random.default_rng(nside).uniform(0, 1, 5000)
    w[::7] = 0.0
    got = gwx.skymap(torch.from_numpy(th).cuda(), nside, weights=torch.from_numpy(w).cuda()).cpu().numpy()
    ref = sk.skymap(th[9], th[10], w, nside)
    assert np.array_equal(got > 0, ref > 0)                 # the same pixels are hit
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    assert abs(got.sum() - 1.0) < 1e-12


def test_skymap_unweighted_and_empty(gwx):
    th = np.zeros((11, 3))
    th[9] = [0.1, 0.1, 3.0]
    th[10] = [0.5, 0.5, -1.2]
    m = gwx.skymap(torch.from_numpy(th).cuda(), 4).cpu().numpy()
    p0 = sk.ang2pix_nest(4, math.pi / 2 - 0.5, 0.1)
    p1 = sk.ang2pix_nest(4, math.pi / 2 + 1.2, 3.0)
    assert abs(m[p0] - 2 / 3) < 1e-15 and abs(m[p1] - 1 / 3) < 1e-15 and abs(m.sum() - 1) < 1e-15
    z = gwx.skymap(torch.from_numpy(th).cuda(), 4, weights=torch.zeros(3, dtype=torch.float64, device="cuda"))
    assert float(z.abs().sum()) == 0.0


# ---------------------------------------------------------------- the flow's sky density
def _flow_case(nside, seed):
    import math
    import workloads
    from oracle import flow as fl, learn
    from oracle import skymap as sk
    import rounding_bounds as rb
    from paper_2407_19048_gb300.flow import FlowPosterior
    wl = workloads.workload("small")
    G = 16
    th_std = workloads.random_theta(300, 5000, wl["prior"])
    r_std = fl.coords(th_std)
    mean, scale = [float(v) for v in r_std.mean(axis=0)], [float(v) for v in r_std.std(axis=0)]
    fp = FlowPosterior(wl, layers=4, hidden=64, context=32, embed_hidden=64, group=G, seed=1)
    shape = workloads.flow_shape(features=fp.shape["features"], group=G, embed_hidden=64, context=32, layers=4,
                                 hidden=64)
    params = workloads.random_flow_params(seed, shape, gain=1.0, last_gain=0.5)
    fp.set_tensors(params)
    fp.mean, fp.scale = list(mean), list(scale)
    y = workloads.random_strain(seed + 1, (1, 2, wl["N"]), 1.0).astype(np.float32)
    S = 50
    theta = workloads.random_theta(seed + 2, S, wl["prior"])
    log_q = np.random.default_rng(seed + 3).normal(size=S)
    got = gwx_mod().flow_skymap(fp.shape, fp.params, fp.params16, mean, scale, torch.from_numpy(y).cuda(), wl["fs"],
                                wl["f_lo"], torch.from_numpy(theta).cuda(), torch.from_numpy(log_q).cuda(), nside)
    got = got.cpu().numpy()
    # the oracle: features, context, density at every pixel centre
    k_lo = int(math.ceil(wl["f_lo"] * wl["N"] / wl["fs"] - 1e-9))
    yd = y.astype(np.float64)
    f = learn.features(yd, k_lo, G, fp.shape["features"])
    ng = (wl["N"] // 2 - k_lo) // G
    col = 2 * ng
    for fn in (learn.cross_features, learn.lag_features):
        c = fn(yd, k_lo, G)
        f[:, col:col + c.shape[1]] = c
        col += c.shape[1]
    emb, layers = fl.split_params(params, 4)
    ctx, _ = fl.embed(fl.round_bf16(f), emb)
    r_fixed = fl.coords(theta[:, [int(np.argmax(log_q))]])[0]

    def log_q_at(r):
        z, ss, _ = fl.density(fl.standardise(r, mean, scale), np.repeat(ctx, len(r), axis=0), layers)
        return fl.log_normal(z) - ss - np.sum(np.log(scale))

    ref = sk.density_map(log_q_at, r_fixed, nside)
    ra, sd = sk.pixel_centres(nside)
    rows = np.tile(r_fixed, (len(ra), 1))
    rows[:, 4], rows[:, 5] = ra, sd
    # per-pixel bound of ln q (rounding of the flow's chain), with the feature row shared
    _, e = rb.log_prob(np.repeat(f, len(ra), axis=0), fl.standardise(rows, mean, scale), params, 4,
                       np.sum(np.log(scale)))
    return got, ref, e


def gwx_mod():
    import paper_2407_19048_gb300 as m
    return m


@pytest.mark.parametrize("nside", [4, 32])
def test_flow_sky_density_matches_oracle(gwx, nside):
    """The flow's density at every pixel centre, normalised: element by element within
    the propagated bound of ln q (the normalisation can move ln map by at most the largest
    per-pixel bound)."""
    got, ref, e = _flow_case(nside, 911 + nside)
    assert got.shape == ref.shape == (12 * nside * nside,)
    assert abs(got.sum() - 1.0) < 1e-9 and np.all(got >= 0.0)
    live = ref > 1e-12 * ref.max()
    dl = np.abs(np.log(got[live]) - np.log(ref[live]))
    tol = e[live] + e.max() + 1e-9
    assert np.all(dl <= tol), (float(dl.max()), float(np.max(dl / tol)))

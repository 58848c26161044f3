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

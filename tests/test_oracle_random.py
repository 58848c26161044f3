"""Pins for the oracle's Philox generator and prior draws (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox, prior
from oracle import constants as C
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*[np.uint32(x) for x in v[:6]])
        assert [int(o) for o in out] == v[6:]


def test_philox_vectorised_matches_scalar():
    idx = np.arange(17, dtype=np.uint32)
    vec = philox.philox4x32_10(idx, 3, 1, 9, 11, 12)
    for i in range(17):
        one = philox.philox4x32_10(np.uint32(i), 3, 1, 9, 11, 12)
        assert [int(a[i]) for a in vec] == [int(o) for o in one]


def test_uniform_maps_are_exact_and_open():
    assert philox.uniform52(0, 0) == 0.5 * 2.0 ** -52
    assert philox.uniform52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -52
    assert philox.uniform24(0) == 0.5 * 2.0 ** -24
    assert philox.uniform24(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -24
    assert np.float32(philox.uniform24(0x12345678)) == philox.uniform24(0x12345678)
    assert int(philox.bounded_index(0xFFFFFFFF, 7)) == 6
    assert int(philox.bounded_index(0, 7)) == 0


@pytest.fixture(scope="module")
def big_draw():
    wl = workloads.workload("small")
    th, off = prior.sample_prior(wl["prior"], 7, 3, 200000, wl["L"], wl["N"])
    return wl, th, off


def _ks_uniform(x, lo, hi):
    return stats.kstest((np.asarray(x) - lo) / (hi - lo), "uniform").pvalue


def test_prior_marginals(big_draw):
    wl, th, off = big_draw
    p = wl["prior"]
    assert _ks_uniform(th[C.M1], p["m_lo"], p["m_hi"]) > 1e-3
    assert _ks_uniform(th[C.M2], p["m_lo"], p["m_hi"]) > 1e-3
    assert _ks_uniform(th[C.CHI1], p["chi_lo"], p["chi_hi"]) > 1e-3
    assert _ks_uniform(th[C.DIST], p["d_lo"], p["d_hi"]) > 1e-3
    assert _ks_uniform(th[C.TC], p["tc_lo"], p["tc_hi"]) > 1e-3
    # Table 1: theta_jn ~ sine, dec ~ cosine, ra uniform on [0, 2 pi)
    assert _ks_uniform(np.cos(th[C.THETAJN]), -1.0, 1.0) > 1e-3
    assert _ks_uniform(np.sin(th[C.DEC]), -1.0, 1.0) > 1e-3
    assert _ks_uniform(th[C.RA], 0.0, 2 * math.pi) > 1e-3
    assert th[C.THETAJN].min() >= 0 and th[C.THETAJN].max() <= math.pi
    assert np.abs(th[C.DEC]).max() <= math.pi / 2


def test_prior_streams_independent(big_draw):
    wl, th, off = big_draw
    cc = np.corrcoef(th)
    off_diag = cc - np.diag(np.diag(cc))
    assert np.abs(off_diag).max() < 0.02


def test_offsets_uniform(big_draw):
    wl, th, off = big_draw
    n = wl["L"] - wl["N"] + 1
    assert off.min() >= 0 and off.max() <= n - 1
    counts = np.bincount(off * 16 // n, minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-3


def test_prior_counter_and_seed_change_stream():
    wl = workloads.workload("small")
    a, _ = prior.sample_prior(wl["prior"], 1, 0, 8, wl["L"], wl["N"])
    b, _ = prior.sample_prior(wl["prior"], 1, 1, 8, wl["L"], wl["N"])
    c, _ = prior.sample_prior(wl["prior"], 2, 0, 8, wl["L"], wl["N"])
    d, _ = prior.sample_prior(wl["prior"], 1, 0, 16, wl["L"], wl["N"])
    assert not np.allclose(a, b) and not np.allclose(a, c)
    np.testing.assert_array_equal(a, d[:, :8])   # draw b does not depend on the batch size

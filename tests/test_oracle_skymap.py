"""Pins of the HEALPix sky-map oracle (oracle/skymap.py): the nested hierarchy, equal
pixel areas, the twelve base faces, and the map's normalisation."""
import math

import numpy as np

from oracle import skymap as sk


def _uniform_sphere(rng, n):
    z = rng.uniform(-1, 1, n)
    return np.arccos(z), rng.uniform(0, 2 * math.pi, n)


def test_nested_hierarchy():
    rng = np.random.default_rng(1)
    theta, phi = _uniform_sphere(rng, 3000)
    for nside in (1, 2, 4, 8, 16, 32, 64):
        for t, p in zip(theta, phi):
            assert sk.ang2pix_nest(2 * nside, t, p) >> 2 == sk.ang2pix_nest(nside, t, p)


def test_pixels_have_equal_area():
    rng = np.random.default_rng(2)
    nside, n = 4, 192000
    theta, phi = _uniform_sphere(rng, n)
    counts = np.bincount([sk.ang2pix_nest(nside, t, p) for t, p in zip(theta, phi)], minlength=12 * nside ** 2)
    assert len(counts) == 12 * nside ** 2
    expect = n / len(counts)
    chi2 = np.sum((counts - expect) ** 2 / expect)
    dof = len(counts) - 1
    assert abs(chi2 - dof) < 5 * math.sqrt(2 * dof), chi2


def test_base_faces():
    for k in range(4):
        assert sk.ang2pix_nest(1, math.acos(2 / 3 + 0.1), math.pi / 4 + k * math.pi / 2) == k
        assert sk.ang2pix_nest(1, math.pi / 2, k * math.pi / 2 + 1e-3) == 4 + k
        assert sk.ang2pix_nest(1, math.acos(-2 / 3 - 0.1), math.pi / 4 + k * math.pi / 2) == 8 + k
    # the pixels of one face at nside 2 are the four children 4 f .. 4 f + 3
    rng = np.random.default_rng(3)
    theta, phi = _uniform_sphere(rng, 2000)
    for t, p in zip(theta, phi):
        assert sk.ang2pix_nest(2, t, p) // 4 == sk.ang2pix_nest(1, t, p)


def test_map_normalisation_and_weights():
    rng = np.random.default_rng(4)
    n = 500
    ra = rng.uniform(0, 2 * math.pi, n)
    dec = np.arcsin(rng.uniform(-1, 1, n))
    w = rng.uniform(0, 1, n)
    w[:100] = 0.0
    m = sk.skymap(ra, dec, w, 8)
    assert abs(m.sum() - 1.0) < 1e-12
    m2 = sk.skymap(ra[100:], dec[100:], w[100:], 8)
    np.testing.assert_allclose(m, m2, atol=1e-15)
    # a single sample puts all its mass in its own pixel
    m3 = sk.skymap(ra[:1], dec[:1], None, 16)
    assert m3.max() == 1.0 and np.argmax(m3) == sk.ang2pix_nest(16, math.pi / 2 - dec[0], ra[0])

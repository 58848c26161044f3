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


def test_pixel_centres_invert_the_pinned_pixel_index():
    for nside in (1, 2, 4, 8, 16, 32):
        for p in range(12 * nside * nside):
            assert sk.ang2pix_nest(nside, *sk.pix2ang_nest(nside, p)) == p


def test_pixel_centres_lie_on_the_rings():
    """4 nside - 1 iso-latitude rings: 4, 8, .., 4 (nside - 1) pixels in each polar ring,
    4 nside in each of the 2 nside + 1 rings of the belt; the centres balance (the sum of
    their unit vectors is zero) and their z take the rings' values."""
    nside = 8
    ra, sd = sk.pixel_centres(nside)
    z, counts = np.unique(np.round(sd, 12), return_counts=True)
    assert len(z) == 4 * nside - 1
    cap = [4 * i for i in range(1, nside)]
    assert list(counts) == cap + [4 * nside] * (2 * nside + 1) + cap[::-1]
    v = np.stack([np.sqrt(1 - sd ** 2) * np.cos(ra), np.sqrt(1 - sd ** 2) * np.sin(ra), sd])
    assert np.abs(v.sum(axis=1)).max() < 1e-9
    # the first north-cap ring sits at z = 1 - 1 / (3 nside^2)
    assert abs(z.max() - (1 - 1 / (3 * nside ** 2))) < 1e-12


def test_density_map_of_a_factorised_density():
    """A flow with identity layers is the standard normal in standardised coordinates, so
    its density factorises: the sky map is the product of the two normal factors of
    (RA, sin dec), whatever the other coordinates are held at."""
    mean = np.array([20.0, 0.6, 1000.0, 0.0, 2.5, 0.3, 3.0, 3.0])
    scale = np.array([5.0, 0.2, 400.0, 0.5, 0.7, 0.25, 1.8, 1.8])

    def log_q(r):
        x = (r - mean) / scale
        return -0.5 * np.sum(x * x, axis=1)

    nside = 16
    ra, sd = sk.pixel_centres(nside)
    want = np.exp(-0.5 * ((ra - mean[4]) / scale[4]) ** 2 - 0.5 * ((sd - mean[5]) / scale[5]) ** 2)
    want /= want.sum()
    for other in ([15.0, 0.9, 600.0, 0.2, 0.0, 0.0, 1.0, 5.0], [30.0, 0.3, 1500.0, -0.5, 0.0, 0.0, 4.0, 0.5]):
        m = sk.density_map(log_q, other, nside)
        np.testing.assert_allclose(m, want, rtol=1e-12, atol=1e-300)
    assert abs(m.sum() - 1.0) < 1e-12

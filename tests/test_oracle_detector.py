"""Pins for the oracle's detector response, delays and projection (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import detector, taylorf2
from oracle import constants as C
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def angles(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0, 2 * math.pi, n), np.arcsin(rng.uniform(-1, 1, n)), rng.uniform(0, 2 * math.pi, n))


def test_textbook_antenna_for_axis_aligned_detector():
    """Arms on the x and y axes: the tensor form reduces to the detector-frame formula
    (e.g. Sathyaprakash & Schutz, Living Rev. Rel. 12, 2 (2009))."""
    D = 0.5 * (np.outer([1, 0, 0], [1, 0, 0]) - np.outer([0, 1, 0], [0, 1, 0]))
    ra, dec, psi = angles(1000, 1)
    fp, fc = detector.antenna_from_tensor(D, ra, dec, psi, gmst=0.4)
    th = math.pi / 2 - dec
    ph = ra - 0.4
    a = 0.5 * (1 + np.cos(th) ** 2) * np.cos(2 * ph)
    b = np.cos(th) * np.sin(2 * ph)
    np.testing.assert_allclose(fp, a * np.cos(2 * psi) - b * np.sin(2 * psi), atol=1e-13)
    np.testing.assert_allclose(fc, a * np.sin(2 * psi) + b * np.cos(2 * psi), atol=1e-13)


@pytest.mark.parametrize("name", ["H1", "L1", "V1"])
def test_polarisation_rotation(name):
    ra, dec, psi = angles(500, 2)
    f0p, f0c = detector.antenna(name, ra, dec, np.zeros_like(psi))
    fp, fc = detector.antenna(name, ra, dec, psi)
    # sum of squares invariant; (F+, Fx) rotate by 2 psi
    np.testing.assert_allclose(fp ** 2 + fc ** 2, f0p ** 2 + f0c ** 2, atol=1e-14)
    np.testing.assert_allclose(fp, np.cos(2 * psi) * f0p - np.sin(2 * psi) * f0c, atol=1e-14)
    np.testing.assert_allclose(fc, np.sin(2 * psi) * f0p + np.cos(2 * psi) * f0c, atol=1e-14)
    assert np.all(fp ** 2 + fc ** 2 <= 1 + 1e-12)
    fpp, fcp = detector.antenna(name, ra, dec, psi + math.pi)
    np.testing.assert_allclose(fpp, fp, atol=1e-13)


@pytest.mark.parametrize("name", ["H1", "L1", "V1"])
def test_detector_tensor_structure(name):
    D, r = detector.geometry(name)
    np.testing.assert_allclose(D, D.T, atol=1e-15)
    assert abs(np.trace(D)) < 1e-15
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(D)), [-0.5, 0.0, 0.5], atol=1e-12)
    # null eigenvector is the local vertical: arms lie in the tangent plane
    w, V = np.linalg.eigh(D)
    up = V[:, np.argmin(np.abs(w))]
    lat, lon = map(math.radians, detector.SITES[name][:2])
    normal = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    assert abs(abs(up @ normal) - 1.0) < 1e-12
    assert 6.35e6 < np.linalg.norm(r) < 6.40e6


def test_baselines_match_published_light_times():
    for line in open(os.path.join(GOLDEN, "detector_baselines.txt")):
        if line.startswith("#"):
            continue
        a, b, ms, tol = line.split()
        ra_, rb = detector.geometry(a)[1], detector.geometry(b)[1]
        assert abs(np.linalg.norm(ra_ - rb) / C.C_MS * 1e3 - float(ms)) < float(tol)


def test_time_delays():
    ra, dec, _ = angles(4000, 3)
    tH = detector.time_delay("H1", ra, dec)
    tL = detector.time_delay("L1", ra, dec)
    rH, rL = detector.geometry("H1")[1], detector.geometry("L1")[1]
    bound = np.linalg.norm(rH - rL) / C.C_MS
    assert np.max(np.abs(tH - tL)) <= bound * (1 + 1e-12)
    assert np.max(np.abs(tH - tL)) > 0.95 * bound
    # antipodal directions: opposite delays
    np.testing.assert_allclose(detector.time_delay("H1", ra + math.pi, -dec), -tH, atol=1e-15)
    # a source overhead of a site arrives there |r| cos(angle) / c early
    lat, lon = map(math.radians, detector.SITES["H1"][:2])
    t = detector.time_delay("H1", np.array([lon]), np.array([lat]))
    assert t[0] < -0.021 and t[0] > -0.0213


def test_integer_sample_shift_is_a_roll():
    wl = workloads.workload("small")
    N, fs = wl["N"], wl["fs"]
    df = fs / N
    F = N // 2 + 1
    th = workloads.random_theta(5, 3, wl["prior"])
    hp, hc = taylorf2.generate_waveforms(th, wl["f_lo"], df, F)
    th2 = th.copy()
    th[C.TC] = 0.0
    m = np.array([17, 301, 1024])
    ra, dec = th[C.RA], th[C.DEC]
    base = detector.project(hp, hc, th, ["H1"], 0.0, df)
    # choose tc so that tc + delay is an integer number of samples
    th2[C.TC] = m / fs - detector.time_delay("H1", ra, dec)
    shifted = detector.project(hp, hc, th2, ["H1"], 0.0, df)
    dt0 = detector.time_delay("H1", ra, dec)
    for b in range(3):
        # base includes its own delay; undo it exactly in the frequency domain before rolling
        undo = np.exp(2j * math.pi * np.arange(F) * df * dt0[b])
        x0 = np.fft.irfft(base[b, 0] * undo, n=N)
        x1 = np.fft.irfft(shifted[b, 0], n=N)
        np.testing.assert_allclose(x1, np.roll(x0, m[b]), atol=1e-12 * np.abs(x0).max())

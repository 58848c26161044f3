"""Pins of oracle.learn: brute-force DFT, closed forms, finite differences."""
import math

import numpy as np

import workloads
from oracle import learn


def test_features_brute_force_dft():
    rng = np.random.default_rng(1)
    B, D, N, k_lo, G, F = 2, 2, 64, 3, 4, 32
    y = rng.normal(0.0, 1.0, (B, D, N))
    f = learn.features(y, k_lo, G, F)
    n = np.arange(N)
    ng = (N // 2 - k_lo) // G
    for b in range(B):
        for d in range(D):
            for g in range(ng):
                p = []
                for k in range(k_lo + g * G, k_lo + g * G + G):
                    X = sum(y[b, d, j] * complex(math.cos(2 * math.pi * k * j / N), -math.sin(2 * math.pi * k * j / N))
                            for j in n)
                    p.append(abs(X) ** 2 / N)
                assert abs(f[b, d * ng + g] - math.log(sum(p) / G)) < 1e-10
    assert np.all(f[:, D * ng:] == 0.0)


def test_features_of_white_noise_are_near_log_variance():
    rng = np.random.default_rng(2)
    y = rng.normal(0.0, 3.0, (64, 1, 4096))
    f = learn.features(y, 40, 64, 64)[:, :(2048 - 40) // 64]
    assert abs(np.mean(np.exp(f)) - 9.0) < 0.1     # E |Y_k|^2 / N = sigma^2


def test_chirp_mass_and_targets():
    assert abs(learn.chirp_mass(10.0, 10.0) - 10.0 * 2.0 ** -0.2) < 1e-12
    th = np.zeros((11, 2))
    th[0] = [10.0, 30.0]
    th[1] = [10.0, 20.0]
    th[4] = [500.0, 1500.0]
    t = learn.targets(th, [1.0, 2.0, 3.0], [2.0, 4.0, 5.0])
    np.testing.assert_allclose(t[:, 1], [(20.0 - 2.0) / 4.0, (50.0 - 2.0) / 4.0])
    np.testing.assert_allclose(t[:, 2], [(500.0 - 3.0) / 5.0, (1500.0 - 3.0) / 5.0])
    np.testing.assert_allclose(t[1, 0], ((600.0 ** 0.6 / 50.0 ** 0.2) - 1.0) / 2.0)


def test_gauss_nll_value_and_gradient():
    rng = np.random.default_rng(3)
    B, P = 5, 3
    out = rng.normal(0.0, 0.5, (B, 8))
    t = rng.normal(0.0, 1.0, (B, P))
    loss, mean, g = learn.gauss_nll(out, t)
    assert abs(mean - loss.mean()) < 1e-15
    z = out.copy()
    z[:, :P] = t
    z[:, P:2 * P] = 0.0
    assert np.all(learn.gauss_nll(z, t)[0] == 0.0)            # mu = t, sigma = 1
    h = 1e-6
    for (i, j) in [(0, 0), (2, 1), (4, 3), (1, 5), (3, 7)]:
        e = np.zeros_like(out)
        e[i, j] = h
        fd = (learn.gauss_nll(out + e, t)[1] - learn.gauss_nll(out - e, t)[1]) / (2 * h)
        assert abs(fd - g[i, j]) < 1e-8


def test_adamw_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    z = np.zeros(3)
    p1, m1, v1 = learn.adamw(p, g, z, z, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01, step=1)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)
    want = p - 0.1 * (g / (np.abs(g) + 1e-8) + 0.01 * p)
    np.testing.assert_allclose(p1, want, rtol=1e-15)


def test_mass_jacobian_by_finite_differences():
    for m1, m2 in [(30.0, 12.0), (11.0, 45.0), (25.0, 24.0)]:
        h = 1e-6
        def f(a, b):
            return np.array([learn.chirp_mass(a, b), a + b])
        J = np.column_stack([(f(m1 + h, m2) - f(m1 - h, m2)) / (2 * h), (f(m1, m2 + h) - f(m1, m2 - h)) / (2 * h)])
        Mc = learn.chirp_mass(m1, m2)
        assert abs(abs(np.linalg.det(J)) - 0.6 * Mc * abs(m1 - m2) / (m1 * m2)) < 1e-7


def test_proposal_round_trip_and_support():
    prior = workloads.workload("small")["prior"]
    mean, scale = [20.0, 60.0, 1100.0], [5.0, 15.0, 500.0]
    rng = np.random.default_rng(4)
    n = 200
    mu = rng.normal(0.0, 0.3, (n, 3))
    s = rng.normal(-1.0, 0.2, (n, 3))
    z = rng.normal(0.0, 1.0, (n, 3))
    u = rng.uniform(0.0, 1.0, n)
    m1, m2, D, lr = learn.proposal(mu, s, mean, scale, z, u, prior)
    x = np.asarray(mean) + np.asarray(scale) * (mu + np.exp(s) * z)
    ok = np.isfinite(m1)
    np.testing.assert_allclose(learn.chirp_mass(m1[ok], m2[ok]), x[ok, 0], rtol=1e-12)
    np.testing.assert_allclose((m1 + m2)[ok], x[ok, 1], rtol=1e-12)
    fin = np.isfinite(lr)
    assert fin.sum() > 50
    assert np.all((m1[fin] >= prior["m_lo"]) & (m1[fin] <= prior["m_hi"]) & (D[fin] >= prior["d_lo"]))
    # the order of the masses follows u
    both = ok & (m1 != m2)
    assert np.all((m1[both] < m2[both]) == (u[both] < 0.5))


def test_sample_proposal_prior_mode_and_angles():
    prior = workloads.workload("small")["prior"]
    truth = np.zeros((11, 2))
    truth[2], truth[3], truth[5] = [0.1, -0.2], [0.3, 0.0], [1.2, 1.4]
    offs = [0, 3000, 5000]
    th, lr = learn.sample_proposal(None, None, None, prior, truth, offs, seed=9, counter=1)
    assert np.all(lr == 0.0)
    assert np.all((th[0] >= prior["m_lo"]) & (th[0] <= prior["m_hi"]))
    np.testing.assert_array_equal(th[5][:3000], 1.2)
    np.testing.assert_array_equal(th[2][3000:], -0.2)
    # isotropic orientation and sky: cos(theta_JN) and sin(dec) uniform on [-1, 1]
    assert abs(np.mean(np.cos(th[7]))) < 0.05 and abs(np.mean(np.sin(th[10]))) < 0.05
    assert abs(np.var(np.cos(th[7])) - 1.0 / 3.0) < 0.03
    # the same (seed, counter) reproduces the draws
    th2, _ = learn.sample_proposal(None, None, None, prior, truth, offs, seed=9, counter=1)
    np.testing.assert_array_equal(th, th2)


def test_sample_proposal_normals():
    """Box-Muller normals of the proposal have mean 0 and variance 1."""
    u = learn.proposal_uniforms(3, 0, np.arange(20000))
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    z0, z1 = r * np.cos(2 * math.pi * u[:, 1]), r * np.sin(2 * math.pi * u[:, 1])
    for z in (z0, z1):
        assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.04
    assert abs(np.mean(z0 * z1)) < 0.03


def test_cross_features_brute_force_and_invariances():
    rng = np.random.default_rng(61)
    B, D, N, k_lo, G = 3, 3, 64, 3, 4
    y = rng.normal(size=(B, D, N))
    got = learn.cross_features(y, k_lo, G)
    # brute-force DFT
    n = np.arange(N)
    Y = np.array([[[np.sum(y[b, d] * np.exp(-2j * np.pi * k * n / N)) for k in range(N // 2 + 1)]
                   for d in range(D)] for b in range(B)])
    ng = (N // 2 - k_lo) // G
    pairs = learn.detector_pairs(D)
    assert pairs == [(0, 1), (0, 2), (1, 2)]
    for p, (a, c) in enumerate(pairs):
        for g in range(ng):
            ks = range(k_lo + g * G, k_lo + (g + 1) * G)
            num = sum(Y[:, a, k] * np.conj(Y[:, c, k]) for k in ks)
            den = np.sqrt(sum(abs(Y[:, a, k]) ** 2 for k in ks) * sum(abs(Y[:, c, k]) ** 2 for k in ks))
            np.testing.assert_allclose(got[:, 2 * p * ng + g], (num / den).real, atol=1e-12)
            np.testing.assert_allclose(got[:, (2 * p + 1) * ng + g], (num / den).imag, atol=1e-12)
    # Cauchy-Schwarz
    for p in range(len(pairs)):
        re, im = got[:, 2 * p * ng:(2 * p + 1) * ng], got[:, (2 * p + 1) * ng:(2 * p + 2) * ng]
        assert np.all(re * re + im * im <= 1.0 + 1e-12)
    # a common circular shift of every detector leaves the features unchanged
    np.testing.assert_allclose(learn.cross_features(np.roll(y, 7, axis=-1), k_lo, G), got, atol=1e-12)
    # identical channels are fully coherent
    same = np.repeat(y[:, :1], 2, axis=1)
    f = learn.cross_features(same, k_lo, G)
    np.testing.assert_allclose(f[:, :ng], 1.0, atol=1e-12)
    np.testing.assert_allclose(f[:, ng:], 0.0, atol=1e-12)


def test_cross_features_phase_of_a_delayed_tone():
    N, k0, tau, k_lo, G = 256, 37, 5, 20, 4
    n = np.arange(N)
    x = np.cos(2 * np.pi * k0 * n / N)
    y = np.stack([x, np.roll(x, tau)])[None]          # detector 1 lags detector 0 by tau samples
    f = learn.cross_features(y, k_lo, G)
    ng = (N // 2 - k_lo) // G
    g = (k0 - k_lo) // G
    # Y1 = Y0 e^{-2 pi i k tau / N}, so rho = e^{+2 pi i k0 tau / N}
    assert abs(f[0, g] - np.cos(2 * np.pi * k0 * tau / N)) < 1e-9
    assert abs(f[0, ng + g] - np.sin(2 * np.pi * k0 * tau / N)) < 1e-9


def test_lag_features_brute_force_and_track():
    rng = np.random.default_rng(71)
    B, D, N, k_lo, G = 2, 2, 64, 3, 4
    y = rng.normal(size=(B, D, N))
    got = learn.lag_features(y, k_lo, G)
    n = np.arange(N)
    Y = np.array([[[np.sum(y[b, d] * np.exp(-2j * np.pi * k * n / N)) for k in range(N // 2 + 1)]
                   for d in range(D)] for b in range(B)])
    ng = (N // 2 - k_lo) // G
    for d in range(D):
        for g in range(ng):
            ks = range(k_lo + g * G, k_lo + (g + 1) * G)
            num = sum(Y[:, d, k] * np.conj(Y[:, d, k + 1]) for k in ks)
            den = np.sqrt(sum(abs(Y[:, d, k]) ** 2 for k in ks) * sum(abs(Y[:, d, k + 1]) ** 2 for k in ks))
            np.testing.assert_allclose(got[:, 2 * d * ng + g], (num / den).real, atol=1e-12)
            np.testing.assert_allclose(got[:, (2 * d + 1) * ng + g], (num / den).imag, atol=1e-12)
    re, im = got[:, :ng], got[:, ng:2 * ng]
    assert np.all(re * re + im * im <= 1.0 + 1e-12)
    # an impulse at sample tau: Y_k = e^{-2 pi i k tau / N}, so lam = e^{+2 pi i tau / N} in every group
    tau = 11
    imp = np.zeros((1, 1, N))
    imp[0, 0, tau] = 1.0
    f = learn.lag_features(imp, k_lo, G)
    np.testing.assert_allclose(f[0, :ng], np.cos(2 * np.pi * tau / N), atol=1e-12)
    np.testing.assert_allclose(f[0, ng:], np.sin(2 * np.pi * tau / N), atol=1e-12)
    # a common circular shift by s samples rotates every lam by 2 pi s / N
    s = 5
    f0 = learn.lag_features(y, k_lo, G)
    f1 = learn.lag_features(np.roll(y, s, axis=-1), k_lo, G)
    l0 = f0[:, :ng] + 1j * f0[:, ng:2 * ng]
    l1 = f1[:, :ng] + 1j * f1[:, ng:2 * ng]
    np.testing.assert_allclose(l1, l0 * np.exp(2j * np.pi * s / N), atol=1e-12)


def test_adamw_clip_invariances():
    rng = np.random.default_rng(81)
    p, g = rng.normal(size=50), rng.normal(size=50) * 10.0
    z = np.zeros(50)
    # Adam's first step does not see the gradient's scale (eps aside), so clipping leaves it
    a = learn.adamw(p, g, z, z, 1e-2, 0.9, 0.999, 1e-12, 0.0, 1)
    b = learn.adamw(p, g, z, z, 1e-2, 0.9, 0.999, 1e-12, 0.0, 1, clip=0.5)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-9)
    # a clipped gradient's first moment has norm (1 - beta1) clip
    assert abs(np.linalg.norm(b[1]) - 0.1 * 0.5) < 1e-12
    # a clip above the norm changes nothing
    c = learn.adamw(p, g, z, z, 1e-2, 0.9, 0.999, 1e-8, 0.0, 1, clip=1e9)
    d = learn.adamw(p, g, z, z, 1e-2, 0.9, 0.999, 1e-8, 0.0, 1)
    for x, y in zip(c, d):
        np.testing.assert_array_equal(x, y)

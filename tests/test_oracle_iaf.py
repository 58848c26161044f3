"""Pins of the inverse-autoregressive flow oracle (Sec. 5.1), on the CPU: the paper's
parameter count, the autoregressive structure (exact independence, mask path counts, a
triangular Jacobian), the change of variables against a numerical Jacobian, an affine
special case against scipy's multivariate normal, normalisation by quadrature, the
paper's pass counts (one to sample, D for a density), a planted self-connection that
breaks invertibility, and the training gradient against central differences (weights,
data and context), masked weights without gradient and a planted dropped term."""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import iaf


def _rows(B, D, C, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, D)), rng.standard_normal((B, C))


def test_parameter_count_is_the_papers():
    """60 transforms x 6 masked layers of 100 units over D = 8 with the 8-dimensional
    representation as context: the paper's ~3.2 million."""
    n = iaf.n_params(8, 8)
    assert n == 3_228_960
    assert abs(n / 3.2e6 - 1.0) < 0.02
    stack = iaf.init(8, 8, seed=0)
    assert sum(t.size for layer in stack for t in layer) == n


@pytest.mark.parametrize("H,n_hidden,wide", [(100, 6, True), (7, 2, False)])
def test_outputs_ignore_their_own_and_later_coordinates(H, n_hidden, wide):
    """Exactly unchanged up to the perturbed coordinate at any width; changed after it at
    the paper's width (with one unit per degree, H = 7, a ReLU that is off for every row
    can cut the only path)."""
    D, C = 8, 8
    layer = iaf.init(D, C, H=H, n_hidden=n_hidden, K=1, seed=3, out_scale=1.0)[0]
    v, c = _rows(4, D, C, 7)
    mu0, s0 = iaf.made(layer, v, c)
    for j in range(D):
        w = v.copy()
        w[:, j] += 1.7
        mu1, s1 = iaf.made(layer, w, c)
        # exactly unchanged up to coordinate j, changed after it
        assert np.array_equal(mu1[:, :j + 1], mu0[:, :j + 1]) and np.array_equal(s1[:, :j + 1], s0[:, :j + 1])
        if wide and j < D - 1:
            assert np.all(np.abs(mu1[:, j + 1:] - mu0[:, j + 1:]).max(axis=0) > 0)


def test_mask_paths_reach_exactly_the_earlier_coordinates():
    D, C = 8, 8
    ms = iaf.masks(D, C)
    P = ms[0][:, :D]
    for m in ms[1:]:
        P = m @ P
    for block in (P[:D], P[D:]):          # shifts, log-scales
        for i in range(D):
            assert np.all(block[i, i:] == 0) and np.all(block[i, :i] > 0)
    assert np.all(ms[0][:, D:] == 1)     # the context reaches every first-layer unit


def test_round_trip():
    D, C = 8, 8
    stack = iaf.init(D, C, H=32, n_hidden=6, K=12, seed=2, out_scale=0.5)
    z, c = _rows(16, D, C, 1)
    x, lq = iaf.sample(stack, z, c)
    lq2, z2 = iaf.log_prob(stack, x, c)
    assert np.abs(z2 - z).max() < 1e-11
    assert np.abs(lq2 - lq).max() < 1e-10


def _jacobian(f, z, h=1e-6):
    D = z.shape[0]
    J = np.empty((D, D))
    for j in range(D):
        e = np.zeros(D)
        e[j] = h
        J[:, j] = (f(z + e) - f(z - e)) / (2 * h)
    return J


def test_one_transform_has_a_triangular_jacobian_with_diagonal_e_s():
    D, C = 8, 8
    layer = iaf.init(D, C, H=24, n_hidden=3, K=1, seed=4, out_scale=1.0)[0]
    v, c = _rows(1, D, C, 5)
    J = _jacobian(lambda u: iaf.forward(layer, u[None, :], c)[0][0], v[0])
    _, s = iaf.made(layer, v, c)
    assert np.abs(np.triu(J, 1)).max() == 0.0
    assert np.allclose(np.diag(J), np.exp(s[0]), rtol=1e-8, atol=0)


def test_density_is_the_change_of_variables():
    """ln q(x) = ln N(z) - ln|det dx/dz|, the determinant from a numerical Jacobian."""
    D, C = 8, 8
    stack = iaf.init(D, C, H=24, n_hidden=3, K=5, seed=6, out_scale=0.7)
    z, c = _rows(3, D, C, 8)
    for b in range(3):
        f = lambda u: iaf.sample(stack, u[None, :], c[b:b + 1])[0][0]
        _, logdet = np.linalg.slogdet(_jacobian(f, z[b]))
        _, lq = iaf.sample(stack, z[b:b + 1], c[b:b + 1])
        assert abs((iaf.log_normal(z[b:b + 1])[0] - logdet) - lq[0]) < 1e-6


def test_constant_autoencoders_give_scipys_gaussian():
    """With the output weights zero every transform is affine with constant shift and
    scale, so x is Gaussian: scipy's multivariate normal gives its density."""
    D, C, K = 4, 2, 3
    stack = iaf.init(D, C, H=10, n_hidden=2, K=K, seed=9)
    rng = np.random.default_rng(10)
    A, b = np.eye(D), np.zeros(D)
    R = np.eye(D)[::-1]                     # coordinate reversal
    for k, layer in enumerate(stack):
        layer[-2][:] = 0.0
        layer[-1][:] = rng.uniform(-1.5, 1.5, 2 * D)
        mu, s = layer[-1][:D], iaf.S_MAX * np.tanh(layer[-1][D:] / iaf.S_MAX)
        if k:
            A, b = R @ A, R @ b
        A, b = np.diag(np.exp(s)) @ A, np.exp(s) * b + mu
    x, c = _rows(6, D, C, 11)
    lq, _ = iaf.log_prob(stack, x, c)
    ref = multivariate_normal(mean=b, cov=A @ A.T).logpdf(x)
    assert np.abs(lq - ref).max() < 1e-10


def test_two_dimensional_density_integrates_to_one():
    D, C = 2, 1
    stack = iaf.init(D, C, H=8, n_hidden=2, K=4, seed=12, out_scale=0.6)
    h = 0.04
    g = np.arange(-12.0, 12.0, h) + h / 2
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    c = np.full((len(pts), C), 0.3)
    lq, _ = iaf.log_prob(stack, pts, c)
    assert abs(np.exp(lq).sum() * h * h - 1.0) < 2e-3


def test_pass_counts_one_to_sample_d_for_a_density():
    D, C, K = 8, 8, 5
    stack = iaf.init(D, C, H=16, n_hidden=2, K=K, seed=13)
    z, c = _rows(2, D, C, 14)
    st = {}
    x, _ = iaf.sample(stack, z, c, stats=st)
    assert st["made"] == K
    st = {}
    iaf.log_prob(stack, x, c, stats=st)
    assert st["made"] == K * D


def test_a_self_connection_breaks_the_inverse():
    """Planted mistake: output masks that keep degree-equal weights (>= instead of >) let
    mu_i see v_i, and the sequential inverse no longer recovers the input."""
    D, C = 8, 8
    layer = iaf.init(D, C, H=24, n_hidden=2, K=1, seed=15, out_scale=1.0)[0]
    d_in, d_h, d_out = iaf.degrees(D, 24, 2)
    rng = np.random.default_rng(16)
    bad = (d_out[:, None] >= d_h[-1][None, :]).astype(np.float64)
    layer[-2] = rng.standard_normal(bad.shape) / np.sqrt(24) * bad
    v, c = _rows(4, D, C, 17)
    y, _ = iaf.forward(layer, v, c)
    v2, _ = iaf.inverse(layer, y, c)
    assert np.abs(v2 - v).max() > 1e-3


def _fd_setup():
    D, C, H, nh, K = 4, 3, 6, 2, 3
    stack = iaf.init(D, C, H=H, n_hidden=nh, K=K, seed=21, out_scale=0.8)
    x, c = _rows(5, D, C, 22)
    return stack, x, c, iaf.masks(D, C, H, nh)


def _loss(stack, x, c):
    return -iaf.log_prob(stack, x, c)[0].mean()


def test_loss_is_the_mean_negative_log_density():
    stack, x, c, _ = _fd_setup()
    loss, _, _, _ = iaf.loss_and_grads(stack, x, c)
    assert abs(loss - _loss(stack, x, c)) < 1e-12


def test_gradient_against_central_differences():
    stack, x, c, ms = _fd_setup()
    _, G, dc, dx = iaf.loss_and_grads(stack, x, c)
    rng = np.random.default_rng(23)
    h = 1e-6

    def fd(arr, idx):
        arr[idx] += h
        lp = _loss(stack, x, c)
        arr[idx] -= 2 * h
        lm = _loss(stack, x, c)
        arr[idx] += h
        return (lp - lm) / (2 * h)

    for k in range(len(stack)):
        for t, arr in enumerate(stack[k]):
            for _ in range(4):
                idx = tuple(int(rng.integers(0, n)) for n in arr.shape)
                if t % 2 == 0 and ms[t // 2][idx] == 0:
                    continue
                assert abs(fd(arr, idx) - G[k][t][idx]) <= 1e-6 * max(abs(G[k][t][idx]), 1e-3), (k, t, idx)
    for i, j in [(0, 0), (2, 1), (4, 3)]:
        assert abs(fd(x, (i, j)) - dx[i, j]) <= 1e-6 * max(abs(dx[i, j]), 1e-3)
        if j < c.shape[1]:
            assert abs(fd(c, (i, j)) - dc[i, j]) <= 1e-6 * max(abs(dc[i, j]), 1e-3)


def test_masked_weights_get_no_gradient():
    stack, x, c, ms = _fd_setup()
    _, G, _, _ = iaf.loss_and_grads(stack, x, c)
    for k in range(len(stack)):
        for l, m in enumerate(ms):
            assert np.all(G[k][2 * l][m == 0] == 0.0)


def test_dropping_the_log_determinant_term_is_caught(monkeypatch):
    """Planted mistake: the backward pass without the log-determinant's weight on s."""
    stack, x, c, _ = _fd_setup()
    _, G_good, _, _ = iaf.loss_and_grads(stack, x, c)
    orig = iaf.inverse_backward
    monkeypatch.setattr(iaf, "inverse_backward", lambda layer, ms, passes, v, g, ws: orig(layer, ms, passes, v, g, 0 * ws))
    _, G_bad, _, _ = iaf.loss_and_grads(stack, x, c)
    out = len(G_good[0]) - 1                # the output layer's bias
    assert np.abs(G_bad[0][out] - G_good[0][out]).max() > 1e-3


def _proposal_setup():
    import workloads
    from oracle import flow as fl
    prior = workloads.workload("small")["prior"]
    r = fl.coords(workloads.random_theta(48, 4000, prior))
    return prior, r.mean(axis=0), r.std(axis=0), fl


def test_posterior_draws_and_density_agree():
    """ln q_r returned with each draw equals the D-pass density of its theta."""
    prior, mean, scale, fl = _proposal_setup()
    stack = iaf.init(8, 8, H=16, n_hidden=2, K=3, seed=31, out_scale=0.5)
    c_events = np.random.default_rng(32).standard_normal((3, 8))
    offsets = np.array([0, 5, 5, 40])
    theta, log_q, lr = iaf.sample_posterior(stack, c_events, mean, scale, prior, offsets, 99, 1)
    ok = np.isfinite(lr)
    assert ok.sum() > 5
    lp = iaf.log_prob_theta(stack, c_events[fl.event_of(offsets, 40)], theta, mean, scale)
    assert np.max(np.abs(lp[ok] - log_q[ok])) < 1e-7


@pytest.mark.parametrize("K", [3, 2])
def test_identity_stack_proposes_its_base_draws(K):
    """Zero output layers make every transform the identity: the draws are the Philox base
    normals themselves (reversed once for an even number of transforms), with no
    log-determinant, through the coupling flow's map to theta."""
    prior, mean, scale, fl = _proposal_setup()
    stack = iaf.init(8, 8, H=16, n_hidden=2, K=K, seed=33)
    for layer in stack:
        layer[-2][:] = 0.0
        layer[-1][:] = 0.0
    offsets = np.array([0, 30])
    got = iaf.sample_posterior(stack, np.zeros((1, 8)), mean, scale, prior, offsets, 7, 3)
    z, coin = fl.base_normals(7, 3, np.arange(30))
    x = z if K % 2 else z[:, ::-1]
    ref = fl.proposal_params(x, z, np.zeros(30), mean, scale, prior, coin,
                             fl.nuisance_uniforms(7, 3, np.arange(30)))
    for a, b in zip(got, ref):
        assert np.array_equal(np.isfinite(a), np.isfinite(b))
        assert np.allclose(a[np.isfinite(a)], b[np.isfinite(b)], rtol=0, atol=1e-12)

"""Pins of oracle.gemm: the bfloat16 format and the product, against brute force and
closed forms."""
import struct

import numpy as np

import workloads
from oracle import gemm


def test_bf16_known_patterns():
    bits = np.array([0x3F80, 0xC000, 0x0000, 0x8000, 0x3F81, 0x4049, 0x7F7F, 0x0080], dtype=np.uint16)
    want = [1.0, -2.0, 0.0, -0.0, 1.0 + 2.0 ** -7, 3.140625, (2.0 - 2.0 ** -7) * 2.0 ** 127, 2.0 ** -126]
    np.testing.assert_array_equal(gemm.bf16_to_f64(bits), want)


def test_bf16_decode_is_upper_half_of_binary32():
    for v in (0.15625, -1234.5, 7.0e-3, 3.0e30):
        word = struct.unpack("<I", struct.pack("<f", v))[0]
        hi = np.array([word >> 16], dtype=np.uint16)
        lo_zeroed = struct.unpack("<f", struct.pack("<I", word & 0xFFFF0000))[0]
        assert gemm.bf16_to_f64(hi)[0] == lo_zeroed


def test_round_to_nearest_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even pattern 0x3F80
    assert gemm.f64_to_bf16(1.0 + 2.0 ** -8) == 0x3F80
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: ties to 0x3F82
    assert gemm.f64_to_bf16(1.0 + 3 * 2.0 ** -8) == 0x3F82
    assert gemm.f64_to_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 0x3F81
    bits = workloads.random_bf16_bits(1, 1000)
    np.testing.assert_array_equal(gemm.f64_to_bf16(gemm.bf16_to_f64(bits)), bits)


def test_product_brute_force():
    a = workloads.random_bf16_bits(2, (5, 7))
    b = workloads.random_bf16_bits(3, (4, 7))
    A, B = gemm.bf16_to_f64(a), gemm.bf16_to_f64(b)
    C = gemm.gemm_nt(a, b)
    for m in range(5):
        for n in range(4):
            assert C[m, n] == sum(A[m, k] * B[n, k] for k in range(7))


def test_product_closed_forms():
    one = np.full((3, 9), 0x3F80, dtype=np.uint16)                # all ones
    np.testing.assert_array_equal(gemm.gemm_nt(one, one), np.full((3, 3), 9.0))
    eye = gemm.f64_to_bf16(np.eye(6))
    x = workloads.random_bf16_bits(4, (6, 6))
    np.testing.assert_array_equal(gemm.gemm_nt(x, eye), gemm.bf16_to_f64(x))    # X I^T = X
    np.testing.assert_array_equal(gemm.gemm_nt(eye, x), gemm.bf16_to_f64(x).T)  # I X^T = X^T
    np.testing.assert_array_equal(gemm.abs_product_sum(one, one), np.full((3, 3), 9.0))


def test_dense_activations():
    import math
    x = gemm.f64_to_bf16(np.array([[1.0, -2.0], [0.5, 0.25]]))
    w = gemm.f64_to_bf16(np.array([[1.0, 1.0], [2.0, -1.0], [0.0, 0.0]]))
    b = np.array([0.5, -1.0, 3.0])
    z = np.array([[1.0 - 2.0 + 0.5, 2.0 + 2.0 - 1.0, 3.0], [0.75 + 0.5, 1.0 - 0.25 - 1.0, 3.0]])
    np.testing.assert_array_equal(gemm.dense(x, w, b), z)
    np.testing.assert_array_equal(gemm.dense(x, w, b, gemm.RELU), np.maximum(z, 0))
    g = gemm.dense(x, w, b, gemm.GELU)
    # GELU(0) = 0, GELU(z) - GELU(-z) = z, GELU(z) -> z for large z
    for (i, j), v in np.ndenumerate(z):
        assert abs(g[i, j] - v * 0.5 * math.erfc(-v / math.sqrt(2.0))) < 1e-15
    big = gemm.dense(gemm.f64_to_bf16(np.array([[8.0]])), gemm.f64_to_bf16(np.array([[1.0]])), None, gemm.GELU)
    assert abs(big[0, 0] - 8.0) < 1e-12
    p = gemm.dense(x, w, None, gemm.GELU) - gemm.dense(gemm.f64_to_bf16(-gemm.bf16_to_f64(x)), w, None, gemm.GELU)
    np.testing.assert_allclose(p, gemm.gemm_nt(x, w), rtol=1e-14, atol=1e-14)


def _loss(x_bits, w_bits, b, act, g):
    """L = sum(g * Y) with X, W given as FP64 values (no bfloat16 rounding)."""
    return float(np.sum(g * gemm.dense(x_bits, w_bits, b, act)))


def test_dense_backward_matches_finite_differences():
    """Central differences of L = sum(G * act(X W^T + b)) in FP64, perturbing the decoded
    inputs (the oracle differentiates the exact-value function)."""
    rng = np.random.default_rng(5)
    M, N, K = 3, 4, 5
    x = workloads.random_bf16_bits(6, (M, K), exp_lo=-2, exp_hi=0)
    w = workloads.random_bf16_bits(7, (N, K), exp_lo=-2, exp_hi=0)
    b = rng.normal(0.0, 0.3, N)
    g = rng.normal(0.0, 1.0, (M, N))
    X, W = gemm.bf16_to_f64(x), gemm.bf16_to_f64(w)
    for act in (0, gemm.RELU, gemm.GELU):
        dX, dW, db, _ = gemm.dense_backward(x, w, b, act, g)

        def L(Xv, Wv, bv):
            z = Xv @ Wv.T + bv[None, :]
            if act == gemm.RELU:
                y = np.maximum(z, 0)
            elif act == gemm.GELU:
                import math
                y = z * 0.5 * (1 + np.vectorize(math.erf)(z / math.sqrt(2)))
            else:
                y = z
            return float(np.sum(g * y))
        h = 1e-6
        for (i, j) in [(0, 0), (2, 4), (1, 2)]:
            e = np.zeros_like(X); e[i, j] = h
            assert abs((L(X + e, W, b) - L(X - e, W, b)) / (2 * h) - dX[i, j]) < 1e-6
        for (i, j) in [(0, 0), (3, 4), (2, 1)]:
            e = np.zeros_like(W); e[i, j] = h
            assert abs((L(X, W + e, b) - L(X, W - e, b)) / (2 * h) - dW[i, j]) < 1e-6
        for j in range(N):
            e = np.zeros(N); e[j] = h
            assert abs((L(X, W, b + e) - L(X, W, b - e)) / (2 * h) - db[j]) < 1e-6


def test_act_grad_closed_forms():
    import math
    z = np.array([-2.0, -0.5, 0.0, 0.5, 3.0])
    np.testing.assert_array_equal(gemm.act_grad(z, gemm.RELU), [0, 0, 0, 1, 1])
    gz = gemm.act_grad(z, gemm.GELU)
    assert gz[2] == 0.5                                   # GELU'(0) = 1/2
    for v, d in zip(z, gz):                               # GELU'(z) + GELU'(-z) = 1
        assert abs(d + gemm.act_grad(np.array([-v]), gemm.GELU)[0] - 1.0) < 1e-15
    np.testing.assert_array_equal(gemm.act_grad(z, 0), np.ones(5))

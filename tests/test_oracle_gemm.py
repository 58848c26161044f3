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

"""Dense products for the learned part (oracle; test infrastructure).

The network that the simulated batches train (the embedding network of Sec. 4 and the
normalizing flow of Sec. 5) is a stack of dense contractions; its GPU kernels take
bfloat16 operands and accumulate in FP32.  The oracle states the product in FP64 on
the exact values of the bfloat16 operands:

    C[m][n] = sum_k A[m][k] B[n][k]        (A is M x K, B is N x K, both row-major),

and the bfloat16 format itself: 1 sign bit, 8 exponent bits (bias 127) and 7 stored
mantissa bits, i.e. the upper half of an IEEE binary32 word.
"""
import numpy as np


def bf16_to_f64(bits):
    """Decode bfloat16 bit patterns (uint16 array) exactly: the pattern is the upper
    16 bits of a binary32 value."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def f64_to_bf16(x):
    """Round to the nearest bfloat16, ties to even (finite inputs), as bit patterns."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    return r.astype(np.uint16)


def gemm_nt(a_bits, b_bits):
    """C = A B^T in FP64 from bfloat16 operands A [M][K], B [N][K]."""
    return bf16_to_f64(a_bits) @ bf16_to_f64(b_bits).T


def abs_product_sum(a_bits, b_bits):
    """sum_k |A[m][k]| |B[n][k]|: the scale of the rounding error of the FP32 sum."""
    return np.abs(bf16_to_f64(a_bits)) @ np.abs(bf16_to_f64(b_bits)).T


RELU, GELU = 1, 2


def dense(x_bits, w_bits, bias=None, act=0):
    """A dense layer Y = act(X W^T + b) in FP64: X bfloat16 [M][K], W bfloat16 [N][K],
    b [N] (FP64 values of the FP32 bias), act 0 = identity, 1 = ReLU max(0, z),
    2 = GELU z Phi(z) with Phi the standard normal CDF, (1 + erf(z / sqrt 2)) / 2."""
    import math
    z = gemm_nt(x_bits, w_bits)
    if bias is not None:
        z = z + np.asarray(bias, dtype=np.float64)[None, :]
    if act == RELU:
        return np.maximum(z, 0.0)
    if act == GELU:
        erf = np.vectorize(math.erf)
        return z * 0.5 * (1.0 + erf(z / math.sqrt(2.0)))
    return z


def act_grad(z, act):
    """d act / dz: ReLU 1 for z > 0 else 0; GELU Phi(z) + z phi(z) (phi the standard
    normal density)."""
    import math
    z = np.asarray(z, dtype=np.float64)
    if act == RELU:
        return (z > 0).astype(np.float64)
    if act == GELU:
        erf = np.vectorize(math.erf)
        return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return np.ones_like(z)


def dense_backward(x_bits, w_bits, bias, act, dy):
    """Gradients of L with dL/dY = dy for Y = act(X W^T + b), by the chain rule in FP64:
    dZ = dy * act'(Z), dX = dZ W, dW = dZ^T X, db = sum over rows of dZ.
    Returns (dX [M][K], dW [N][K], db [N], dZ [M][N])."""
    X, W = bf16_to_f64(x_bits), bf16_to_f64(w_bits)
    z = X @ W.T
    if bias is not None:
        z = z + np.asarray(bias, dtype=np.float64)[None, :]
    dz = np.asarray(dy, dtype=np.float64) * act_grad(z, act)
    return dz @ W, dz.T @ X, dz.sum(axis=0), dz

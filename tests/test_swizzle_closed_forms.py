"""The shared-memory addressing of the radix-16 passes (CPU, no GPU).

The passes keep complex points at the swizzled slot sw16(i) = i ^ ((i >> 4) & 15) and
address x[a + b] with a per-thread part a < 2^s and a compile-time part b = r 2^s, r < 16.
The kernels form the slot from sw16(a) alone: as (sw16(a) ^ ((b >> 4) & 15)) + b for loads
(a = j < n/R) and for stores at strides Ns >= 16, and as sw16(a) ^ b ^ ((b >> 4) & 15) for
stores at smaller strides, where a's mask reaches into b's bits.  This test checks those
forms against sw16 itself for every radix, stride and transform size the kernels
instantiate, so a wrong field split fails here before a GPU run."""
import pytest


def sw16(i):
    return i ^ ((i >> 4) & 15)


def slot_add(sa, b):
    return (sa ^ ((b >> 4) & 15)) + b


def slot_xor(sa, b):
    return sa ^ b ^ ((b >> 4) & 15)


@pytest.mark.parametrize("logn", range(7, 14))
def test_strided_loads(logn):
    n = 1 << logn
    for R in (2, 4, 8, 16):
        nR = n // R
        for j in range(nR):
            for r in range(R):
                assert slot_add(sw16(j), r * nR) == sw16(j + r * nR), (R, nR, j, r)


@pytest.mark.parametrize("logn", range(7, 14))
def test_pass_stores(logn):
    n = 1 << logn
    for R in (2, 4, 8, 16):
        Ns = 1
        while R * Ns <= n:
            for j in range(n // R):
                jm = j & (Ns - 1)
                idx = (j - jm) * R + jm
                slot = slot_add if Ns >= 16 else slot_xor
                for r in range(R):
                    assert slot(sw16(idx), r * Ns) == sw16(idx + r * Ns), (R, Ns, j, r)
            Ns *= 2


def test_the_mask_of_b_matters():
    """The check is sharp: leaving out b's share of the mask misplaces points."""
    n, R = 1024, 16
    nR = n // R
    assert any(sw16(j) + r * nR != sw16(j + r * nR) for j in range(nR) for r in range(R))
    # and the additive form is wrong for stores at strides below 16
    Ns = 2
    assert any(slot_add(sw16((j - (j & 1)) * R + (j & 1)), r * Ns) != sw16((j - (j & 1)) * R + (j & 1) + r * Ns)
               for j in range(nR) for r in range(R))

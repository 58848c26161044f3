"""The ResNet's stride-1 convolutions as implicit GEMMs (gwx_conv1d_bf16 and its
backward; needs a GPU) against oracle.resnet, element by element.

Inputs are bfloat16 values, so both sides multiply the same numbers; the GPU sums FP32
products in the tensor cores' order, the oracle in FP64.  Each FP32 output is held to
2 K 2^-24 sum |a b| over its K terms (+ the addend's own rounding), the bound of any
summation order of K FP32 terms.  The backward rounds dz to bfloat16 before its
products, which the oracle does as well (round_bf16).  Shapes: several tiles of 128
times, one to three channel blocks, k = 5 and k = 1, an addend; the training shape of the
first stage (512 windows x 512 times x 64 channels) on sampled outputs, and its weight
gradient in full at 64 windows (32,768 summed rows per element)."""
import numpy as np
import pytest

from oracle import resnet as rn
from oracle.flow import round_bf16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def _bf(rng, shape, scale=1.0):
    return round_bf16(rng.standard_normal(shape) * scale)


def _dev16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)


def _dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.float().cpu().numpy().astype(np.float64)


def _bound(absA, absB, K, extra=0.0):
    """2 K 2^-24 sum |a||b| for every output of absA @ absB.T (+ slack for an addend)."""
    return 2.0 * K * U32 * (absA @ absB.T) + extra + 1e-30


CASES = [
    # B, T, C, O, k
    (2, 256, 64, 64, 5),
    (3, 128, 128, 256, 5),
    (1, 384, 64, 128, 1),
    (2, 128, 192, 64, 3),
]


@pytest.mark.parametrize("B,T,C,O,k", CASES)
@pytest.mark.parametrize("with_addend", [False, True])
def test_conv_forward_matches_oracle(gwx, B, T, C, O, k, with_addend):
    rng = np.random.default_rng(B * 1000 + T + C + O + k)
    x = _bf(rng, (B, T, C))
    W = _bf(rng, (O, k * C), 1.0 / np.sqrt(k * C))
    add = rng.standard_normal((B, T, O)).astype(np.float32).astype(np.float64) if with_addend else None
    p = (k - 1) // 2
    ref = rn.conv(x, W, k, 1, p)[0] + (add if add is not None else 0.0)
    cols = rn.im2col(np.abs(x), k, 1, p).reshape(B * T, -1)
    bound = _bound(cols, np.abs(W), k * C, 0.0 if add is None else U32 * np.abs(add).reshape(B * T, O) * 2)
    z = gwx.conv1d_bf16(_dev16(x), _dev16(W), k, addend=_dev32(add) if add is not None else None)
    got = _host(z).reshape(B * T, O)
    err = np.abs(got - ref.reshape(B * T, O))
    assert np.all(err <= bound), (err.max(), np.unravel_index(np.argmax(err - bound), err.shape))
    assert gwx._lib.load().gwx_device_status() == 0


@pytest.mark.parametrize("B,T,C,O,k", CASES)
def test_conv_backward_matches_oracle(gwx, B, T, C, O, k):
    rng = np.random.default_rng(7 * B + T + 3 * C + O + k)
    x = _bf(rng, (B, T, C))
    W = _bf(rng, (O, k * C), 1.0 / np.sqrt(k * C))
    dz = rng.standard_normal((B, T, O)).astype(np.float32).astype(np.float64)
    add = rng.standard_normal((B, T, C)).astype(np.float32).astype(np.float64)
    p = (k - 1) // 2
    dzr = round_bf16(dz).reshape(B * T, O)
    cols = rn.im2col(x, k, 1, p).reshape(B * T, -1)
    dx_ref = rn.col2im((dzr @ W).reshape(B, T, -1), T, C, k, 1, p) + add
    dW_ref = dzr.T @ cols
    # bounds: dx sums k O products per element, dW sums B T
    dcols_abs = (np.abs(dzr) @ np.abs(W)).reshape(B, T, -1)
    dx_bound = 2.0 * k * O * U32 * rn.col2im(dcols_abs, T, C, k, 1, p) + 2 * U32 * np.abs(add) + 1e-30
    dW_bound = _bound(np.abs(dzr).T, np.abs(cols).T, B * T)
    dx, dW = gwx.conv1d_bf16_backward(_dev32(dz), _dev16(x), _dev16(W), k, addend=_dev32(add))
    e1 = np.abs(_host(dx) - dx_ref)
    assert np.all(e1 <= dx_bound), (e1.max(), np.unravel_index(np.argmax(e1 - dx_bound), e1.shape))
    e2 = np.abs(_host(dW) - dW_ref)
    assert np.all(e2 <= dW_bound), (e2.max(), np.unravel_index(np.argmax(e2 - dW_bound), e2.shape))
    assert gwx._lib.load().gwx_device_status() == 0


def test_conv_at_training_shape_sampled(gwx):
    """Stage 1 of the summary at its training shape: 512 windows, 512 times, 64 channels,
    k = 5; forward and input gradient on sampled (b, t) rows, all output channels."""
    B, T, C, O, k = 512, 512, 64, 64, 5
    p = 2
    rng = np.random.default_rng(5)
    x = _bf(rng, (B, T, C))
    W = _bf(rng, (O, k * C), 1.0 / np.sqrt(k * C))
    dz = rng.standard_normal((B, T, O)).astype(np.float32).astype(np.float64)
    xd, Wd = _dev16(x), _dev16(W)
    z = _host(gwx.conv1d_bf16(xd, Wd, k))
    dx, _ = gwx.conv1d_bf16_backward(_dev32(dz), xd, Wd, k, want_dW=False)
    dx = _host(dx)
    dzr = round_bf16(dz)
    Wr = W.reshape(O, k, C)
    samples = [(0, 0), (0, 1), (B - 1, T - 1), (B - 1, T - 2), (7, 127), (7, 128), (300, 255), (301, 256)]
    samples += [(int(b), int(t)) for b, t in zip(rng.integers(0, B, 24), rng.integers(0, T, 24))]
    for b, t in samples:
        zr = np.zeros(O)
        za = np.zeros(O)
        dr = np.zeros(C)
        da = np.zeros(C)
        for j in range(k):
            ts = t + j - p
            if 0 <= ts < T:
                zr += Wr[:, j, :] @ x[b, ts]
                za += np.abs(Wr[:, j, :]) @ np.abs(x[b, ts])
            to = t - j + p          # output rows that read x[b][t] through tap j
            if 0 <= to < T:
                dr += Wr[:, j, :].T @ dzr[b, to]
                da += np.abs(Wr[:, j, :]).T @ np.abs(dzr[b, to])
        assert np.all(np.abs(z[b, t] - zr) <= 2 * k * C * U32 * za + 1e-30), (b, t)
        assert np.all(np.abs(dx[b, t] - dr) <= 2 * k * O * U32 * da + 1e-30), (b, t)
    assert gwx._lib.load().gwx_device_status() == 0


def test_conv_weight_gradient_over_32768_rows(gwx):
    """dW of the first stage's convolution summed over 64 windows x 512 times, in full."""
    B, T, C, O, k = 64, 512, 64, 64, 5
    rng = np.random.default_rng(11)
    x = _bf(rng, (B, T, C))
    W = _bf(rng, (O, k * C), 1.0 / np.sqrt(k * C))
    dz = rng.standard_normal((B, T, O)).astype(np.float32).astype(np.float64)
    _, dW = gwx.conv1d_bf16_backward(_dev32(dz), _dev16(x), _dev16(W), k, want_dx=False)
    dzr = round_bf16(dz).reshape(B * T, O)
    cols = rn.im2col(x, k, 1, 2).reshape(B * T, -1)
    ref = dzr.T @ cols
    bound = _bound(np.abs(dzr).T, np.abs(cols).T, B * T)
    err = np.abs(_host(dW) - ref)
    assert np.all(err <= bound), (err.max(), np.unravel_index(np.argmax(err - bound), err.shape))


def test_conv_matches_the_im2col_path_bit_for_bit_in_the_forward(gwx):
    """The implicit product reads the same bfloat16 operands in the same K order as the
    materialised im2col rows times W^T on the same kernel and tile shape (256 output
    channels: 128 x 256 tiles on both), so the two agree exactly."""
    B, T, C, O, k = 4, 256, 128, 256, 5
    rng = np.random.default_rng(3)
    xd = _dev16(_bf(rng, (B, T, C)))
    Wd = _dev16(_bf(rng, (O, k * C), 1.0 / np.sqrt(k * C)))
    z = gwx.conv1d_bf16(xd, Wd, k)
    cols = torch.empty((B * T, k * C), dtype=torch.bfloat16, device="cuda")
    lib = gwx._lib.load()
    gwx._check(lib.gwx_im2col(gwx._ptr(xd), B, T, C, k, 1, 2, k * C, gwx._ptr(cols), gwx._stream()))
    z2 = gwx.dense_bf16(cols, Wd, None, act=gwx.ACT_NONE, out_dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.equal(z.reshape(B * T, O), z2)


def test_resnet_with_implicit_convolutions_matches_the_im2col_network(gwx):
    """The whole summary (stem, (5, 3, 3) blocks of 64 / 128 / 256 channels) on 16 windows
    of 2 x 2048 samples with its stride-1 convolutions as implicit GEMMs, against the same
    network and parameters on im2col rows.  Both paths are checked against the oracle
    operation by operation above and in test_gpu_resnet.py; here the plumbing (tape,
    inputs, addends) is compared: the representation and every gradient tensor agree to
    1e-2 of their norm (the two differ only in FP32 summation order, which moves a few
    bfloat16 activations by one unit)."""
    from paper_2407_19048_gb300.resnet import ResNet1D
    rng = np.random.default_rng(21)
    y = torch.from_numpy(rng.standard_normal((16, 2, 2048)).astype(np.float32)).cuda()
    a = ResNet1D(2, 64, seed=4, implicit=True)
    b = ResNet1D(2, 64, seed=4, implicit=False)
    ca = a.forward(y)
    cb = b.forward(y)
    dc = torch.from_numpy(rng.standard_normal((16, 64)).astype(np.float32)).cuda()
    ga = a.backward(dc)
    gb = b.backward(dc)
    torch.cuda.synchronize()
    used = [t for t in a.tape["blocks"] if t[1] is None]
    # blocks whose first convolution ran implicitly: the five of stage 1 and the two
    # non-entry blocks of stages 2 and 3 (every block's second convolution does too)
    assert len(used) == 9
    assert all(t[5] is None for t in a.tape["blocks"])
    assert torch.linalg.norm(ca - cb) <= 1e-2 * torch.linalg.norm(cb)
    for name in gb:
        assert torch.linalg.norm(ga[name] - gb[name]) <= 1e-2 * torch.linalg.norm(gb[name]) + 1e-30, name
    assert gwx._lib.load().gwx_device_status() == 0

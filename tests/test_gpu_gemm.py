"""Parity of gwx_gemm_bf16 (tcgen05 tensor cores) with oracle.gemm (needs a GPU).

Both sides take the same bfloat16 bit patterns.  The kernel forms exact products and
sums them in FP32, so |C - C_oracle| <= 2 K 2^-24 sum_k |A_mk| |B_nk| (a bound on
recursive FP32 summation of K terms); a bfloat16 output adds the rounding to 8
significant bits, at most 2^-8 |C|.
"""
import numpy as np
import pytest

import workloads
from oracle import gemm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def _bf16(bits):
    return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)


def _check(gwx, M, N, K, seed, out_dtype=torch.float32):
    a = workloads.random_bf16_bits(seed, (M, K))
    b = workloads.random_bf16_bits(seed + 1, (N, K))
    C = gwx.gemm_bf16(_bf16(a), _bf16(b), out_dtype=out_dtype)
    gwx.device_status()
    got = C.float().cpu().numpy().astype(np.float64)
    ref = gemm.gemm_nt(a, b)
    tol = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(a, b)
    if out_dtype == torch.bfloat16:
        tol = tol * (1.0 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= tol + 1e-30), (float(err.max()), float((err / (tol + 1e-30)).max()))


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 512, 256), (384, 768, 1024), (128, 256, 8)])
def test_gemm_full_tiles(gwx, M, N, K):
    _check(gwx, M, N, K, 60 + K)


@pytest.mark.parametrize("M,N,K", [(1, 1, 8), (200, 300, 72), (1000, 700, 520), (129, 257, 136)])
def test_gemm_ragged(gwx, M, N, K):
    """Rows, columns and the K tail past the 128 x 256 x 64 tiles."""
    _check(gwx, M, N, K, 70 + M)


@pytest.mark.parametrize("M,N,K", [(256, 512, 192), (130, 300, 64)])
def test_gemm_bf16_output(gwx, M, N, K):
    _check(gwx, M, N, K, 80 + N, out_dtype=torch.bfloat16)


def test_gemm_large(gwx):
    """A 2048 x 4096 x 4096 product (many tiles, 64 k-blocks: the stage ring wraps)."""
    M, N, K = 2048, 4096, 4096
    a = workloads.random_bf16_bits(90, (M, K))
    b = workloads.random_bf16_bits(91, (N, K))
    C = gwx.gemm_bf16(_bf16(a), _bf16(b))
    gwx.device_status()
    rows = np.array([0, 1, 127, 128, 1000, 2047])
    got = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    ref = gemm.gemm_nt(a[rows], b)
    tol = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(a[rows], b)
    assert np.all(np.abs(got - ref) <= tol)


def _rows(M, seed, extra=12):
    """Rows at and next to every 128-row boundary, the last row, and a few at random."""
    b = [r for t in range(0, M, 128) for r in (t - 1, t, t + 1) if 0 <= r < M] + [M - 1]
    return np.unique(np.concatenate([b, np.random.default_rng(seed).integers(0, M, extra)]))


@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_gemm_wide_tiles_ragged(gwx, out_dtype):
    """Large products run on 256 x 256 tiles (two M 128 x N 256 products per CTA sharing
    each B tile) once a full wave of them exists and K >= 1024; 4000 x 2600 gives 16 x 11
    = 176 such tiles on a 152-SM GB300, with ragged rows (4000 = 15 x 256 + 160), columns
    (2600 = 10 x 256 + 40) and K tail (1096 = 17 x 64 + 8).  Sampled rows at every 128-row
    boundary, all columns."""
    M, N, K = 4000, 2600, 1096
    a = workloads.random_bf16_bits(140, (M, K))
    b = workloads.random_bf16_bits(141, (N, K))
    C = gwx.gemm_bf16(_bf16(a), _bf16(b), out_dtype=out_dtype)
    gwx.device_status()
    rows = _rows(M, 142)
    got = C[torch.from_numpy(rows).cuda()].float().cpu().numpy().astype(np.float64)
    ref = gemm.gemm_nt(a[rows], b)
    tol = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(a[rows], b)
    if out_dtype == torch.bfloat16:
        tol = tol * (1.0 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= tol + 1e-30), (float(err.max()), float((err / (tol + 1e-30)).max()))


def test_dense_layer_wide_tiles(gwx):
    """Y = ReLU(X W^T + b) with a bfloat16 output on the 256 x 256 tiles (4096 x 2560 x 1024:
    16 x 10 tiles; GELU layers keep the 128 x 256 tiles): the fused epilogue on both
    accumulator halves of a tile."""
    M, N, K, act = 4096, 2560, 1024, 1
    x = workloads.random_bf16_bits(150, (M, K))
    w = workloads.random_bf16_bits(151, (N, K))
    bias = np.random.default_rng(152).normal(0.0, 0.5, N).astype(np.float32)
    Y = gwx.dense_bf16(_bf16(x), _bf16(w), torch.from_numpy(bias).cuda(), act=act, out_dtype=torch.bfloat16)
    gwx.device_status()
    rows = _rows(M, 153)
    got = Y[torch.from_numpy(rows).cuda()].float().cpu().numpy().astype(np.float64)
    ref = gemm.dense(x[rows], w, bias.astype(np.float64), act)
    z = gemm.dense(x[rows], w, bias.astype(np.float64), 0)
    tol_z = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(x[rows], w) + 2.0 ** -23 * np.abs(z)
    tol = tol_z * (1.0 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref)   # ReLU is 1-Lipschitz
    err = np.abs(got - ref)
    assert np.all(err <= tol + 1e-30), (float(err.max()), float((err / (tol + 1e-30)).max()))


def test_gemm_rejects_bad_arguments(gwx):
    a = torch.zeros((16, 12), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(gwx.GwxError):
        gwx.gemm_bf16(a, a)          # K = 12 is not a multiple of 8


@pytest.mark.parametrize("act", [0, 1, 2])
@pytest.mark.parametrize("M,N,K,out_dtype", [(256, 512, 128, torch.float32), (300, 260, 72, torch.float32),
                                             (128, 512, 256, torch.bfloat16)])
def test_dense_layer(gwx, act, M, N, K, out_dtype):
    """Y = act(X W^T + b): the sum's bound plus one FP32 rounding of the bias add; ReLU is
    1-Lipschitz, GELU's slope is below 1.13 and erfc adds a few FP32 ulps; a bfloat16
    output adds 2^-8 |Y|."""
    x = workloads.random_bf16_bits(100 + act, (M, K))
    w = workloads.random_bf16_bits(110 + act, (N, K))
    b = np.random.default_rng(120 + act).normal(0.0, 0.5, N).astype(np.float32)
    Y = gwx.dense_bf16(_bf16(x), _bf16(w), torch.from_numpy(b).cuda(), act=act, out_dtype=out_dtype)
    gwx.device_status()
    got = Y.float().cpu().numpy().astype(np.float64)
    ref = gemm.dense(x, w, b.astype(np.float64), act)
    z = gemm.dense(x, w, b.astype(np.float64), 0)
    tol_z = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(x, w) + 2.0 ** -23 * np.abs(z)
    tol = tol_z * (1.13 if act == 2 else 1.0) + (8 * 2.0 ** -24 * np.abs(ref) + 1e-37 if act == 2 else 0.0)
    if out_dtype == torch.bfloat16:
        tol = tol * (1.0 + 2.0 ** -8) + 2.0 ** -8 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= tol + 1e-30), (float(err.max()), float((err / (tol + 1e-30)).max()))


def test_gemm_autotune_keeps_results(gwx):
    """The autotuner picks a raster band among its candidates; the tuned product of that
    shape still matches the oracle."""
    M, N, K = 1024, 2048, 512
    a = workloads.random_bf16_bits(130, (M, K))
    b = workloads.random_bf16_bits(131, (N, K))
    A, B = _bf16(a), _bf16(b)
    out = torch.empty((M, N), dtype=torch.float32, device="cuda")
    g = gwx.gemm_autotune(A, B, out)
    assert g in (1, 2, 4, 8, 16, 32, 64)
    C = gwx.gemm_bf16(A, B)
    gwx.device_status()
    ref = gemm.gemm_nt(a, b)
    tol = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(a, b)
    assert np.all(np.abs(C.cpu().numpy().astype(np.float64) - ref) <= tol)


@pytest.mark.parametrize("act", [0, 1, 2])
@pytest.mark.parametrize("M,N,K", [(256, 512, 128), (200, 136, 72), (4000, 64, 328), (8192, 256, 256)])
def test_dense_backward(gwx, act, M, N, K):
    """dX, dW, db against the FP64 chain rule.  Bounds: dZ enters the products rounded to
    bfloat16 (2^-8 relative) after FP32 evaluation (2^-20), its activation derivative is
    taken at the FP32 pre-activation (|act''| <= 0.4 times that error), and each product
    adds its FP32 summation bound; dY is zeroed where ReLU's kink is within reach of
    the pre-activation error.  The last two shapes have few dW tiles and a long batch, so
    dW is computed in K slices (13 ragged slices of 5 and 3 K blocks; 32 slices of 4) and
    summed afterwards."""
    rng = np.random.default_rng(140 + act)
    x = workloads.random_bf16_bits(150 + act, (M, K), exp_lo=-3, exp_hi=0)
    w = workloads.random_bf16_bits(160 + act, (N, K), exp_lo=-3, exp_hi=0)
    b = rng.normal(0.0, 0.5, N).astype(np.float32)
    dy = rng.normal(0.0, 1.0, (M, N)).astype(np.float32)
    X, W = gemm.bf16_to_f64(x), gemm.bf16_to_f64(w)
    z = X @ W.T + b.astype(np.float64)[None, :]
    tol_z = 2.0 * K * 2.0 ** -24 * (np.abs(X) @ np.abs(W).T) + 2.0 ** -23 * np.abs(z)
    if act == 1:
        dy[np.abs(z) <= 4 * tol_z] = 0.0
    dX_ref, dW_ref, db_ref, dz = gemm.dense_backward(x, w, b.astype(np.float64), act, dy.astype(np.float64))
    dX, dW, db = gwx.dense_bf16_backward(_bf16(x), _bf16(w), torch.from_numpy(b).cuda(),
                                         torch.from_numpy(dy).cuda(), act=act)
    gwx.device_status()
    e_dz = (2.0 ** -8 + 2.0 ** -20) * np.abs(dz) + (0.4 if act == 2 else 0.0) * np.abs(dy) * tol_z
    tol_dX = e_dz @ np.abs(W) + 2.0 * N * 2.0 ** -24 * (np.abs(dz) @ np.abs(W))
    tol_dW = e_dz.T @ np.abs(X) + 2.0 * M * 2.0 ** -24 * (np.abs(dz).T @ np.abs(X))
    e_db = 2.0 ** -20 * np.abs(dz) + (0.4 if act == 2 else 0.0) * np.abs(dy) * tol_z
    tol_db = e_db.sum(axis=0) + 2.0 * 32 * 2.0 ** -24 * np.abs(dz).sum(axis=0)
    for got, ref, tol in ((dX, dX_ref, tol_dX), (dW, dW_ref, tol_dW), (db, db_ref, tol_db)):
        err = np.abs(got.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= tol * (1.0 + 1e-6) + 1e-30), (float(err.max()), float((err / (tol + 1e-30)).max()))


def test_bounded_wait_expiry_is_reported_and_the_context_survives(gwx):
    """A kernel waiting on an mbarrier that nothing arrives at gives up after its poll
    limit (the bounded-wait helper every tensor-core kernel uses), records the expiry,
    and returns: device_status reports GWX_ETIMEOUT once, then OK, and a product run
    afterwards is still correct."""
    gwx.device_status()                                   # start from a clean record
    gwx.selftest_bounded_wait(256)
    with pytest.raises(gwx.GwxError) as err:
        gwx.device_status()
    assert err.value.status == -5
    gwx.device_status()                                   # the record was cleared
    M, N, K = 256, 256, 128
    a = workloads.random_bf16_bits(170, (M, K))
    b = workloads.random_bf16_bits(171, (N, K))
    C = gwx.gemm_bf16(_bf16(a), _bf16(b))
    gwx.device_status()
    ref = gemm.gemm_nt(a, b)
    tol = 2.0 * K * 2.0 ** -24 * gemm.abs_product_sum(a, b)
    assert np.all(np.abs(C.cpu().numpy().astype(np.float64) - ref) <= tol)

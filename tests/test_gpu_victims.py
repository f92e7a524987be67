"""GPU parity of the victim kernels against the oracle (fp64 definitions)."""
import numpy as np
import pytest
import torch

import ifr_inputs as I
import oracle
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from tests.gpu_common import BF16_TOL, assert_fp32_close, bf16_bits, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ifr.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n", [1, 5, 4096 + 3, 1 << 22])
def test_triad(ctx, n):
    b = I.torch_uniform_pm1(0, n, "cuda")
    c = I.torch_uniform_pm1(0, n, "cuda", start=n)
    a = torch.empty(n, device="cuda")
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.5, repeats=2))
    assert t["status"] == 0 and t["t_end_ns"] > t["t_start_ns"] and t["repeats"] == 2
    ref = oracle.triad(I.np_uniform_pm1(0, np.arange(n)), I.np_uniform_pm1(0, np.arange(n, 2 * n)), 1.5)
    assert_fp32_close(a.cpu().numpy(), ref)


@pytest.mark.parametrize("rows,cols", [(1, 4), (7, 1000), (33, 4096), (5, 6000), (3, 12000), (16384, 4096)])
def test_layernorm(ctx, rows, cols):
    x = I.torch_uniform_pm1(4, rows * cols, "cuda").view(rows, cols)
    y = torch.empty_like(x)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    sel = np.unique(np.linspace(0, rows - 1, min(rows, 24)).astype(np.int64))
    xs = I.np_uniform_pm1(4, np.arange(rows * cols)).reshape(rows, cols)
    ref = oracle.layernorm_rows(xs, sel, 1e-5)
    assert_fp32_close(y.cpu().numpy()[sel], ref)


@pytest.mark.parametrize("rows,cols", [(1, 4), (9, 1000), (17, 8192), (4, 20000), (8192, 8192)])
def test_softmax(ctx, rows, cols):
    x = (I.torch_uniform_pm1(6, rows * cols, "cuda") * 4).view(rows, cols)
    y = torch.empty_like(x)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    sel = np.unique(np.linspace(0, rows - 1, min(rows, 16)).astype(np.int64))
    xs = (I.np_uniform_pm1(6, np.arange(rows * cols)) * 4).reshape(rows, cols)
    ref = oracle.softmax_rows(xs, sel)
    assert_fp32_close(y.cpu().numpy()[sel], ref)


# rows of up to 256 columns take the short-row kernel (several rows per warp)
@pytest.mark.parametrize("rows,cols", [(1, 8), (37, 1000), (300, 4096), (8192, 8192), (1000, 128), (77, 256),
                                       (333, 200), (5, 64), (100003, 8)])
def test_gemv(ctx, rows, cols):
    Ab = I.torch_normal_bf16(7, rows * cols, "cuda").view(rows, cols)
    xb = I.torch_normal_bf16(8, cols, "cuda")
    y = torch.empty(rows, device="cuda")
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=rows, k=cols))
    assert t["status"] == 0
    sel = np.unique(np.linspace(0, rows - 1, min(rows, 64)).astype(np.int64))
    A_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(7, np.arange(rows * cols))).reshape(rows, cols)
    x_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(8, np.arange(cols)))
    assert np.array_equal(bf16_bits(xb), x_np)
    ref = oracle.gemv_rows(A_np, x_np, sel)
    got = y.cpu().numpy()[sel].astype(np.float64)
    rms = np.sqrt(np.mean(ref * ref))
    assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms))
    assert np.linalg.norm(got - ref) <= BF16_TOL * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [1, 3, 1000003, 1 << 26])
def test_histogram_bit_exact(ctx, n):
    keys = I.torch_key256(2, n, "cuda")
    bins = torch.full((256,), 7, dtype=torch.int32, device="cuda")
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_HIST, keys, None, bins, n=n, repeats=3))
    assert t["status"] == 0
    want = oracle.histogram(I.np_key256(2, np.arange(n)))
    got = bins.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got, want)
    assert int(got.sum()) == n


def test_victim_bad_args(ctx):
    import ctypes as C

    L = A.load()
    x = torch.empty(64, device="cuda")
    t = A.ifr_timing()
    bad = [
        ifr.victim_cfg(A.IFR_V_TRIAD, x, x, x, n=0),
        ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, x, m=2, n=30),  # cols not a multiple of 4
        ifr.victim_cfg(A.IFR_V_GEMV, x, x, x, m=2, k=12),          # cols not a multiple of 8
        ifr.victim_cfg(A.IFR_V_TRIAD, x[1:], x, x, n=8),           # misaligned
        ifr.victim_cfg(17, x, x, x, n=8),
    ]
    for cfg in bad:
        assert L.ifr_victim_launch(ctx._h, C.byref(cfg), None, C.byref(t)) == A.IFR_ERR_ARG

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


# every row is compared, up to the full 16384 x 4096 (and 8192 x 8192 softmax)
# workloads; widths that are not a multiple of 4, and rows that do not start on a
# 16-byte boundary (offset 1: the base pointer is 4 bytes past an aligned one), take
# the column-by-column path
LN_SHAPES = [(1, 4), (7, 1000), (33, 4096), (5, 6000), (3, 12000), (16384, 4096), (37, 4095), (5, 13), (1, 1),
             (1000, 1001), (3, 32767), (9, 30)]


def _rows_input(seed, rows, cols, offset, scale=1.0):
    full = I.torch_uniform_pm1(seed, rows * cols + offset, "cuda") * scale
    x = full[offset:].view(rows, cols)
    ref = (I.np_uniform_pm1(seed, np.arange(rows * cols + offset)) * np.float32(scale))[offset:].reshape(rows, cols)
    return full, x, ref


@pytest.mark.parametrize("rows,cols", LN_SHAPES)
@pytest.mark.parametrize("offset", [0, 1])
def test_layernorm_every_row(ctx, rows, cols, offset):
    if offset and rows * cols > 1 << 22:
        pytest.skip("the unaligned path is covered on the smaller shapes")
    full, x, xs = _rows_input(4, rows, cols, offset)
    yfull = torch.empty(rows * cols + offset, device="cuda")
    y = yfull[offset:].view(rows, cols)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    ref = oracle.layernorm_rows(xs, np.arange(rows), 1e-5)
    assert_fp32_close(y.cpu().numpy(), ref)


def test_layernorm_constant_rows(ctx):
    """Rows of one repeated value have zero variance: the output is 0 (up to the
    rounding of the fp32 mean, far inside the tolerance's rms floor)."""
    rows, cols = 64, 4096
    xs = I.np_uniform_pm1(21, np.arange(rows * cols)).reshape(rows, cols).copy()
    consts = [0.0, 0.1, 3.0, -2.5, 1e-20, 7.25e3]
    for i, c in enumerate(consts):
        xs[5 * i] = np.float32(c)
    x = torch.tensor(xs, device="cuda")
    y = torch.empty_like(x)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    ref = oracle.layernorm_rows(xs, np.arange(rows), 1e-5)
    for i in range(len(consts)):
        assert np.all(ref[5 * i] == 0.0)
    assert_fp32_close(y.cpu().numpy(), ref)


SM_SHAPES = [(1, 4), (9, 1000), (17, 8192), (4, 20000), (8192, 8192), (37, 4095), (5, 13), (1, 1), (1000, 1001),
             (2, 32767)]


@pytest.mark.parametrize("rows,cols", SM_SHAPES)
@pytest.mark.parametrize("offset", [0, 1])
def test_softmax_every_row(ctx, rows, cols, offset):
    if offset and rows * cols > 1 << 22:
        pytest.skip("the unaligned path is covered on the smaller shapes")
    full, x, xs = _rows_input(6, rows, cols, offset, scale=4.0)
    yfull = torch.empty(rows * cols + offset, device="cuda")
    y = yfull[offset:].view(rows, cols)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    ref = oracle.softmax_rows(xs, np.arange(rows))
    assert_fp32_close(y.cpu().numpy(), ref)
    assert np.allclose(y.double().sum(dim=1).cpu().numpy(), 1.0, rtol=0, atol=1e-5)


@pytest.mark.parametrize("cols", [4096, 1001])
def test_softmax_wide_dynamic_range(ctx, cols):
    """Rows spanning +-80 (exp(x - max) down to e^-160, far below the fp32 range)
    and rows with one dominant entry."""
    rows = 256
    xs = (I.np_uniform_pm1(23, np.arange(rows * cols)) * np.float32(80.0)).reshape(rows, cols).copy()
    xs[7] = np.float32(-80.0)
    xs[7, 100] = np.float32(80.0)
    xs[11] = np.float32(0.0)
    x = torch.tensor(xs, device="cuda")
    y = torch.empty_like(x)
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, y, m=rows, n=cols))
    assert t["status"] == 0
    ref = oracle.softmax_rows(xs, np.arange(rows))
    got = y.cpu().numpy()
    assert_fp32_close(got, ref)
    assert got[7, 100] == 1.0 and np.all(np.delete(got[7], 100) == 0.0)
    assert np.allclose(got[11], 1.0 / cols, rtol=1e-6)


# variant 0: rows of up to 256 columns take the short-row kernel (several rows per
# warp).  Variant 1 (rows streamed into shared memory in 4 KiB segments, a ring of two
# per warp): rows shorter than a segment, rows that end in a short segment (1000, 2056
# and 4104 columns), more warps than rows, several rows per warp, the widest x (24576
# columns), and the full 8192 x 8192 matrix; three launches each.
@pytest.mark.parametrize("variant,rows,cols", [(0, 1, 8), (0, 37, 1000), (0, 300, 4096), (0, 8192, 8192),
                                               (0, 1000, 128), (0, 77, 256), (0, 333, 200), (0, 5, 64),
                                               (0, 100003, 8),
                                               (1, 1, 8), (1, 37, 1000), (1, 300, 4096), (1, 8192, 8192),
                                               (1, 5, 2056), (1, 2401, 4104), (1, 100003, 8), (1, 64, 24576)])
def test_gemv(ctx, variant, rows, cols):
    Ab = I.torch_normal_bf16(7, rows * cols, "cuda").view(rows, cols)
    xb = I.torch_normal_bf16(8, cols, "cuda")
    y = torch.full((rows,), float("nan"), device="cuda")
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=rows, k=cols, variant=variant,
                                         repeats=3 if variant else 1))
    assert t["status"] == 0
    sel = np.arange(rows)  # every row
    A_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(7, np.arange(rows * cols))).reshape(rows, cols)
    x_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(8, np.arange(cols)))
    assert np.array_equal(bf16_bits(xb), x_np)
    ref = oracle.gemv_rows(A_np, x_np, sel)
    got = y.cpu().numpy()[sel].astype(np.float64)
    rms = np.sqrt(np.mean(ref * ref))
    assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms))
    assert np.linalg.norm(got - ref) <= BF16_TOL * np.linalg.norm(ref)


def test_gemv_bulk_variant_is_solo_only(ctx):
    # the bulk-copy GEMV holds 64 KiB of rings plus x per block: solo launches
    # only; GEMV has no variant 2, and the other row victims have no variant 1
    Ab = I.torch_normal_bf16(7, 256 * 1024, "cuda").view(256, 1024)
    xb = I.torch_normal_bf16(8, 1024, "cuda")
    y = torch.empty(256, device="cuda")
    bulk = ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=256, k=1024, variant=1)
    plain = ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=256, k=1024, variant=0)
    fma = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=1, block=128, max_rounds=1)
    for call in (lambda: ctx.sweep([bulk], [], repeats=1), lambda: ctx.corun(bulk, plain),
                 lambda: ctx.corun(plain, bulk), lambda: ctx.colocate(fma, bulk)):
        with pytest.raises(ifr.IfrError) as e:
            call()
        assert e.value.status == A.IFR_ERR_ARG
    assert ctx.victim_launch(bulk)["status"] == 0
    x = torch.empty(256 * 256, device="cuda")
    for bad in (ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=256, k=1024, variant=2),
                ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, x, m=256, n=256, variant=1)):
        with pytest.raises(ifr.IfrError):
            ctx.victim_launch(bad)


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


class _Ptr:
    """A raw device address in the shape victim_cfg expects (something with data_ptr())."""

    def __init__(self, p):
        self.p = p

    def data_ptr(self):
        return self.p


def test_victim_bad_args(ctx):
    import ctypes as C

    L = A.load()
    x = torch.empty(64, device="cuda")
    t = A.ifr_timing()
    bad = [
        ifr.victim_cfg(A.IFR_V_TRIAD, x, x, x, n=0),
        ifr.victim_cfg(A.IFR_V_LAYERNORM, x, None, x, m=2, n=40000),  # wider than a row can be held
        ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, x, m=0, n=8),                # no rows
        ifr.victim_cfg(A.IFR_V_SOFTMAX, _Ptr(x.data_ptr() + 2), None, x, m=2, n=8),  # not 4-byte aligned
        ifr.victim_cfg(A.IFR_V_GEMV, x, x, x, m=2, k=12),          # cols not a multiple of 8
        ifr.victim_cfg(A.IFR_V_TRIAD, x[1:], x, x, n=8),           # misaligned
        ifr.victim_cfg(17, x, x, x, n=8),
    ]
    for cfg in bad:
        assert L.ifr_victim_launch(ctx._h, C.byref(cfg), None, C.byref(t)) == A.IFR_ERR_ARG

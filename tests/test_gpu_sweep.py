"""GPU sweep (plain and graph-batched) on the smallest configuration: FP32 triad
victim, HBM stream stressor at 0/25/50/100 % of SMs; the library's reduction must
equal the oracle's recomputation from the same raw timestamps."""
import math

import numpy as np
import pytest
import torch

import ifr_inputs as I
from oracle import reduction as R
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    ctx = ifr.Context(0)
    S = ctx.info["num_sms"]
    n = 1 << 22
    b = I.torch_uniform_pm1(0, n, "cuda")
    c = I.torch_uniform_pm1(0, n, "cuda", start=n)
    a = torch.empty(n, device="cuda")
    buf = I.torch_u32_as_i32(1, (256 << 20) // 4, "cuda")
    victims = [ifr.victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.5, repeats=8)]
    fr = [0.25, 0.5, 1.0]
    levels = [[ifr.stressor_cfg(A.IFR_S_HBM, sm_count=max(1, round(f * S)), blocks_per_sm=2, block=512,
                                working_set_bytes=256 << 20, buf=buf, seed=1) for f in fr]]
    yield ctx, victims, levels, (b, c, a, buf)
    ctx.close()


def _check(cells, n_levels, repeats):
    assert len(cells) == repeats * (1 + (n_levels + 1))
    d = ifr.cells_to_dicts(cells)
    valid = [x for x in d if x["valid"]]
    assert len(valid) >= 0.8 * len(d)
    for x in d:
        assert x["valid"] == (1 if R.cell_valid(x) else 0)
    got = ifr.ifr_sensitivity(cells, 0, 1, n_levels)
    want = R.sensitivity(d, 0, 1, n_levels)
    assert got["t0"] == want["t0"]
    for l in range(n_levels + 1):
        assert ifr.isclose_nan(got["slowdown"][0][l], want["slowdown"][0][l])
    assert got["monotone"] == want["monotone"]
    return got


def test_plain_sched_chain_too_short_is_measured_again(setup):
    """A scheduler chain far shorter than its victim (one launch of 4096 blocks beside
    a triad repeated 8 times) ends before the victim, the constant-interference rule's
    one failure.  The plain sweep measures that cell again with 4, 16 and 64 launches
    until the chain outlasts the victim, and the cell keeps the last measurement."""
    ctx, victims, _, _ = setup
    S = ctx.info["num_sms"]
    sb = 4096
    lv = [[ifr.stressor_cfg(A.IFR_S_SCHED, sm_count=S, sched_blocks=sb, sched_launches=1, sched_cycles=100,
                            seed=2)]]
    cells = ctx.sweep(victims, lv, repeats=1, batched=False)
    cc = [c for c in cells if c.stressor == 0 and c.level == 1]
    assert len(cc) == 1
    c = cc[0]
    launches = c.stress.blocks_launched // sb
    assert c.stress.blocks_launched == launches * sb and launches in (4, 16, 64), launches
    assert c.valid or launches == 64
    d = ifr.cells_to_dicts([c])[0]
    assert c.valid == (1 if R.cell_valid(d) else 0)
    if c.valid:
        assert c.stress.t_start_last_ns <= c.timing.t_start_ns and c.stress.t_end_first_ns >= c.timing.t_end_ns


def test_plain_sweep_config1(setup):
    ctx, victims, levels, _ = setup
    cells = ctx.sweep(victims, levels, repeats=3, batched=False)
    got = _check(cells, 3, 3)
    sd = got["slowdown"][0]
    # harness-only launch (level 0) does not slow the victim; the full HBM stressor does
    assert abs(sd[0] - 1.0) <= 3 * got["noise"] + 0.1
    assert sd[3] > 1.2
    # the slowdown is monotone in the HBM stressor's intensity (0, 25, 50, 100 % of
    # the SMs), within three times the solo noise
    assert got["monotone"] == [1], sd
    # every colocated cell recorded a running stressor
    for c in cells:
        if c.stressor >= 0 and c.level > 0:
            assert c.stress.blocks_active > 0 and c.stress.work > 0


def test_batched_sweep_config1(setup):
    ctx, victims, levels, _ = setup
    cells = ctx.sweep(victims, levels, repeats=3, batched=True)
    got = _check(cells, 3, 3)
    assert got["slowdown"][0][3] > 1.2
    assert got["monotone"] == [1], got["slowdown"][0]


def test_corun_two_kernels_valid_and_consistent(setup):
    """Kernel-with-kernel colocation: the chain covers the victim's window, the
    reduction of the raw timestamps equals the reported slowdown, and two
    HBM-bound kernels slow each other down (they share the DRAM bandwidth)."""
    ctx, victims, _levels, _ = setup
    n = 1 << 24
    b = torch.empty(n, device="cuda").uniform_(-1, 1)
    c = torch.empty(n, device="cuda").uniform_(-1, 1)
    a = torch.empty(n, device="cuda")
    # the co-runner leaves room on every SM (2 blocks of 256 threads) so both can be resident
    co = ifr.victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=0.5, repeats=1, grid=2 * ctx.info["num_sms"])
    r = ctx.corun(victims[0], co)
    assert r["valid"] == 1 and r["status"] == 0 and r["corunner_launches"] >= 2, r
    vs, vc = r["victim_solo"], r["victim_corun"]
    assert vc["t_start_ns"] >= r["corunner_corun"]["t_start_ns"]
    assert vc["t_end_ns"] <= r["corunner_corun"]["t_end_ns"]

    def meas(t):
        return dict(t_start=t["t_start_ns"], t_end=t["t_end_ns"], k=t["repeats"])

    # the library reduces the raw stamps itself; the oracle's definition on the same stamps
    want = R.corun_slowdown(meas(vs), meas(vc))
    assert math.isclose(r["victim_slowdown"], want, rel_tol=1e-12)
    want_c = R.corun_slowdown(meas(r["corunner_solo"]), meas(r["corunner_corun"]))
    assert math.isclose(r["corunner_slowdown"], want_c, rel_tol=1e-12)
    assert r["victim_slowdown"] > 1.1
    assert r["blocked"] == 0 and r["corunner_corun"]["t_start_ns"] <= r["victim_release_ns"] <= vc["t_start_ns"]



# ---------------------------------------------------------------- failure paths (bounded, no fault)
def test_unreachable_residency_is_reported_not_waited_for(setup):
    # two 1024-thread stream blocks per SM need 2 x 1024 x 40 registers: the second
    # cannot become resident beside the first.  Whichever bounded wait ends first
    # reports it: the stressor's head-of-line watch (50 ms without victim progress)
    # or the victim's residency wait (200 ms); the sweep goes on.
    import time
    ctx, victims, _levels, (b, c, a, buf) = setup
    S = ctx.info["num_sms"]
    lv = [[ifr.stressor_cfg(A.IFR_S_HBM, sm_count=S, blocks_per_sm=2, block=1024, working_set_bytes=256 << 20,
                            buf=buf, seed=1)]]
    t0 = time.perf_counter()
    cells = ctx.sweep(victims, lv, repeats=1, batched=False)
    assert time.perf_counter() - t0 < 1.5
    co = [x for x in cells if x.stressor == 0 and x.level == 1]
    assert co and not co[0].valid
    assert co[0].status in (A.IFR_ERR_NOT_RESIDENT, A.IFR_ERR_HOL)
    solo = [x for x in cells if x.stressor < 0]
    assert solo[0].valid  # the rest of the sweep is unaffected


def test_head_of_line_blocked_cell_is_recorded(setup):
    # a victim block that needs the whole register file cannot join a stressor block:
    # the stressor sees no victim progress, gives up with IFR_ERR_HOL, the victim runs
    # after it and the cell is recorded as invalid instead of stalling to the deadline
    import time
    ctx, _victims, _levels, (_b, _c, _a, buf) = setup
    S = ctx.info["num_sms"]
    x = I.torch_uniform_pm1(44, 256 * 16384, "cuda").view(256, 16384)
    y = torch.empty_like(x)
    v = ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, y, m=256, n=16384, repeats=1)
    assert ctx.victim_profile(v)["block"] == 1024
    lv = [[ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=1, block=128, ilp=4, seed=2)]]
    t0 = time.perf_counter()
    cells = ctx.sweep([v], lv, repeats=1, batched=False)
    assert time.perf_counter() - t0 < 1.5  # 50 ms head-of-line window, far below the 2 s deadline
    co = [c for c in cells if c.stressor == 0 and c.level == 1]
    assert co and not co[0].valid
    assert co[0].stress.status == A.IFR_ERR_HOL and co[0].status == A.IFR_ERR_HOL


def test_grouped_solo_sweep_ragged_row_victims(setup):
    """Grouped persistent victims on their own (no stressor): layernorm victims of one
    template with 1, 7 and 3001 rows, two of them of a width that is not a multiple of
    4 (a group of its own, the unaligned load path), softmax victims of one row and
    2049 rows, GEMV victims of 9 and 4097 rows, and GEMMs of both tile widths (a
    one-tile problem beside 2- to 150-tile ones; the 128-wide group holds more tiles
    than the GPU has SMs); three launches each.  Every output
    against the oracle, every victim on its own record, and a plan mode outside 0..2
    refused."""
    import oracle
    from tests.gpu_common import BF16_TOL, assert_fp32_close

    ctx = setup[0]
    specs = [("ln", 1, 1024), ("ln", 7, 1024), ("ln", 3001, 1024), ("ln", 5, 1023), ("ln", 333, 1023),
             ("sm", 1, 2048), ("sm", 2049, 2048), ("gemv", 9, 4096), ("gemv", 4097, 4096),
             ("gemm", 256, 256, 64), ("gemm", 384, 640, 192), ("gemm", 2048, 1024, 1024), ("gemm", 128, 128, 64),
             ("gemm", 1280, 1920, 256)]
    victims, keep = [], []
    for i, (k, rows, cols, *kk) in enumerate(specs):
        if k == "gemm":
            Ab = I.torch_normal_bf16(70 + i, rows * kk[0], "cuda").view(rows, kk[0])
            Bb = I.torch_normal_bf16(90 + i, cols * kk[0], "cuda").view(cols, kk[0])
            y = torch.full((rows, cols), float("nan"), device="cuda")
            victims.append(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Bb, y, m=rows, n=cols, k=kk[0], repeats=3))
            inputs = (Ab, Bb)
        elif k == "gemv":
            Ab = I.torch_normal_bf16(70 + i, rows * cols, "cuda").view(rows, cols)
            xb = I.torch_normal_bf16(90 + i, cols, "cuda")
            y = torch.full((rows,), float("nan"), device="cuda")
            victims.append(ifr.victim_cfg(A.IFR_V_GEMV, Ab, xb, y, m=rows, k=cols, repeats=3))
            inputs = (Ab, xb)
        else:
            x = I.torch_uniform_pm1(70 + i, rows * cols, "cuda").view(rows, cols)
            y = torch.full_like(x, float("nan"))
            kind = A.IFR_V_LAYERNORM if k == "ln" else A.IFR_V_SOFTMAX
            victims.append(ifr.victim_cfg(kind, x, None, y, m=rows, n=cols, repeats=3))
            inputs = (x,)
        keep.append((k, rows, cols, y, inputs))  # the configs hold raw pointers: keep the tensors
    cells = ctx.sweep(victims, [], repeats=1, batched=True, grouped=True)
    assert len(cells) == len(victims)
    for c in cells:
        assert c.valid and c.timing.t_end_ns > c.timing.t_start_ns and c.timing.blocks > 0
    for i, (k, rows, cols, y, inputs) in enumerate(keep):
        if k == "gemm":
            ref = inputs[0].double().cpu() @ inputs[1].double().cpu().T
            got = y.double().cpu()
            rms = float(ref.pow(2).mean().sqrt())
            assert bool(((got - ref).abs() <= BF16_TOL * torch.maximum(ref.abs(), torch.tensor(rms))).all()), i
        elif k == "gemv":
            A_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(70 + i, np.arange(rows * cols))).reshape(rows, cols)
            x_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(90 + i, np.arange(cols)))
            ref = oracle.gemv_rows(A_np, x_np, np.arange(rows))
            got = y.cpu().numpy().astype(np.float64)
            rms = np.sqrt(np.mean(ref * ref))
            assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms)), i
        else:
            xs = I.np_uniform_pm1(70 + i, np.arange(rows * cols)).reshape(rows, cols)
            ref = oracle.layernorm_rows(xs, np.arange(rows), 1e-5) if k == "ln" else oracle.softmax_rows(
                xs, np.arange(rows))
            assert_fp32_close(y.cpu().numpy(), ref)
    import ctypes as C

    plan = A.ifr_sweep_plan(1, (A.ifr_victim_cfg * 1)(victims[0]), 0, 0, (A.ifr_stressor_cfg * 1)(), 1, 3)
    out = (A.ifr_cell_result * 4)()
    n = C.c_size_t(0)
    assert A.load().ifr_sweep(ctx._h, C.byref(plan), out, 4, C.byref(n)) == A.IFR_ERR_ARG

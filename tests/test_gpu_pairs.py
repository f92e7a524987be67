"""FP64 stressor parity (Sec. 4.4.3), explicit SM masks (the disjoint partitions of
Sec. 4.3's inter-SM runs) and ifr_stressor_pair (the kernel-against-kernel runs of
Sec. 3, Sec. 4.3 and Table 3), through the C ABI."""
import pytest

import oracle
from oracle import reduction as R
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300.experiments import with_mask
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

FP64_WORK = 1024  # multiplies per thread per round


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ifr.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("ilp", [1, 2, 4, 8])
def test_fp64_block_checksums_match_oracle(ctx, ilp):
    block, sms, rounds, seed = 64, 6, 2, 9 + ilp
    cfg = ifr.stressor_cfg(A.IFR_S_FP64, sm_count=sms, blocks_per_sm=1, block=block, ilp=ilp, seed=seed,
                           max_rounds=rounds)
    res, logs = ctx.run_stressor(cfg)
    assert res["status"] == A.IFR_OK
    assert len(logs) == sms
    steps = FP64_WORK // ilp
    for L in logs:
        assert L["work"] == rounds * steps
        assert (L["checksum"], L["checksum2"]) == oracle.fp64_block(seed, L["index"], block, ilp, steps, rounds)


def test_fp64_ragged_block_and_many_rounds(ctx):
    # a block size that is not a power of two, and more rounds than the fold period
    block, rounds, seed = 96, 5, 77
    cfg = ifr.stressor_cfg(A.IFR_S_FP64, sm_count=3, blocks_per_sm=2, block=block, ilp=4, seed=seed,
                           max_rounds=rounds)
    res, logs = ctx.run_stressor(cfg)
    assert res["status"] == A.IFR_OK and len(logs) == 6
    for L in logs:
        assert (L["checksum"], L["checksum2"]) == oracle.fp64_block(seed, L["index"], block, 4, FP64_WORK // 4, rounds)


def test_explicit_mask_confines_blocks(ctx):
    S = ctx.info["num_sms"]
    ids = [0, 3, 17, S - 1]
    cfg = with_mask(ifr.stressor_cfg(A.IFR_S_FMA, blocks_per_sm=2, block=128, ilp=4, seed=1, max_rounds=2), ids)
    res, logs = ctx.run_stressor(cfg)
    assert res["status"] == A.IFR_OK
    assert {L["smid"] for L in logs} == set(ids)
    assert res["sms_used"] == len(ids) and res["blocks_active"] == 2 * len(ids)


def test_explicit_mask_rejects_inconsistent_masks(ctx):
    S = ctx.info["num_sms"]
    cfg = with_mask(ifr.stressor_cfg(A.IFR_S_FMA, block=128, max_rounds=1), [1, 2])
    cfg.sm_count = 3  # does not match the two bits set
    with pytest.raises(ifr.IfrError) as e:
        ctx.stressor_launch(cfg)
    assert e.value.status == A.IFR_ERR_ARG
    if S < A.IFR_MAX_SMS:
        beyond = with_mask(ifr.stressor_cfg(A.IFR_S_FMA, block=128, max_rounds=1), [S])  # no such SM
        with pytest.raises(ifr.IfrError) as e:
            ctx.stressor_launch(beyond)
        assert e.value.status == A.IFR_ERR_ARG
    green = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=4, block=128, max_rounds=1, mask_mode=1)
    with pytest.raises(ifr.IfrError) as e:
        ctx.stressor_launch(green)
    assert e.value.status == A.IFR_ERR_UNSUPPORTED


def test_pair_on_disjoint_halves(ctx):
    S = ctx.info["num_sms"]
    h = S // 2
    a = with_mask(ifr.stressor_cfg(A.IFR_S_FMA, blocks_per_sm=1, block=128, ilp=4, seed=1, max_rounds=16), range(h))
    b = with_mask(ifr.stressor_cfg(A.IFR_S_FMA, blocks_per_sm=1, block=128, ilp=4, seed=2, max_rounds=16),
                  range(h, S))
    r = ctx.stressor_pair(a, b)
    assert r["status"] == A.IFR_OK and r["overlapped"] == 1
    # the same fixed work gives the same checksums alone and together
    assert r["co_a"]["checksum"] == r["solo_a"]["checksum"]
    assert r["co_b"]["checksum"] == r["solo_b"]["checksum"]
    assert {r["co_a"]["sms_used"], r["co_b"]["sms_used"]} == {h, S - h}
    # arithmetic-only kernels on disjoint SMs do not interfere beyond noise
    assert 0.8 < r["co_a_ns"] / r["solo_a_ns"] < 1.25
    assert r["seq_ns"] == pytest.approx(r["solo_a_ns"] + r["solo_b_ns"])
    assert r["col_ns"] >= max(r["co_a_ns"], r["co_b_ns"]) - 1.0
    # two halves at once take about as long as one: speedup near 2
    assert 1.5 < r["seq_ns"] / r["col_ns"] < 2.5
    # spans and the seq/col speedup follow the oracle's reading of Table 3 on the raw stamps
    for k in ("solo_a", "solo_b", "co_a", "co_b"):
        assert r[k + "_ns"] == r[k]["t_end_ns"] - r[k]["t_start_ns"]
    sp = R.corun_speedup(r["solo_a_ns"], r["solo_b_ns"], r["co_a"]["t_start_ns"], r["co_a"]["t_end_ns"],
                         r["co_b"]["t_start_ns"], r["co_b"]["t_end_ns"])
    assert r["seq_ns"] / r["col_ns"] == pytest.approx(sp, rel=1e-12)


def test_pair_same_sms_fp64_speedup_bounded(ctx):
    S = ctx.info["num_sms"]
    a = ifr.stressor_cfg(A.IFR_S_FP64, sm_count=S, blocks_per_sm=1, block=128, ilp=4, seed=3, max_rounds=2)
    b = ifr.stressor_cfg(A.IFR_S_FP64, sm_count=S, blocks_per_sm=1, block=128, ilp=4, seed=4, max_rounds=2)
    r = ctx.stressor_pair(a, b)
    assert r["status"] == A.IFR_OK and r["overlapped"] == 1
    assert r["co_a"]["checksum"] == r["solo_a"]["checksum"]
    # two identical kernels sharing every SM: no faster than twice, no slower than back to back
    assert 0.8 < r["seq_ns"] / r["col_ns"] < 2.2


def test_pair_rejects_unbounded_or_scheduler_kinds(ctx):
    S = ctx.info["num_sms"]
    bounded = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, block=128, max_rounds=1)
    unbounded = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, block=128)
    sched = ifr.stressor_cfg(A.IFR_S_SCHED, sm_count=S, max_rounds=1)
    for a, b in ((bounded, unbounded), (sched, bounded)):
        with pytest.raises(ifr.IfrError) as e:
            ctx.stressor_pair(a, b)
        assert e.value.status == A.IFR_ERR_ARG


# ---------------------------------------------------------------- sleep kernel and ifr_colocate (Sec. 4.2)
def _sleep(S, rounds, period_ns, smem=0):
    return ifr.stressor_cfg(A.IFR_S_SLEEP, sm_count=S, blocks_per_sm=1, block=128, period_ns=period_ns,
                            max_rounds=rounds, working_set_bytes=smem, seed=1)


def test_sleep_stressor_rounds_and_span(ctx):
    S = ctx.info["num_sms"]
    res, logs = ctx.run_stressor(_sleep(S, 10, 20000))
    assert res["status"] == A.IFR_OK and res["sms_used"] == S
    assert all(L["rounds"] == 10 and L["work"] == 10 for L in logs)
    assert all(L["t_end_ns"] - L["t_start_ns"] >= 10 * 20000 for L in logs)


def test_colocate_small_victim_runs_beside_sleep(ctx):
    import torch
    import ifr_inputs as I
    S = ctx.info["num_sms"]
    A_ = I.torch_normal_bf16(41, 1024 * 4096, "cuda").view(1024, 4096)
    x = I.torch_normal_bf16(42, 4096, "cuda")
    y = torch.empty(1024, device="cuda")
    v = ifr.victim_cfg(A.IFR_V_GEMV, A_, x, y, m=1024, k=4096, repeats=4)
    r = ctx.colocate(_sleep(S, 20, 100000), v)  # 2 ms of sleep
    assert r["status"] == A.IFR_OK and r["blocked"] == 0
    assert r["victim_co_ns"] < 0.5 * r["stress_co_ns"]  # done long before the sleep kernel ends


def test_colocate_register_file_victim_waits_for_sleep(ctx):
    import torch
    import ifr_inputs as I
    S = ctx.info["num_sms"]
    x = I.torch_uniform_pm1(43, 512 * 16384, "cuda").view(512, 16384)
    y = torch.empty_like(x)
    v = ifr.victim_cfg(A.IFR_V_SOFTMAX, x, None, y, m=512, n=16384, repeats=1)
    vp, sp = ctx.victim_profile(v), ctx.stressor_profile(_sleep(S, 20, 100000))
    regs = lambda p: p["block"] * (-(-p["regs_per_thread"] // 8) * 8)
    # premise (Sec. 2.1): one victim block and one sleep block exceed the register file
    assert regs(vp) + regs(sp) > ctx.info["regs_per_sm"]
    r = ctx.colocate(_sleep(S, 20, 100000), v)
    assert r["status"] == A.IFR_OK and r["blocked"] == 1
    assert r["victim_co"]["t_start_ns"] >= r["stress_co"]["t_end_first_ns"]
    # latency from the victim's release covers the rest of the 2 ms of sleep
    assert r["stress_co_ns"] > 1.5e6 and r["victim_co_ns"] > 0.9 * r["stress_co_ns"]


# ---------------------------------------------------------------- green-context partitions (Sec. 4.1)
def test_partition_confines_victims_and_stressors(ctx):
    import torch
    import ifr_inputs as I
    S = ctx.info["num_sms"]
    info = ctx.partition(S // 2, fine=True)
    try:
        nv, ns = info["victim_sms"], info["stressor_sms"]
        assert nv >= S // 2 and nv + ns <= S and ns > 0
        # a stressor on every SM of its partition (mask_mode 1) stays there
        cfg = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=ns, blocks_per_sm=1, block=128, ilp=4, seed=5, max_rounds=4,
                               mask_mode=1)
        res, logs = ctx.run_stressor(cfg)
        assert res["status"] == A.IFR_OK and res["sms_used"] == ns
        stress_sms = {L["smid"] for L in logs}
        # a victim with more blocks than SMs touches only the victim partition's SMs
        n = 1 << 22
        b = I.torch_uniform_pm1(0, n, "cuda")
        c = I.torch_uniform_pm1(0, n, "cuda", start=n)
        a = torch.empty(n, device="cuda")
        v = ifr.victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.5, repeats=2)
        t = ctx.victim_launch(v)
        assert t["status"] == A.IFR_OK and 0 < t["sms_touched"] <= nv
        # a sweep cell: victim beside the stressor on disjoint SMs, both valid
        lv = [[ifr.stressor_cfg(A.IFR_S_FMA, sm_count=ns, blocks_per_sm=1, block=128, ilp=4, seed=5, mask_mode=1)]]
        cells = ctx.sweep([v], lv, repeats=1, batched=False)
        co = [x for x in cells if x.stressor == 0 and x.level == 1]
        assert co and all(x.valid for x in co)
        assert co[0].stress.sms_used == ns and co[0].timing.sms_touched <= nv
        assert len(stress_sms) == ns
    finally:
        ctx.partition_release()
    # released: a full-SM stressor reaches every SM again
    res, _ = ctx.run_stressor(ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=1, block=128, max_rounds=1))
    assert res["sms_used"] == S


def test_partition_isolates_sm_private_stressors(ctx):
    """Harness invariant (Sec. 4.1, Sec. 4.3): stressors of resources private to an SM
    (the FP32 pipe, the tensor pipe, shared memory) confined to the other green-context
    partition leave an HBM-bound victim's latency within its solo noise.  The 6 % floor
    allows for the SM clock, which both partitions share under the power cap: a
    tensor-pipe stressor at full power on the other half of the SMs slowed the triad
    (on 74 SMs, partly clock-bound) by 5.1 % on one B300, with a solo noise of 1.2 %."""
    import torch
    import ifr_inputs as I
    S = ctx.info["num_sms"]
    n = 1 << 24  # three 64 MiB vectors: more than L2, so the triad streams from HBM
    b = I.torch_uniform_pm1(0, n, "cuda")
    c = I.torch_uniform_pm1(0, n, "cuda", start=n)
    a = torch.empty(n, device="cuda")
    kinds = [A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_32W]
    info = ctx.partition(S // 2)
    try:
        v = ifr.victim_cfg(A.IFR_V_TRIAD, b, c, a, n=n, scalar=1.5, repeats=4)
        lv = [[ifr.stressor_cfg(k, sm_count=info["stressor_sms"], seed=3, mask_mode=1)] for k in kinds]
        cells = ctx.sweep([v], lv, repeats=5, batched=False)
    finally:
        ctx.partition_release()
    red = R.sensitivity(ifr.cells_to_dicts(cells), 0, len(kinds), 1)
    for r, k in enumerate(kinds):
        sd = red["slowdown"][r][1]
        assert sd <= 1.0 + max(3.0 * red["noise"], 0.06), (A.STRESSOR_NAMES[k], sd, red["noise"])


def test_partition_argument_errors(ctx):
    S = ctx.info["num_sms"]
    ctx.partition_release()  # no split active: a no-op
    for bad in (0, S, -1):
        with pytest.raises(ifr.IfrError) as e:
            ctx.partition(bad)
        assert e.value.status == A.IFR_ERR_ARG
    info = ctx.partition(S // 4)
    try:
        with pytest.raises(ifr.IfrError) as e:  # one split at a time
            ctx.partition(S // 2)
        assert e.value.status == A.IFR_ERR_ARG
        too_many = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, block=128, max_rounds=1, mask_mode=1)
        with pytest.raises(ifr.IfrError) as e:  # more SMs than either partition has
            ctx.stressor_launch(too_many)
        assert e.value.status == A.IFR_ERR_ARG
        assert info["victim_sms"] >= S // 4 and info["victim_sms"] + info["stressor_sms"] <= S
    finally:
        ctx.partition_release()

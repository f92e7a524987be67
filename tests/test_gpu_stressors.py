"""GPU parity of the stressor kernels against the oracle's checksums."""
import time

import numpy as np
import pytest
import torch

import ifr_inputs as I
import oracle
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import peaks as P
from tests.gpu_common import need_gpu, spread_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ifr.Context(0)
    yield c
    c.close()


def _stream_check(ctx, kind, nbytes, block, bps, sm_count, rounds=0, stop_after_s=None, sample=None, staging=0):
    n = nbytes // 4
    buf = I.torch_u32_as_i32(1, n, "cuda")
    cfg = ifr.stressor_cfg(kind, sm_count=sm_count, blocks_per_sm=bps, block=block, working_set_bytes=nbytes,
                           buf=buf, max_rounds=rounds, seed=0, staging=staging)
    fold = oracle.FOLD_BULK if staging == 1 else oracle.FOLD_LOADS
    h = ctx.stressor_launch(cfg)
    if stop_after_s is not None:
        time.sleep(stop_after_s)
        ctx.stressor_stop(h)
    r = ctx.stressor_wait(h, 20000)
    logs = ctx.stressor_block_logs(h)
    ctx.stressor_release(h)
    assert r["status"] == 0
    planned = sm_count * bps
    assert r["planned_active"] == planned
    assert len(logs) == r["blocks_active"] <= planned
    hbuf = buf.cpu().numpy().view(np.uint32)
    chunk = block * 16
    mask = spread_mask(ctx.info["num_sms"], sm_count)
    assert {L["smid"] for L in logs} <= mask
    per_sm = {}
    for L in logs:
        per_sm[L["smid"]] = per_sm.get(L["smid"], 0) + 1
    assert max(per_sm.values()) <= bps
    chk = logs if sample is None else logs[:sample]
    for L in chk:
        want = oracle.stream_block_checksum(hbuf, chunk, planned, L["index"], L["work"], fold)
        assert L["checksum"] == want, L
        if rounds:
            n_chunks = n // chunk
            exp = P.STREAM_CHUNKS_PER_ROUND * rounds if L["index"] < n_chunks else 0
            assert L["work"] == exp
    xor = 0
    for L in logs:
        xor ^= L["checksum"]
    assert r["checksum"] == xor
    return r, logs


# staging 0: loads into registers (the first word of every 16-byte group); 1: TMA bulk
# copies into a shared-memory ring
@pytest.mark.parametrize("staging", [0, 1])
def test_hbm_stressor_fixed_rounds_all_sms(ctx, staging):
    S = ctx.info["num_sms"]
    _stream_check(ctx, A.IFR_S_HBM, 64 << 20, 512, 2, S, rounds=3, staging=staging)


@pytest.mark.parametrize("staging", [0, 1])
def test_l2_stressor_subset_ragged(ctx, staging):
    # 37 SMs, 1 block each, 256-thread blocks; the chunk count is not a multiple of the stride;
    # 11 passes, so the bulk path folds every quarter
    _stream_check(ctx, A.IFR_S_L2, (16384 * 211), 256, 1, 37, rounds=30, staging=staging)


@pytest.mark.parametrize("staging", [0, 1])
def test_stream_stressor_more_blocks_than_chunks(ctx, staging):
    S = ctx.info["num_sms"]
    # 40 chunks of 32 KiB for 2*S blocks: most blocks have no chunk and read nothing
    r, logs = _stream_check(ctx, A.IFR_S_HBM, 40 * 32768, 512, 2, S, rounds=2, staging=staging)
    assert sum(1 for L in logs if L["work"] > 0) == 40


@pytest.mark.parametrize("staging", [0, 1])
def test_stream_stressor_stop_flag_arbitrary_counts(ctx, staging):
    # stopped from the host after about 2 ms: every block's arbitrary chunk count is
    # checked against the oracle (a block that skipped work would show)
    S = ctx.info["num_sms"]
    r, logs = _stream_check(ctx, A.IFR_S_HBM, 256 << 20, 512, 2, S, rounds=0, stop_after_s=0.002, staging=staging)
    assert r["work"] > 0 and all(L["status"] == 0 for L in logs)
    assert len(logs) == 2 * S and len({L["work"] for L in logs}) > 1


# every instantiation of the register-load kernel (block sizes fixed at compile time,
# and 384 and 1024 read at run time): 13 SMs x 2 blocks over 291 chunks, so each block cycles
# through 11 or 12 chunks; 5 rounds of 8 chunks run whole rounds from one pointer and
# rounds that wrap to the block's first chunk part-way, over 3 or 4 passes
@pytest.mark.parametrize("block", [128, 256, 384, 512, 1024])
def test_stream_stressor_block_sizes_wrap_inside_rounds(ctx, block):
    n_chunks = 13 * 2 * 11 + 5
    _stream_check(ctx, A.IFR_S_HBM, n_chunks * block * 64, block, 2, 13, rounds=5)


def test_stream_stressor_staging_needs_a_stream_kind(ctx):
    import ctypes as C

    L = A.load()
    h = C.c_int()
    for cfg in (ifr.stressor_cfg(A.IFR_S_FMA, sm_count=1, staging=1),
                ifr.stressor_cfg(A.IFR_S_HBM, sm_count=1, staging=2, block=512, working_set_bytes=1 << 20,
                                 buf=torch.empty(1 << 18, dtype=torch.int32, device="cuda"))):
        assert L.ifr_stressor_launch(ctx._h, C.byref(cfg), None, C.byref(h)) == A.IFR_ERR_ARG


def test_stressor_deadline_returns_timeout_status(ctx):
    # no stop request and no round limit: the device deadline ends the run with a status
    n = 8 << 20
    buf = I.torch_u32_as_i32(1, n // 4, "cuda")
    cfg = ifr.stressor_cfg(A.IFR_S_HBM, sm_count=4, blocks_per_sm=1, block=512, working_set_bytes=n, buf=buf,
                           deadline_ns=3_000_000)
    h = ctx.stressor_launch(cfg)
    r = ctx.stressor_wait(h, 5000)
    ctx.stressor_release(h)
    assert r["status"] == A.IFR_ERR_TIMEOUT
    assert r["blocks_active"] == 4


@pytest.mark.parametrize("ilp", [1, 4, 8])
def test_fma_stressor_matches_oracle(ctx, ilp):
    S = ctx.info["num_sms"]
    cfg = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=2, block=128, ilp=ilp, max_rounds=2, seed=7)
    r, logs = ctx.run_stressor(cfg, 20000)
    assert r["status"] == 0 and len(logs) == 2 * S
    for L in logs[:: max(1, len(logs) // 5)]:
        steps = 16384 // ilp  # steps per chain per round
        r0, fin = oracle.fma_block(7, L["index"], 128, ilp, steps, 2)
        assert (L["checksum"], L["checksum2"]) == (r0, fin)
        assert L["rounds"] == 2 and L["work"] == 2 * steps


@pytest.mark.parametrize("kind,ways", [(A.IFR_S_SMEM_CF, 0), (A.IFR_S_SMEM_32W, 0), (A.IFR_S_SMEM_CF, 8)])
def test_smem_stressor_matches_oracle(ctx, kind, ways):
    S = ctx.info["num_sms"]
    cfg = ifr.stressor_cfg(kind, sm_count=S // 2, blocks_per_sm=2, block=256, smem_ways=ways, max_rounds=3, seed=5)
    r, logs = ctx.run_stressor(cfg, 20000)
    assert r["status"] == 0 and len(logs) == 2 * (S // 2)
    for L in logs:
        w = ways or (1 if kind == A.IFR_S_SMEM_CF else 32)
        passes = max(1, 32 // w)  # passes over the warp array per round
        assert L["checksum"] == oracle.smem_block(5, L["index"], 8, 3, passes)
        assert L["work"] == 3 * passes * 32
    assert {L["smid"] for L in logs} <= spread_mask(S, S // 2)


def test_sched_stressor_checksum(ctx):
    S = ctx.info["num_sms"]
    cfg = ifr.stressor_cfg(A.IFR_S_SCHED, sm_count=S, sched_blocks=5000, sched_launches=3, sched_cycles=100,
                           seed=0xABCDEF)
    r, _ = ctx.run_stressor(cfg, 20000)
    assert r["status"] == 0
    assert r["checksum"] == oracle.sched_checksum(0xABCDEF, 15000, 16)
    assert r["work"] == 15000 and r["blocks_launched"] == 15000


def test_sched_zero_sms_does_no_work_but_checksums(ctx):
    cfg = ifr.stressor_cfg(A.IFR_S_SCHED, sm_count=0, sched_blocks=2000, sched_launches=2, seed=3)
    r, _ = ctx.run_stressor(cfg, 20000)
    assert r["work"] == 0
    assert r["checksum"] == oracle.sched_checksum(3, 4000, 16)


def test_bad_stressor_args_rejected_on_host(ctx):
    L = A.load()
    import ctypes as C

    h = C.c_int()
    bad = [
        ifr.stressor_cfg(99),
        ifr.stressor_cfg(A.IFR_S_FMA, sm_count=ctx.info["num_sms"] + 1),
        ifr.stressor_cfg(A.IFR_S_FMA, ilp=3),
        ifr.stressor_cfg(A.IFR_S_HBM, sm_count=1, working_set_bytes=1000, buf=torch.empty(1000, device="cuda")),
        ifr.stressor_cfg(A.IFR_S_SMEM_CF, smem_ways=3),
        ifr.stressor_cfg(A.IFR_S_FMA, block=33),
    ]
    for cfg in bad:
        assert L.ifr_stressor_launch(ctx._h, C.byref(cfg), None, C.byref(h)) == A.IFR_ERR_ARG

"""Static co-residence budget: at full intensity every stressor leaves room on each SM
for one block of every benchmark victim (Sec. 2.1: registers, threads, shared memory
and block slots decide which blocks share an SM; TMEM is the fifth such resource on
this part).  Registers and warp slots are split over the SM's four sub-partitions
(a 16 K-register file and 16 warp slots each) and a block's warps are spread over
them, so a 6-warp victim puts two warps on some sub-partition: the budget is checked
per sub-partition, which is the binding constraint beside a stressor that fills every
sub-partition evenly.  A victim block that does not fit waits for the stressor to finish, the
cell is head-of-line blocked and the sweep loses it, so this is checked from the
kernels' own attributes rather than discovered as invalid cells."""
import pytest

import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import workloads
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

RESERVED_SMEM_PER_BLOCK = 1024  # bytes the runtime keeps per resident block
REG_ALLOC_UNIT = 256            # registers are granted per warp in units of 256
TMEM_COLS = 512
SUBPARTITIONS = 4


def _ceil(a, b):
    return -(-a // b)


def _usage(p, blocks):
    """Per-SM and worst-sub-partition use of `blocks` blocks of the profiled kernel."""
    warps = _ceil(p["block"], 32) * blocks
    regs_warp = _ceil(p["regs_per_thread"] * 32, REG_ALLOC_UNIT) * REG_ALLOC_UNIT
    part = _ceil(warps, SUBPARTITIONS)
    return {
        "regs_subpartition": part * regs_warp,
        "warps_subpartition": part,
        "threads": p["block"] * blocks,
        "smem": (p["static_smem"] + p["dynamic_smem"] + RESERVED_SMEM_PER_BLOCK) * blocks,
        "tmem": p["tmem_cols"] * blocks,
        "blocks": blocks,
    }


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    ctx = ifr.Context(0)
    wl = workloads.config2(ctx.info["num_sms"], hbm_bytes=1 << 28)
    yield ctx, wl
    ctx.close()


def test_full_intensity_stressors_leave_room_for_each_victim(setup):
    ctx, wl = setup
    info = ctx.info
    limit = {"regs_subpartition": info["regs_per_sm"] // SUBPARTITIONS,
             "warps_subpartition": info["max_threads_per_sm"] // 32 // SUBPARTITIONS,
             "threads": info["max_threads_per_sm"], "smem": info["smem_per_sm"], "tmem": TMEM_COLS,
             "blocks": info["max_blocks_per_sm"]}
    victims = [(A.VICTIM_NAMES[k], _usage(ctx.victim_profile(v), 1)) for v, k in zip(wl.victims, wl.victim_kinds)]
    bad = []
    for row in wl.levels:
        cfg = row[-1]
        if cfg.kind == A.IFR_S_SCHED:
            continue  # short blocks that retire by themselves; no resident set to share
        sp = ctx.stressor_profile(cfg)
        assert sp["sm_count"] == info["num_sms"]
        sr = _usage(sp, sp["blocks_per_sm"])
        for name, vr in victims:
            for res, cap in limit.items():
                used = sr[res] + vr[res]
                if used > cap:
                    bad.append("%s + %s: %s %d > %d" % (A.STRESSOR_NAMES[cfg.kind], name, res, used, cap))
    assert not bad, bad

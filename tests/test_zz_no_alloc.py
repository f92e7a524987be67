"""GPU test of the allocation-free stream-stressor entry point.

Callers that cannot call cudaMalloc (latency-critical loops that must not block
on the allocator, hosts with a fixed device-memory budget and no library
context) use
ifr_stream_stressor_noalloc, whose control state lives in a file-scope device
array.  Its per-block results must equal those of the context-based entry point
(ifr_stressor_launch + ifr_stressor_wait + ifr_stressor_block_logs) for the same
fixed-work configuration, on two calls in a row (the second call must clear what
the first left in the shared array); every block's checksum must also equal the
oracle's, so that a fault shared by both entry points is still caught; and calls
after the first must leave the device's free memory unchanged.  This file is
collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import ifr_inputs as I
import oracle
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A

pytestmark = pytest.mark.gpu


def _noalloc_logs(L, kind, buf, nbytes, sm_count, bps, block, rounds, stream):
    cap = sm_count * bps
    raw = torch.zeros(cap * C.sizeof(A.ifr_block_log), dtype=torch.uint8, device="cuda")
    st = L.ifr_stream_stressor_noalloc(kind, C.c_void_p(buf.data_ptr()), nbytes, sm_count, bps, block, rounds, 0,
                                       C.c_void_p(stream.cuda_stream), C.c_void_p(raw.data_ptr()), cap)
    A.check(st, "ifr_stream_stressor_noalloc")
    stream.synchronize()
    host = raw.cpu().numpy().tobytes()
    logs = (A.ifr_block_log * cap).from_buffer_copy(host)
    return {lg.index: (lg.checksum, lg.work, lg.rounds, lg.status) for lg in logs if lg.index >= 0}


def test_noalloc_matches_context_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = A.load()
    kind, nbytes, block, bps, rounds = A.IFR_S_HBM, 48 << 20, 512, 2, 5
    buf = I.torch_u32_as_i32(1, nbytes // 4, "cuda")
    with ifr.Context(0) as ctx:
        S = ctx.info["num_sms"]
        sm_count = S // 2 + 3
        cfg = ifr.stressor_cfg(kind, sm_count=sm_count, blocks_per_sm=bps, block=block, working_set_bytes=nbytes,
                               buf=buf, max_rounds=rounds, seed=0)
        r, logs = ctx.run_stressor(cfg, 20000)
        assert r["status"] == 0
        want = {lg["index"]: (lg["checksum"], lg["work"], lg["rounds"], lg["status"]) for lg in logs}
    assert len(want) == sm_count * bps
    hbuf = buf.cpu().numpy().view(np.uint32)
    planned = sm_count * bps
    for k, (cs, work, rnd, status) in want.items():
        assert status == 0 and rnd == rounds
        assert cs == oracle.stream_block_checksum(hbuf, block * 16, planned, k, work), k
    stream = torch.cuda.Stream()
    free_before = None
    for call in range(3):
        got = _noalloc_logs(L, kind, buf, nbytes, sm_count, bps, block, rounds, stream)
        assert got == want, call
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if free_before is None:
            # the first call may load the entry point's kernels; later calls change nothing
            free_before, alloc_before = free, torch.cuda.memory_allocated()
        else:
            assert free == free_before and torch.cuda.memory_allocated() == alloc_before, call


def test_noalloc_rejects_bad_sizes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = A.load()
    buf = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
    logs = torch.empty(64 * C.sizeof(A.ifr_block_log), dtype=torch.uint8, device="cuda")
    p, lp = C.c_void_p(buf.data_ptr()), C.c_void_p(logs.data_ptr())
    # logs array smaller than sm_count * blocks_per_sm
    assert L.ifr_stream_stressor_noalloc(A.IFR_S_HBM, p, 4 << 20, 40, 2, 512, 1, 0, None, lp, 64) == A.IFR_ERR_CAPACITY
    # wrong kind, unaligned size, no rounds, too many SMs
    assert L.ifr_stream_stressor_noalloc(A.IFR_S_FMA, p, 4 << 20, 4, 1, 512, 1, 0, None, lp, 64) == A.IFR_ERR_ARG
    assert L.ifr_stream_stressor_noalloc(A.IFR_S_HBM, p, 1000, 4, 1, 512, 1, 0, None, lp, 64) == A.IFR_ERR_ARG
    assert L.ifr_stream_stressor_noalloc(A.IFR_S_HBM, p, 4 << 20, 4, 1, 512, 0, 0, None, lp, 64) == A.IFR_ERR_ARG
    assert L.ifr_stream_stressor_noalloc(A.IFR_S_HBM, p, 4 << 20, 4096, 1, 512, 1, 0, None, lp, 64) == A.IFR_ERR_ARG

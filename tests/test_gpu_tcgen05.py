"""GPU parity of the tcgen05 kernels: the BF16 tensor-pipe stressor (bit-exact
small-integer tiles) and the BF16 GEMM victim (fp64 oracle, 2e-2 relative)."""
import numpy as np
import pytest
import torch

import ifr_inputs as I
import oracle
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from tests.gpu_common import BF16_TOL, need_gpu, spread_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ifr.Context(0)
    yield c
    c.close()


def _gemm(ctx, M, N, K, seed=11, repeats=1, variant=0):
    Ab = I.torch_normal_bf16(seed, M * K, "cuda").view(M, K)
    Bb = I.torch_normal_bf16(seed + 1, N * K, "cuda").view(N, K)
    C = torch.full((M, N), float("nan"), device="cuda")
    t = ctx.victim_launch(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Bb, C, m=M, n=N, k=K, repeats=repeats, variant=variant))
    return Ab, Bb, C, t


# the last two shapes have more output tiles than SMs (160 tiles of 128 x 256, 192 of
# 128 x 128), so most tiles are handed out by the device counter
# variant 3 (two accumulators): K is too short for a split last wave at these shapes
@pytest.mark.parametrize("variant", [0, 1, 3])  # colocation-friendly (3 stages) / throughput (4) / 2 accumulators
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 256, 128), (256, 384, 192), (384, 512, 1024),
                                   (2048, 2560, 128), (8192, 384, 64)])
def test_gemm_small_all_entries(ctx, M, N, K, variant, repeats=1):
    Ab, Bb, C, t = _gemm(ctx, M, N, K, variant=variant, repeats=repeats)
    assert t["status"] == 0
    ref = Ab.double().cpu() @ Bb.double().cpu().T
    got = C.double().cpu()
    assert torch.isfinite(got).all()
    rms = float(ref.pow(2).mean().sqrt())
    err = (got - ref).abs()
    assert bool((err <= BF16_TOL * torch.maximum(ref.abs(), torch.tensor(rms))).all())
    assert float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref)) <= 1e-5


# variant 2: 256 x 256 tiles on CTA pairs (cta_group::2, two accumulators); (2048,
# 2560) is 80 pair tiles for at most 74 pairs, so tiles also come from the device
# counter; K is too short for a split last wave at these shapes
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (256, 512, 128), (512, 768, 192), (768, 256, 1024),
                                   (2048, 2560, 128), (8192, 512, 64)])
def test_gemm_pair_tiles_all_entries(ctx, M, N, K):
    test_gemm_small_all_entries(ctx, M, N, K, 2)


# variant 4: pairs of vertically adjacent 128 x 256 tiles sharing B through TMA
# multicast; (2048, 2560) is 80 tile pairs for at most 74 clusters, so pairs also come
# from the device counter; three launches reuse the counter
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (256, 512, 128), (512, 768, 192), (768, 256, 1024),
                                   (2048, 2560, 128), (8192, 512, 64)])
def test_gemm_multicast_pairs_all_entries(ctx, M, N, K):
    test_gemm_small_all_entries(ctx, M, N, K, 4, repeats=3)


# split last waves (a part must run at least 32 K slices of 64).  Variant 3 (128 x 256
# tiles on 148 CTAs): 72 tiles in 2 K parts (one wave of 144 units), 6 tiles in 4
# parts, and 320 tiles = 296 whole + 24 in 2 parts.  Variant 2 (256 x 256 tiles on 74
# CTA pairs): 32 tiles in 2 parts, 4 tiles in 4 parts, and 160 tiles = 148 whole + 12
# in 2 parts.  Three launches each, so the arrival counters run over several
# launches, and the shapes alternate so the context re-zeroes them when the split
# changes.  Small shapes: every entry against fp64; the large ones: entries of every
# 128 x 128 block against the oracle.
@pytest.mark.parametrize("variant,M,N,K", [(3, 1152, 2048, 4096), (3, 384, 512, 8192), (3, 2560, 4096, 4096),
                                           (3, 1152, 2048, 4096), (2, 1024, 2048, 4096), (2, 512, 512, 8192),
                                           (2, 2560, 4096, 4096), (2, 1024, 2048, 4096)])
def test_gemm_split_wave(ctx, variant, M, N, K):
    if M * N * K <= 1 << 34:
        test_gemm_small_all_entries(ctx, M, N, K, variant, repeats=3)
        return
    Ab, Bb, C, t = _gemm(ctx, M, N, K, seed=31, repeats=3, variant=variant)
    assert t["status"] == 0 and torch.isfinite(C).all()
    rng = np.random.default_rng(1)
    ij = np.array([(bm * 128 + rng.integers(0, 128), bn * 128 + rng.integers(0, 128))
                   for bm in range(M // 128) for bn in range(N // 128) for _ in range(2)], np.int64)
    A_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(31, np.arange(M * K))).reshape(M, K)
    B_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(32, np.arange(N * K))).reshape(N, K)
    ref = oracle.gemm_entries(A_np, B_np, ij)
    got = C.cpu().numpy()[ij[:, 0], ij[:, 1]].astype(np.float64)
    rms = np.sqrt(np.mean(ref * ref))
    assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms))
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("variant", [0, 2, 3, 4])
def test_gemm_full_size_sampled_vs_oracle(ctx, variant):
    M = N = K = 4096
    Ab, Bb, C, t = _gemm(ctx, M, N, K, seed=21, repeats=2, variant=variant)
    assert t["status"] == 0 and t["sms_touched"] > 100
    rng = np.random.default_rng(0)
    ij = np.stack([rng.integers(0, M, 400), rng.integers(0, N, 400)], axis=1)
    ij = np.concatenate([ij, [[0, 0], [M - 1, N - 1], [127, 255], [128, 256]]])
    A_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(21, np.arange(M * K))).reshape(M, K)
    B_np = oracle.f32_bits_to_bf16_bits(I.np_normal_bf16(22, np.arange(N * K))).reshape(N, K)
    ref = oracle.gemm_entries(A_np, B_np, ij)
    got = C.cpu().numpy()[ij[:, 0], ij[:, 1]].astype(np.float64)
    rms = np.sqrt(np.mean(ref * ref))
    assert np.all(np.abs(got - ref) <= BF16_TOL * np.maximum(np.abs(ref), rms))
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    assert torch.isfinite(C).all()


def test_gemm_variant_profiles_and_bad_variant(ctx):
    Ab = I.torch_normal_bf16(1, 256 * 256, "cuda").view(256, 256)
    C = torch.empty(256, 256, device="cuda")
    p0 = ctx.victim_profile(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=0))
    p1 = ctx.victim_profile(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=1))
    p2 = ctx.victim_profile(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=2))
    p3 = ctx.victim_profile(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=3))
    assert p3["tmem_cols"] == 512 and p3["dynamic_smem"] == p1["dynamic_smem"]
    assert p1["dynamic_smem"] - p0["dynamic_smem"] == 128 * 64 * 2 + 256 * 64 * 2  # one more 48 KiB stage
    # pair tiles: six 32 KiB stages (each CTA's halves of A and B), two accumulators
    assert p2["dynamic_smem"] == 6 * 2 * 128 * 64 * 2 + 1024 + 256
    assert p2["tmem_cols"] == 512 and p2["grid"] == 2
    assert max(p["regs_per_thread"] for p in (p0, p1)) <= 96  # the variants that share SMs
    p4 = ctx.victim_profile(ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=4))
    assert p4["tmem_cols"] == 512 and p4["grid"] == 2 and p4["dynamic_smem"] == p1["dynamic_smem"]
    for bad in (ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=5),
                ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=128, n=256, k=256, variant=4),
                ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=128, n=256, k=256, variant=2),
                ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=384, k=256, variant=2),
                ifr.victim_cfg(A.IFR_V_SOFTMAX, C, None, C, m=256, n=256, variant=1)):
        with pytest.raises(ifr.IfrError):
            ctx.victim_launch(bad)


@pytest.mark.parametrize("solo_variant", [2, 3, 4])
def test_pair_gemm_refused_where_kernels_are_colocated(ctx, solo_variant):
    # the CTA pair's TMEM allocation, and the two-accumulator kernel's 512 columns, can
    # wait on other TMEM users: solo launches only
    Ab = I.torch_normal_bf16(1, 256 * 256, "cuda").view(256, 256)
    C = torch.empty(256, 256, device="cuda")
    pair = ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=solo_variant)
    single = ifr.victim_cfg(A.IFR_V_GEMM, Ab, Ab, C, m=256, n=256, k=256, variant=0)
    fma = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=1, block=128, max_rounds=1)
    for call in (lambda: ctx.sweep([pair], [], repeats=1), lambda: ctx.corun(pair, single),
                 lambda: ctx.corun(single, pair), lambda: ctx.colocate(fma, pair)):
        with pytest.raises(ifr.IfrError) as e:
            call()
        assert e.value.status == A.IFR_ERR_ARG
    assert ctx.victim_launch(pair)["status"] == 0


def test_gemm_rejects_bad_shapes(ctx):
    import ctypes as C

    L = A.load()
    x = torch.empty(1 << 16, device="cuda")
    t = A.ifr_timing()
    for m, n, k in [(100, 128, 64), (128, 100, 64), (128, 128, 32), (0, 128, 64)]:
        cfg = ifr.victim_cfg(A.IFR_V_GEMM, x, x, x, m=m, n=n, k=k)
        assert L.ifr_victim_launch(ctx._h, C.byref(cfg), None, C.byref(t)) == A.IFR_ERR_ARG


@pytest.mark.parametrize("sm_frac,bps,rounds", [(1.0, 1, 3), (0.5, 2, 2)])
def test_tensor_stressor_bit_exact(ctx, sm_frac, bps, rounds):
    S = ctx.info["num_sms"]
    n_sm = max(1, int(S * sm_frac))
    cfg = ifr.stressor_cfg(A.IFR_S_TENSOR, sm_count=n_sm, blocks_per_sm=bps, max_rounds=rounds, seed=12)
    r, logs = ctx.run_stressor(cfg, 20000)
    assert r["status"] == 0 and len(logs) == n_sm * bps
    assert {L["smid"] for L in logs} <= spread_mask(S, n_sm)
    for L in logs:
        assert L["rounds"] == rounds and L["work"] == rounds * 64
        assert L["checksum"] == oracle.tensor_block(12, L["index"], 64), L


def test_tensor_stressor_rejects_too_many_blocks(ctx):
    import ctypes as C

    L = A.load()
    h = C.c_int()
    cfg = ifr.stressor_cfg(A.IFR_S_TENSOR, sm_count=1, blocks_per_sm=3)
    assert L.ifr_stressor_launch(ctx._h, C.byref(cfg), None, C.byref(h)) == A.IFR_ERR_ARG

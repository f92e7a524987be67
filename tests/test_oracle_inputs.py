"""Pins for the seeded input generators and the oracle's SplitMix64."""
import os

import numpy as np
import torch

import ifr_inputs as I
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    vals = []
    with open(os.path.join(GOLD, "splitmix64_seed1234567.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line))
    return vals


def test_splitmix64_published_vector_all_implementations():
    want = _golden_splitmix()
    s0 = 1234567
    assert [I.splitmix64_at(s0, i) for i in range(5)] == want
    assert [oracle.splitmix64(s0, i) for i in range(5)] == want
    # numpy path (seed is applied as s0 = seed << 32, so emulate s0 directly)
    with np.errstate(over="ignore"):
        i = np.arange(5, dtype=np.uint64)
        z = np.uint64(s0) + (i + np.uint64(1)) * np.uint64(I.GAMMA)
    got = [I.mix64(int(v)) for v in z]
    assert got == want


def test_numpy_and_torch_generators_bit_identical():
    n = 4099
    for seed in (0, 1, 7, 123456):
        a = I.np_u32(seed, np.arange(n))
        b = I.torch_u32_as_i32(seed, n).numpy().view(np.uint32)
        assert np.array_equal(a, b)
        assert np.array_equal(I.np_uniform_pm1(seed, np.arange(n)), I.torch_uniform_pm1(seed, n).numpy())
        assert np.array_equal(I.np_key256(seed, np.arange(n)), I.torch_key256(seed, n).numpy())
        nb = I.torch_normal_bf16(seed, n).float().numpy()
        assert np.array_equal(I.np_normal_bf16(seed, np.arange(n)), nb)
    # offsets (start) address the same counter positions
    assert np.array_equal(I.torch_uniform_pm1(3, 100, start=1000).numpy(), I.np_uniform_pm1(3, np.arange(1000, 1100)))


def test_scalar_matches_vector():
    for seed in (0, 5):
        for i in (0, 1, 2, 1000, 2**31 + 7):
            assert int(I.np_u64(seed, [i])[0]) == I.splitmix64_at(I.state0(seed), i)


def test_uniform_range_and_exactness():
    x = I.np_uniform_pm1(0, np.arange(1 << 16))
    assert x.min() >= -1.0 and x.max() < 1.0
    # every value is an integer multiple of 2^-23 (exact in fp32)
    assert np.all(np.floor(x.astype(np.float64) * 2**23) == x.astype(np.float64) * 2**23)
    assert abs(float(x.mean())) < 0.02 and abs(float(x.var()) - 1 / 3) < 0.01


def test_normal_moments_and_bf16_exact():
    x = I.np_normal_bf16(9, np.arange(1 << 16)).astype(np.float64)
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n) + 0.01
    assert np.all(np.abs(x) <= 3.0)
    # values are representable in bf16: the low 16 bits of the fp32 pattern are zero
    assert np.all((x.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_bf16_rounding_matches_torch_for_fp32_exact_inputs():
    # when the exact value is already an fp32, the single rounding must agree with torch's
    v = np.arange(-(1 << 20), 1 << 20, 37, dtype=np.int64)
    f64 = v.astype(np.float64) * 2.0**-13
    ours = I._np_round_f64_to_bf16(f64)
    ref = torch.from_numpy(f64.astype(np.float32)).to(torch.bfloat16).float().numpy()
    assert np.array_equal(ours, ref)


def test_keys_uniform():
    k = I.np_key256(2, np.arange(1 << 18))
    assert k.min() == 0 and k.max() == 255
    c = np.bincount(k, minlength=256)
    assert c.min() > 0.8 * (1 << 10) and c.max() < 1.2 * (1 << 10)

"""Pins for the oracle's stressor checksums: brute force on tiny inputs written a
second way, closed forms, and plausible-mistake detection."""
from fractions import Fraction

import numpy as np
import pytest

import ifr_inputs as I
import oracle


def rotl(x, r):
    r &= 31
    return ((x << r) | (x >> (32 - r))) & 0xFFFFFFFF if r else x


# ---------------------------------------------------------------- stream (L2/HBM)
def _stream_brute(buf, chunk, A, k, count, fold):
    """Written a second way: the block's chunk list in reading order, and for every
    chunk the XOR of its first-of-16-bytes words and of each of its four quarters,
    looked up by the pass number."""
    n_chunks = buf.size // chunk
    mine = [c for c in range(n_chunks) if c % A == k]
    if not mine:
        return 0
    q = chunk // 4
    X0 = [int(np.bitwise_xor.reduce(buf[c * chunk:(c + 1) * chunk][0::4])) for c in range(n_chunks)]
    XQ = [[int(np.bitwise_xor.reduce(buf[c * chunk + i * q:c * chunk + (i + 1) * q])) for i in range(4)]
          for c in range(n_chunks)]
    acc = 0
    for j in range(count):
        p = j // len(mine)
        c = mine[j % len(mine)]
        acc ^= rotl(X0[c] if fold == 0 else XQ[c][p % 4], p)
    return acc


@pytest.mark.parametrize("fold", [oracle.FOLD_LOADS, oracle.FOLD_BULK])
@pytest.mark.parametrize("A,k,count", [(3, 0, 1), (3, 2, 7), (5, 4, 40), (7, 1, 0), (4, 3, 13), (16, 9, 3),
                                       (2, 1, 77)])
def test_stream_checksum_brute(A, k, count, fold):
    buf = I.np_u32(1, np.arange(64 * 37))
    assert oracle.stream_block_checksum(buf, 64, A, k, count, fold) == _stream_brute(buf, 64, A, k, count, fold)


def _block_chunks(A, k, n):
    return [c for c in range(n) if c % A == k]


def test_stream_checksum_loads_fold_two_passes_closed_form():
    # fold 0 folds the same words every pass: two passes give Y ^ rotl(Y, 1), Y the XOR
    # of the words 4i of the block's chunks
    buf = I.np_u32(11, np.arange(128 * 20))
    A, k = 4, 1
    mine = _block_chunks(A, k, 20)
    Y = 0
    for c in mine:
        Y ^= int(np.bitwise_xor.reduce(buf[c * 128:(c + 1) * 128:4]))
    assert oracle.stream_block_checksum(buf, 128, A, k, 2 * len(mine), oracle.FOLD_LOADS) == Y ^ rotl(Y, 1)
    # a flipped first word of a 16-byte group changes it, a flipped second word does not
    n = len(mine)
    b0 = buf.copy()
    b0[mine[1] * 128 + 8] ^= 1
    assert oracle.stream_block_checksum(b0, 128, A, k, n, oracle.FOLD_LOADS) != oracle.stream_block_checksum(
        buf, 128, A, k, n, oracle.FOLD_LOADS)
    b1 = buf.copy()
    b1[mine[1] * 128 + 9] ^= 1
    assert oracle.stream_block_checksum(b1, 128, A, k, 3 * n, oracle.FOLD_LOADS) == oracle.stream_block_checksum(
        buf, 128, A, k, 3 * n, oracle.FOLD_LOADS)


def test_stream_checksum_bulk_fold_four_and_eight_passes_closed_form():
    # fold 1, four passes fold quarter p of every chunk in pass p: the checksum is
    # rotl(Y0, 0) ^ rotl(Y1, 1) ^ rotl(Y2, 2) ^ rotl(Y3, 3), Y_q the XOR of quarter q
    # over the block's chunks; eight passes repeat the quarters with shifts 4..7
    buf = I.np_u32(11, np.arange(128 * 20))
    A, k = 4, 1
    mine = _block_chunks(A, k, 20)
    Y = [0, 0, 0, 0]
    for c in mine:
        for q in range(4):
            Y[q] ^= int(np.bitwise_xor.reduce(buf[c * 128 + 32 * q:c * 128 + 32 * (q + 1)]))
    want4 = Y[0] ^ rotl(Y[1], 1) ^ rotl(Y[2], 2) ^ rotl(Y[3], 3)
    assert oracle.stream_block_checksum(buf, 128, A, k, 4 * len(mine), oracle.FOLD_BULK) == want4
    want8 = want4 ^ rotl(Y[0], 4) ^ rotl(Y[1], 5) ^ rotl(Y[2], 6) ^ rotl(Y[3], 7)
    assert oracle.stream_block_checksum(buf, 128, A, k, 8 * len(mine), oracle.FOLD_BULK) == want8


def test_stream_checksum_bulk_fold_covers_the_pass_quarter_only():
    buf = I.np_u32(11, np.arange(128 * 20))
    A, k = 4, 1
    mine = _block_chunks(A, k, 20)
    F = oracle.FOLD_BULK
    one_pass = oracle.stream_block_checksum(buf, 128, A, k, len(mine), F)
    # pass 0 folds quarter 0: a flipped word there changes the checksum ...
    b0 = buf.copy()
    b0[mine[2] * 128 + 5] ^= 1
    assert oracle.stream_block_checksum(b0, 128, A, k, len(mine), F) != one_pass
    # ... a flipped word of quarter 1 does not, until pass 1 has read it
    b1 = buf.copy()
    b1[mine[2] * 128 + 32 + 5] ^= 1
    assert oracle.stream_block_checksum(b1, 128, A, k, len(mine), F) == one_pass
    assert oracle.stream_block_checksum(b1, 128, A, k, 2 * len(mine), F) != oracle.stream_block_checksum(
        buf, 128, A, k, 2 * len(mine), F)
    # another block's chunk is never read by this block
    b2 = buf.copy()
    b2[(mine[0] + 1) * 128 + 5] ^= 1
    assert oracle.stream_block_checksum(b2, 128, A, k, 8 * len(mine), F) == oracle.stream_block_checksum(
        buf, 128, A, k, 8 * len(mine), F)


# ---------------------------------------------------------------- FMA
def _round_f32(q: Fraction) -> float:
    """Correctly rounded (nearest, ties to even) fp32 value of a rational."""
    if q == 0:
        return 0.0
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    scaled = a * Fraction(2) ** (23 - e)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return s * float(Fraction(m) * Fraction(2) ** (e - 23))


def _f32_bits(v: float) -> int:
    return int(np.array([v], np.float32).view(np.uint32)[0])


def _fma_brute(seed, k, block, ilp, steps, rounds):
    s0 = I.state0(seed)
    a = 1 - Fraction(1, 2**12) - Fraction(I.splitmix64_at(s0, 0) >> 53, 2**23)
    b = Fraction((I.splitmix64_at(s0, 1) >> 40) - 2**23, 2**29)
    r0 = fin = 0
    for t in range(block):
        for j in range(ilp):
            g = (k * block + t) * ilp + j
            x = Fraction((I.splitmix64_at(s0, g + 2) >> 40) - 2**23, 2**23)
            for r in range(rounds):
                for _ in range(steps):
                    x = Fraction(_round_f32(x * a + b))
                if r == 0:
                    r0 ^= _f32_bits(float(x))
            fin ^= _f32_bits(float(x))
    return r0, fin


def test_fma_exact_rational_brute_force():
    assert oracle.fma_block(3, 2, 3, 2, 25, 2) == _fma_brute(3, 2, 3, 2, 25, 2)
    assert oracle.fma_block(0, 0, 2, 1, 40, 1) == _fma_brute(0, 0, 2, 1, 40, 1)


def test_fma_rounds_compose_and_fixed_point():
    # two rounds of s steps == one round of 2s steps (final value)
    assert oracle.fma_block(5, 1, 4, 2, 64, 2)[1] == oracle.fma_block(5, 1, 4, 2, 128, 1)[1]
    # with |a| < 1 the chain converges towards b / (1 - a); fp32 rounding stalls it
    # within about ulp(x*) / (1 - a) of the fixed point
    s0 = I.state0(8)
    a = 1 - 2.0**-12 - (I.splitmix64_at(s0, 0) >> 53) * 2.0**-23
    b = ((I.splitmix64_at(s0, 1) >> 40) - 2**23) * 2.0**-29
    _, fin = oracle.fma_block(8, 0, 1, 1, 200000, 1)
    x = np.array([fin], np.uint32).view(np.float32)[0]
    xs = b / (1 - a)
    assert abs(float(x) - xs) <= 2.0 * abs(float(np.spacing(np.float32(xs)))) / (1 - a)


# ---------------------------------------------------------------- FP64 multiply chains
def _round_f64(q: Fraction) -> float:
    """Correctly rounded (nearest, ties to even) fp64 value of a positive normal rational."""
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    if Fraction(2) ** (e + 1) <= q:
        e += 1
    scaled = q * Fraction(2) ** (52 - e)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return float(Fraction(m) * Fraction(2) ** (e - 52))


def _fold64(v: float) -> int:
    u = int(np.array([v], np.float64).view(np.uint64)[0])
    return (u ^ (u >> 32)) & 0xFFFFFFFF


def _fp64_params(seed):
    s0 = I.state0(seed)
    a = 1 - Fraction(1 + (I.splitmix64_at(s0, 0) >> 54), 2**40)
    return s0, a


def _fp64_brute(seed, k, block, ilp, steps, rounds):
    """Exact rational products rounded to fp64 one step at a time (Sec. 4.4.3 chains)."""
    s0, a = _fp64_params(seed)
    r0 = fin = 0
    for t in range(block):
        for j in range(ilp):
            g = (k * block + t) * ilp + j
            x = 1 + Fraction(I.splitmix64_at(s0, g + 2) >> 12, 2**52)
            for r in range(rounds):
                for _ in range(steps):
                    x = Fraction(_round_f64(x * a))
                if r == 0:
                    r0 ^= _fold64(float(x))
            fin ^= _fold64(float(x))
    return r0, fin


def test_fp64_exact_rational_brute_force():
    assert oracle.fp64_block(3, 2, 3, 2, 25, 2) == _fp64_brute(3, 2, 3, 2, 25, 2)
    assert oracle.fp64_block(0, 0, 2, 4, 30, 1) == _fp64_brute(0, 0, 2, 4, 30, 1)


def test_fp64_rounds_compose_and_error_bound():
    assert oracle.fp64_block(5, 1, 4, 2, 64, 2)[1] == oracle.fp64_block(5, 1, 4, 2, 128, 1)[1]
    # one chain (block 1, ilp 1): the rounded product stays within n half-ulps of the
    # exact x0 * a^n (each step adds a relative error of at most 2^-53)
    seed, n = 11, 4000
    s0, a = _fp64_params(seed)
    x0 = 1 + Fraction(I.splitmix64_at(s0, 2) >> 12, 2**52)
    exact = float(x0 * a ** n)
    _, fin = oracle.fp64_block(seed, 0, 1, 1, n, 1)
    # the fold loses the value; recover it by re-running the chain in Python floats
    x = float(x0)
    af = float(a)
    for _ in range(n):
        x = x * af
    assert _fold64(x) == fin
    assert abs(x - exact) <= n * 2.0**-53 * abs(exact) * 1.01
    assert 0 < float(a) < 1 and float(a) == a  # the multiplier is exact in fp64


# ---------------------------------------------------------------- shared memory
def smem_word(lane, j, ways):
    """(row, bank) -> word index for lane `lane`, iteration j, conflict degree `ways`."""
    g, r = divmod(lane, ways)
    groups = 32 // ways
    bank = g + groups * (j % ways)
    row = r + ways * (j // ways)
    return row * 32 + bank


def test_smem_conflict_free_vector_mapping():
    # the conflict-free kernel: lane l, access i (0..7), word e (0..3) -> 128*i + 4*l + e.
    # Every word of the warp's 1024 is visited once per pass, and each quarter-warp
    # phase of a 16-byte request (8 lanes x 4 words) covers the 32 banks once.
    seen = []
    for i in range(8):
        for quarter in range(4):
            banks = set()
            for l in range(8 * quarter, 8 * quarter + 8):
                for e in range(4):
                    w = 128 * i + 4 * l + e
                    seen.append(w)
                    banks.add(w % 32)
            assert banks == set(range(32))
    assert sorted(seen) == list(range(1024))


@pytest.mark.parametrize("ways", [1, 2, 4, 8, 16, 32])
def test_smem_mapping_bijective_and_conflict_degree(ways):
    seen = set()
    for j in range(32):
        banks = {}
        for lane in range(32):
            w = smem_word(lane, j, ways)
            assert w not in seen
            seen.add(w)
            banks.setdefault(w % 32, set()).add(w // 32)
        # every bank touched by this warp instruction sees exactly `ways` distinct rows
        assert all(len(rows) == ways for rows in banks.values())
    assert len(seen) == 1024


@pytest.mark.parametrize("ways", [1, 8, 32])
def test_smem_brute_force_matches(ways):
    seed, k, warps, rounds, passes = 6, 3, 2, 3, 3
    s0 = I.state0(seed)
    acc = 0
    for w in range(warps):
        mem = [I.splitmix64_at(s0, (k * warps + w) * 1024 + q) & 0xFFFFFFFF for q in range(1024)]
        for gp in range(rounds * passes):
            for j in range(32):
                for lane in range(32):
                    q = smem_word(lane, j, ways)
                    v = mem[q]
                    # even passes apply the LCG, odd passes copy the word back
                    mem[q] = (v * 1664525 + 1013904223) & 0xFFFFFFFF if gp % 2 == 0 else v
        for v in mem:
            acc ^= v
    assert oracle.smem_block(seed, k, warps, rounds, passes) == acc


def test_lcg_power_geometric_closed_form():
    a, c = 1664525, 1013904223
    for n in (0, 1, 2, 17, 1000):
        A, C = oracle.lcg_power(n)
        assert A == pow(a, n, 2**32)
        assert C == (c * ((a**n - 1) // (a - 1))) % 2**32


# ---------------------------------------------------------------- tensor
@pytest.mark.parametrize("k,group", [(0, 1), (3, 256), (7, 64)])
def test_tensor_matches_integer_matmul(k, group):
    s0 = I.state0(12)
    idx = np.arange(8192, dtype=np.uint64)
    u_a = I.np_u64(12, np.uint64(k * 16384) + idx)
    u_b = I.np_u64(12, np.uint64(k * 16384 + 8192) + idx)
    A = ((u_a >> np.uint64(32)) % np.uint64(5)).astype(np.int64).reshape(128, 64) - 2
    B = ((u_b >> np.uint64(32)) % np.uint64(5)).astype(np.int64).reshape(128, 64) - 2
    C = (A @ B.T) * group
    assert np.abs(C).max() < 2**24
    want = int(np.bitwise_xor.reduce(C.astype(np.float32).view(np.uint32).ravel()))
    assert oracle.tensor_block(12, k, group) == want
    assert s0 == 12 << 32


# ---------------------------------------------------------------- scheduler
def test_sched_brute_force():
    seed = 0xDEADBEEF12
    acc = 0
    for q in range(1500):
        y = (q ^ seed) & 0xFFFFFFFF
        for _ in range(16):
            y = (y * 1664525 + 1013904223) & 0xFFFFFFFF
        acc ^= y
    assert oracle.sched_checksum(seed, 1500, 16) == acc

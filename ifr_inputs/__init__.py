"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds only the input recipe: a counter-based SplitMix64 generator
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) and fixed conversions from its 64-bit outputs to the value types
the workloads need.  It contains none of the interference method's arithmetic
(no stressor, victim or reduction), so both sides may import it.

Counter-based definition.  For a 64-bit start state ``s0`` the i-th output
(i = 0, 1, ...) is ``mix(s0 + (i + 1) * GAMMA mod 2^64)`` with

    mix(z):  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
             z = (z ^ (z >> 27)) * 0x94D049BB133111EB
             return z ^ (z >> 31)

i.e. exactly the sequence the published sequential generator emits when seeded
with ``s0``.  A workload seed ``seed`` uses ``s0 = seed << 32``.

Conversions (all exact, no floating-point rounding except the documented bf16
round-to-nearest-even):

* ``u32``        low 32 bits of the output.
* ``uniform_pm1`` ``((u >> 40) - 2^23) * 2^-23``: a float32 in [-1, 1), exact.
* ``key256``     ``u >> 56``: an integer in [0, 256).
* ``normal_bf16`` Irwin-Hall(3) approximation of N(0, 1): the sum of three
  consecutive ``uniform_pm1`` draws (indices 3i, 3i+1, 3i+2), each U[-1, 1) with
  variance 1/3, so the sum has mean 0 and variance 1; the exact sum (an integer
  multiple of 2^-23) is rounded once to bf16 with round-to-nearest-even.

Every function has a numpy (CPU) and a torch (any device) implementation that
agree bit for bit; the torch one only uses int64 wrap-around arithmetic.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def state0(seed: int) -> int:
    """Start state of the stream for workload seed ``seed``."""
    return (int(seed) << 32) & MASK64


# ----------------------------------------------------------------------------------
# scalar reference (pure Python integers)
# ----------------------------------------------------------------------------------
def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MUL2) & MASK64
    return z ^ (z >> 31)


def splitmix64_at(s0: int, i: int) -> int:
    """i-th output of SplitMix64 started from state ``s0`` (pure Python)."""
    return mix64((s0 + (i + 1) * GAMMA) & MASK64)


# ----------------------------------------------------------------------------------
# numpy
# ----------------------------------------------------------------------------------
def np_u64(seed: int, idx) -> np.ndarray:
    """SplitMix64 outputs for stream ``seed`` at counter indices ``idx`` (uint64)."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state0(seed)) + (i + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MUL2)
        z = z ^ (z >> np.uint64(31))
    return z


def np_u32(seed: int, idx) -> np.ndarray:
    return (np_u64(seed, idx) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def np_uniform_pm1(seed: int, idx) -> np.ndarray:
    v = (np_u64(seed, idx) >> np.uint64(40)).astype(np.int64) - (1 << 23)
    return (v.astype(np.float64) * 2.0 ** -23).astype(np.float32)


def np_key256(seed: int, idx) -> np.ndarray:
    return (np_u64(seed, idx) >> np.uint64(56)).astype(np.int32)


def _np_round_f64_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bf16 (ties to even); returns float32."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.int64)
    low = np.int64((1 << 45) - 1)
    rnd = ((b >> np.int64(45)) & np.int64(1)) + np.int64((1 << 44) - 1)
    r = (b + rnd) & ~low
    return r.view(np.float64).astype(np.float32)


def np_normal_bf16(seed: int, idx) -> np.ndarray:
    """Irwin-Hall(3) N(0,1) draws rounded to bf16, returned as float32 (exact)."""
    i = np.asarray(idx, dtype=np.uint64)
    s = np.zeros(i.shape, dtype=np.int64)
    for k in range(3):
        s += (np_u64(seed, i * np.uint64(3) + np.uint64(k)) >> np.uint64(40)).astype(np.int64) - (1 << 23)
    return _np_round_f64_to_bf16(s.astype(np.float64) * 2.0 ** -23)


# ----------------------------------------------------------------------------------
# torch (int64 two's-complement arithmetic; bit-identical to the numpy version)
# ----------------------------------------------------------------------------------
def _s64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(t, k: int):
    import torch

    return (t >> k) & ((1 << (64 - k)) - 1)


def torch_u64(seed: int, n: int, device="cpu", start: int = 0):
    """SplitMix64 outputs for indices start..start+n-1 as int64 (bit pattern of the u64)."""
    import torch

    i = torch.arange(start, start + n, dtype=torch.int64, device=device)
    z = (i + 1) * _s64(GAMMA) + _s64(state0(seed))
    z = (z ^ _lsr(z, 30)) * _s64(MUL1)
    z = (z ^ _lsr(z, 27)) * _s64(MUL2)
    return z ^ _lsr(z, 31)


_CHUNK = 1 << 25


def torch_u32_as_i32(seed: int, n: int, device="cpu", start: int = 0):
    """Low 32 bits of each output, returned as int32 (same bits as np_u32)."""
    import torch

    out = torch.empty(n, dtype=torch.int32, device=device)
    for off in range(0, n, _CHUNK):
        m = min(_CHUNK, n - off)
        z = torch_u64(seed, m, device, start + off)
        lo = z & 0xFFFFFFFF
        out[off : off + m] = torch.where(lo >= (1 << 31), lo - (1 << 32), lo).to(torch.int32)
    return out


def torch_uniform_pm1(seed: int, n: int, device="cpu", start: int = 0):
    import torch

    out = torch.empty(n, dtype=torch.float32, device=device)
    for off in range(0, n, _CHUNK):
        m = min(_CHUNK, n - off)
        v = _lsr(torch_u64(seed, m, device, start + off), 40) - (1 << 23)
        out[off : off + m] = (v.to(torch.float64) * 2.0 ** -23).to(torch.float32)
    return out


def torch_key256(seed: int, n: int, device="cpu", start: int = 0):
    import torch

    out = torch.empty(n, dtype=torch.int32, device=device)
    for off in range(0, n, _CHUNK):
        m = min(_CHUNK, n - off)
        out[off : off + m] = _lsr(torch_u64(seed, m, device, start + off), 56).to(torch.int32)
    return out


def torch_normal_bf16(seed: int, n: int, device="cpu", start: int = 0):
    """Irwin-Hall(3) N(0,1) draws rounded to bf16 (returned as a bfloat16 tensor)."""
    import torch

    out = torch.empty(n, dtype=torch.bfloat16, device=device)
    step = _CHUNK // 4
    for off in range(0, n, step):
        m = min(step, n - off)
        i = torch.arange(start + off, start + off + m, dtype=torch.int64, device=device)
        s = torch.zeros(m, dtype=torch.int64, device=device)
        for k in range(3):
            j = i * 3 + k
            z = (j + 1) * _s64(GAMMA) + _s64(state0(seed))
            z = (z ^ _lsr(z, 30)) * _s64(MUL1)
            z = (z ^ _lsr(z, 27)) * _s64(MUL2)
            z = z ^ _lsr(z, 31)
            s += _lsr(z, 40) - (1 << 23)
        b = (s.to(torch.float64) * 2.0 ** -23).view(torch.int64)
        low = (1 << 45) - 1
        b = (b + (((b >> 45) & 1) + ((1 << 44) - 1))) & ~low
        out[off : off + m] = b.view(torch.float64).to(torch.float32).to(torch.bfloat16)
    return out

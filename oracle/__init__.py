"""CPU oracle for the interference-sensitivity hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_2501_16909_b300``) never imports it and shares no code
with it; the only module both sides use is ``ifr_inputs`` (seeded inputs, none
of the method's arithmetic).

Layout:
  ifr_oracle.c   plain C: SplitMix64, stressor checksums, victims in fp64
  reduction.py   slowdown / sensitivity reduction from raw timestamps
  mlp.py         slowdown-predictor MLP forward / backward / Adam in fp64 numpy
  build.py       compiles ifr_oracle.c into liboracle.so with gcc

Every function cites the passage it follows; pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def lib():
    """Load (building on first use) the C oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u64, i64, u32, i32 = C.c_uint64, C.c_int64, C.c_uint32, C.c_int
        p = C.c_void_p
        L.or_splitmix64.restype = u64
        L.or_splitmix64.argtypes = [u64, u64]
        L.or_stream_block_checksum.restype = u32
        L.or_stream_block_checksum.argtypes = [p, i64, i64, i64, i64, i64, i32]
        L.or_fma_block.restype = None
        L.or_fma_block.argtypes = [u64, i64, i32, i32, i32, i64, p, p]
        L.or_fp64_block.restype = None
        L.or_fp64_block.argtypes = [u64, i64, i32, i32, i32, i64, p, p]
        L.or_smem_block.restype = u32
        L.or_smem_block.argtypes = [u64, i64, i32, i64, i32]
        L.or_tensor_block.restype = u32
        L.or_tensor_block.argtypes = [u64, i64, i32]
        L.or_sched_checksum.restype = u32
        L.or_sched_checksum.argtypes = [u64, i64, i32]
        L.or_lcg_power.restype = None
        L.or_lcg_power.argtypes = [i64, p, p]
        L.or_triad.restype = None
        L.or_triad.argtypes = [p, p, C.c_float, i64, p]
        L.or_layernorm_rows.restype = None
        L.or_layernorm_rows.argtypes = [p, i64, C.c_double, p, i64, p]
        L.or_softmax_rows.restype = None
        L.or_softmax_rows.argtypes = [p, i64, p, i64, p]
        L.or_gemv_rows.restype = None
        L.or_gemv_rows.argtypes = [p, p, i64, p, i64, p]
        L.or_gemm_entries.restype = None
        L.or_gemm_entries.argtypes = [p, p, i64, p, i64, p]
        L.or_histogram.restype = None
        L.or_histogram.argtypes = [p, i64, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ generator
def splitmix64(s0: int, i: int) -> int:
    return int(lib().or_splitmix64(s0, i))


# ------------------------------------------------------------------ stressors
# fold of the L2 / HBM stream stressor's checksum: by loads into registers (first
# word of every 16-byte group) or by bulk copies into shared memory (quarter pass
# mod 4 of each chunk); see ifr_oracle.c
FOLD_LOADS, FOLD_BULK = 0, 1


def stream_block_checksum(buf_u32: np.ndarray, chunk_elems: int, active_planned: int, k: int, count: int,
                          fold: int = FOLD_LOADS) -> int:
    b = np.ascontiguousarray(buf_u32, dtype=np.uint32)
    return int(lib().or_stream_block_checksum(_ptr(b), b.size, chunk_elems, active_planned, k, count, fold))


def fma_block(seed: int, k: int, block: int, ilp: int, steps: int, rounds: int):
    r0, fin = C.c_uint32(0), C.c_uint32(0)
    lib().or_fma_block(seed, k, block, ilp, steps, rounds, C.byref(r0), C.byref(fin))
    return int(r0.value), int(fin.value)


def fp64_block(seed: int, k: int, block: int, ilp: int, steps: int, rounds: int):
    """FP64 multiply-chain stressor block (Sec. 4.4.3): (round-0 XOR, final XOR)."""
    r0, fin = C.c_uint32(0), C.c_uint32(0)
    lib().or_fp64_block(seed, k, block, ilp, steps, rounds, C.byref(r0), C.byref(fin))
    return int(r0.value), int(fin.value)


def smem_block(seed: int, k: int, warps: int, rounds: int, passes: int) -> int:
    return int(lib().or_smem_block(seed, k, warps, rounds, passes))


def tensor_block(seed: int, k: int, group: int) -> int:
    return int(lib().or_tensor_block(seed, k, group))


def sched_checksum(seed: int, total_blocks: int, lcg_steps: int) -> int:
    return int(lib().or_sched_checksum(seed, total_blocks, lcg_steps))


def lcg_power(n: int):
    a, c = C.c_uint32(0), C.c_uint32(0)
    lib().or_lcg_power(n, C.byref(a), C.byref(c))
    return int(a.value), int(c.value)


# ------------------------------------------------------------------ victims
def triad(b: np.ndarray, c: np.ndarray, s: float) -> np.ndarray:
    b = np.ascontiguousarray(b, np.float32)
    c = np.ascontiguousarray(c, np.float32)
    out = np.empty(b.size, np.float64)
    lib().or_triad(_ptr(b), _ptr(c), C.c_float(s), b.size, _ptr(out))
    return out


def layernorm_rows(x: np.ndarray, rows, eps: float = 1e-5) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    r = np.ascontiguousarray(rows, np.int64)
    out = np.empty((r.size, x.shape[1]), np.float64)
    lib().or_layernorm_rows(_ptr(x), x.shape[1], eps, _ptr(r), r.size, _ptr(out))
    return out


def softmax_rows(x: np.ndarray, rows) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    r = np.ascontiguousarray(rows, np.int64)
    out = np.empty((r.size, x.shape[1]), np.float64)
    lib().or_softmax_rows(_ptr(x), x.shape[1], _ptr(r), r.size, _ptr(out))
    return out


def gemv_rows(A_bf16_bits: np.ndarray, x_bf16_bits: np.ndarray, rows) -> np.ndarray:
    A = np.ascontiguousarray(A_bf16_bits, np.uint16)
    x = np.ascontiguousarray(x_bf16_bits, np.uint16)
    r = np.ascontiguousarray(rows, np.int64)
    out = np.empty(r.size, np.float64)
    lib().or_gemv_rows(_ptr(A), _ptr(x), A.shape[1], _ptr(r), r.size, _ptr(out))
    return out


def gemm_entries(A_bf16_bits: np.ndarray, B_bf16_bits: np.ndarray, ij) -> np.ndarray:
    A = np.ascontiguousarray(A_bf16_bits, np.uint16)
    B = np.ascontiguousarray(B_bf16_bits, np.uint16)
    ij = np.ascontiguousarray(ij, np.int64).reshape(-1, 2)
    out = np.empty(ij.shape[0], np.float64)
    lib().or_gemm_entries(_ptr(A), _ptr(B), A.shape[1], _ptr(ij), ij.shape[0], _ptr(out))
    return out


def histogram(keys: np.ndarray) -> np.ndarray:
    k = np.ascontiguousarray(keys, np.int32)
    out = np.zeros(256, np.uint64)
    lib().or_histogram(_ptr(k), k.size, _ptr(out))
    return out


def f32_bits_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Bit pattern of float32 values that are already exact bf16 (truncation is exact)."""
    return (np.ascontiguousarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)

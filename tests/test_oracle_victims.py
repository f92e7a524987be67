"""Pins for the oracle's victims: library routines, closed forms and invariants."""
import numpy as np
import torch

import ifr_inputs as I
import oracle


def test_triad_matches_numpy_fp64():
    n = 1000
    b = I.np_uniform_pm1(0, np.arange(n))
    c = I.np_uniform_pm1(0, np.arange(n, 2 * n))
    got = oracle.triad(b, c, 1.5)
    assert np.array_equal(got, b.astype(np.float64) + 1.5 * c.astype(np.float64))
    # s = 0 copies b exactly
    assert np.array_equal(oracle.triad(b, c, 0.0), b.astype(np.float64))


def test_layernorm_invariants_and_closed_form():
    x = I.np_uniform_pm1(4, np.arange(8 * 512)).reshape(8, 512)
    y = oracle.layernorm_rows(x, np.arange(8), 1e-5)
    assert np.allclose(y.mean(axis=1), 0.0, atol=1e-12)
    var = x.astype(np.float64).var(axis=1)
    assert np.allclose((y * y).mean(axis=1), var / (var + 1e-5), rtol=1e-12)
    # a two-valued row {-1, +1} has mean 0 and variance 1: y = x / sqrt(1 + eps)
    r = np.tile(np.array([-1.0, 1.0], np.float32), 8)[None, :]
    assert np.allclose(oracle.layernorm_rows(r, [0], 1e-5), r / np.sqrt(1 + 1e-5), rtol=0, atol=1e-15)
    # a constant row normalises to zero
    assert np.all(oracle.layernorm_rows(np.full((1, 16), 3.0, np.float32), [0]) == 0.0)
    # agrees with torch's layer_norm (library routine) in fp64
    t = torch.nn.functional.layer_norm(torch.from_numpy(x.astype(np.float64)), (512,), eps=1e-5).numpy()
    assert np.allclose(y, t, rtol=1e-12, atol=1e-12)
    # row selection picks the right rows
    assert np.array_equal(oracle.layernorm_rows(x, [5, 2]), y[[5, 2]])


def test_softmax_invariants_and_closed_form():
    x = I.np_uniform_pm1(5, np.arange(4 * 300)).reshape(4, 300) * 8
    x = x.astype(np.float32)
    y = oracle.softmax_rows(x, np.arange(4))
    assert np.allclose(y.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert np.all(y > 0)
    # two-element softmax is the logistic function of the difference
    z = np.array([[0.75, -0.5]], np.float32)
    y2 = oracle.softmax_rows(z, [0])
    assert abs(y2[0, 0] - 1.0 / (1.0 + np.exp(-1.25))) < 1e-15
    t = torch.softmax(torch.from_numpy(x.astype(np.float64)), dim=1).numpy()
    assert np.allclose(y, t, rtol=1e-12, atol=0)


def test_gemv_gemm_match_matmul():
    A = I.np_normal_bf16(7, np.arange(64 * 96)).reshape(64, 96)
    B = I.np_normal_bf16(8, np.arange(40 * 96)).reshape(40, 96)
    x = I.np_normal_bf16(9, np.arange(96))
    Ab, Bb, xb = (oracle.f32_bits_to_bf16_bits(v) for v in (A, B, x))
    y = oracle.gemv_rows(Ab, xb, np.arange(64))
    assert np.allclose(y, A.astype(np.float64) @ x.astype(np.float64), rtol=1e-13, atol=1e-13)
    ij = np.array([[0, 0], [63, 39], [10, 7], [5, 33]])
    c = oracle.gemm_entries(Ab, Bb, ij)
    full = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.allclose(c, full[ij[:, 0], ij[:, 1]], rtol=1e-13, atol=1e-13)
    # a transposed operand would give a different answer (B is K-major: C = A B^T)
    assert not np.allclose(c[2], (A.astype(np.float64) @ B.astype(np.float64).T)[7, 10])


def test_histogram_matches_bincount():
    k = I.np_key256(2, np.arange(100003))
    h = oracle.histogram(k)
    assert np.array_equal(h, np.bincount(k, minlength=256).astype(np.uint64))
    assert int(h.sum()) == 100003
    # keys are reduced modulo 256
    assert int(oracle.histogram(np.array([256 + 3, 3, -1], np.int32))[3]) == 2
    assert int(oracle.histogram(np.array([-1], np.int32))[255]) == 1

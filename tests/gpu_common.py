"""Helpers shared by the GPU parity tests (inputs, mask rule, tolerances)."""
import numpy as np
import pytest
import torch

import ifr_inputs as I

FP32_TOL = 1e-5   # FP32 victims: |y - r| <= 1e-5 * max(|r|, rms(r))
BF16_TOL = 2e-2   # BF16 GEMM / GEMV


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def spread_mask(num_sms, sm_count):
    """SM ids a stressor with sm_count of num_sms SMs may use (the header's rule)."""
    return {s for s in range(num_sms) if (s + 1) * sm_count // num_sms > s * sm_count // num_sms}


def assert_fp32_close(y, r, tol=FP32_TOL):
    y = np.asarray(y, np.float64)
    r = np.asarray(r, np.float64)
    rms = np.sqrt(np.mean(r * r)) if r.size else 0.0
    bound = tol * np.maximum(np.abs(r), rms)
    bad = np.abs(y - r) > bound
    assert not bad.any(), "max err %g at %s (ref %g)" % (np.abs(y - r).max(), np.argmax(np.abs(y - r) - bound),
                                                        r.ravel()[np.argmax(np.abs(y - r) - bound)])


def bf16_bits(t):
    """Bit patterns (uint16 numpy) of a bfloat16 torch tensor."""
    return t.detach().cpu().view(torch.int16).numpy().view(np.uint16)


def u32_buffer(seed, n, device="cuda"):
    return I.torch_u32_as_i32(seed, n, device)

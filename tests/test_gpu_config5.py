"""Configuration 5 end to end on a reduced case: synthetic decoder-layer kernels of a
prefill and a decode stream colocated pairwise (ifr_corun), every pair scored by the
predictor (trained on a reduced set of measured stressor and kernel pairs) and by the
baseline without the network.  The measured slowdowns must be valid, the predictions
finite and positive, and the reported MAPEs must be what the per-pair rows give."""
import math

import numpy as np
import pytest

from paper_2501_16909_b300 import colocate_config5 as C5
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

KERNELS = ["prefill.layernorm", "prefill.oproj", "prefill.silu_mul", "decode.layernorm", "decode.qkv",
           "decode.softmax", "decode.silu_mul"]


def _mape(pred, meas):
    return float(np.mean([abs(p - m) / m for p, m in zip(pred, meas)]))


def test_config5_reduced_end_to_end():
    need_gpu()
    out = C5.main(["--repeats", "1", "--members", "1", "--max-epochs", "15", "--kernels", ",".join(KERNELS),
                   "--rows", "hbm/a,fma/a,tensor/a,smem_32w/a,l2/a", "--co-idx", "0,16,32,48"])
    assert out["kernels"] == KERNELS
    pairs = out["pairs"]
    assert out["config5_pairs"] == len(pairs) >= 6
    for p in pairs:
        assert p["victim"].split(".")[0] != p["corunner"].split(".")[0]  # prefill x decode only
        assert math.isfinite(p["measured"]) and p["measured"] > 0.5
        assert math.isfinite(p["mlp"]) and p["mlp"] > 0 and math.isfinite(p["baseline"]) and p["baseline"] >= 1.0
    meas = [p["measured"] for p in pairs]
    assert abs(_mape([p["mlp"] for p in pairs], meas) - out["mlp_mape"]) <= 1e-3
    assert abs(_mape([p["baseline"] for p in pairs], meas) - out["baseline_mape"]) <= 1e-3
    assert out["training_pairs"] > 1000

"""Host tests of the predictor's measured features (no GPU): shapes, that missing
measurements carry no evidence, and that a stressor's configuration knobs (ILP,
bank-conflict degree, duty) are not inputs — two configurations with the same
measurements get the same features."""
import math

import numpy as np

import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import _abi as A
from paper_2501_16909_b300 import predictor as PR

S = 148
PK = {A.IFR_S_HBM: (6.5e12, ""), A.IFR_S_L2: (23e12, ""), A.IFR_S_TENSOR: (1.7e15, ""), A.IFR_S_FMA: (77e12, ""),
      A.IFR_S_SMEM_CF: (3e11, ""), A.IFR_S_SMEM_32W: (3e11, ""), A.IFR_S_SCHED: (5e9, "")}


def _prof(**kw):
    p = dict(grid=296, block=512, regs_per_thread=40, static_smem=1024, dynamic_smem=0, max_blocks_per_sm=4,
             tmem_cols=0, uses_tensor=0, sm_count=S, blocks_per_sm=2, launches=1, bytes_per_launch=1e8,
             flops_per_launch=1e6)
    p.update(kw)
    return p


def test_victim_features_shape_and_measured_parts():
    f = PR.victim_features(_prof(), 20000.0, 148, [1.0, 1.5, 1.2, 2.0, 3.0, 1.1, float("nan")], PK, S)
    assert f.shape == (24,) and np.isfinite(f).all()
    d = dict(zip(PR.VICTIM_FEATURES, f))
    assert math.isclose(d["frac_hbm"], 1e8 / 20e-6 / 6.5e12)
    assert math.isclose(d["log_sens_fma"], math.log(1.5))
    assert d["log_sens_hbm"] == 0.0  # no valid measurement: no evidence
    assert d["sm_fraction"] == 1.0


def test_stressor_features_ignore_configuration_knobs():
    solo = {"sms_used": 148, "blocks_active": 296, "elapsed_ms": 0.5}
    pres = [1.0, 1.1, 3.0, 1.0, 1.2, 1.0]
    a = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=2, block=128, ilp=1)
    b = ifr.stressor_cfg(A.IFR_S_FMA, sm_count=S, blocks_per_sm=2, block=128, ilp=8, duty=0.5)
    fa = PR.stressor_corunner_features(_prof(block=128), a, 5e13, 0.65, PK, solo, pres, S)
    fb = PR.stressor_corunner_features(_prof(block=128), b, 5e13, 0.65, PK, solo, pres, S)
    assert fa.shape == (24,) and np.array_equal(fa, fb)
    c = ifr.stressor_cfg(A.IFR_S_SMEM_32W, sm_count=S, smem_ways=8)
    d = ifr.stressor_cfg(A.IFR_S_SMEM_32W, sm_count=S, smem_ways=32)
    assert np.array_equal(PR.stressor_corunner_features(_prof(), c, 1e11, 0.4, PK, solo, pres, S),
                          PR.stressor_corunner_features(_prof(), d, 1e11, 0.4, PK, solo, pres, S))


def test_hbm_stream_l2_fraction_is_its_measured_rate_over_the_l2_peak():
    solo = {"sms_used": 148, "blocks_active": 296, "elapsed_ms": 0.4}
    cfg = ifr.stressor_cfg(A.IFR_S_HBM, sm_count=S)
    f = dict(zip(PR.CORUNNER_FEATURES,
                 PR.stressor_corunner_features(_prof(), cfg, 6.0e12, 6.0e12 / 6.5e12, PK, solo, [1.0] * 6, S)))
    assert math.isclose(f["frac_hbm"], 6.0 / 6.5) and math.isclose(f["frac_l2"], 6.0e12 / 23e12)
    assert f["frac_fp32"] == 0.0 and f["frac_tensor"] == 0.0


def test_kernel_corunner_features_pressure_and_fracs():
    f = dict(zip(PR.CORUNNER_FEATURES,
                 PR.kernel_corunner_features(_prof(uses_tensor=1, flops_per_launch=1e11, tmem_cols=256), 1e5, 100,
                                             [2.0, 1.0, 1.0, 1.0, 1.0, float("nan")], PK, S)))
    assert math.isclose(f["frac_tensor"], 1e11 / 1e-4 / 1.7e15) and f["frac_fp32"] == 0.0
    assert math.isclose(f["log_pressure_hbm_triad"], math.log(2.0)) and f["log_pressure_short_gemv"] == 0.0
    assert math.isclose(f["pressure_max"], math.log(2.0))


def test_standardizer_zeroes_features_constant_in_training():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(50, 4))
    X[:, 2] = 0.0  # never varies on the training side
    z = PR.Standardizer(X)
    held = np.array([[0.1, -0.2, 0.97, 1e6]])
    out = z(held)
    assert out[0, 2] == 0.0 and out[0, 3] == PR.Standardizer.Z_CLIP
    assert np.allclose(z(X)[:, [0, 1, 3]].mean(axis=0), 0.0, atol=1e-12)
    assert np.all(z(X)[:, 2] == 0.0)

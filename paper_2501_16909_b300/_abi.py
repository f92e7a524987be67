"""ctypes mirror of include/ifr.h (argument marshalling only).

Every structure here has the exact layout of its C counterpart (a CPU test
compiles the header and compares sizes and offsets).  Loading fails loudly
when libifr.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libifr.so")

IFR_OK = 0
IFR_ERR_ARG = -1
IFR_ERR_CUDA = -2
IFR_ERR_TIMEOUT = -3
IFR_ERR_NOT_RESIDENT = -4
IFR_ERR_LAUNCH = -5
IFR_ERR_BOUNDS = -6
IFR_ERR_UNSUPPORTED = -7
IFR_ERR_NOMEM = -8
IFR_ERR_CAPACITY = -9
IFR_ERR_INVALID_CELL = -10
IFR_ERR_HOL = -11

IFR_MAX_STRESSORS = 16
IFR_MAX_LEVELS = 16
IFR_MAX_SMS = 256

# stressor kinds
(IFR_S_SCHED, IFR_S_FMA, IFR_S_TENSOR, IFR_S_SMEM_CF, IFR_S_SMEM_32W, IFR_S_L2, IFR_S_HBM, IFR_S_FP64,
 IFR_S_SLEEP) = range(9)
STRESSOR_NAMES = ["sched", "fma", "tensor", "smem_cf", "smem_32w", "l2", "hbm", "fp64", "sleep"]
# victim kinds
IFR_V_TRIAD, IFR_V_GEMM, IFR_V_GEMV, IFR_V_LAYERNORM, IFR_V_SOFTMAX, IFR_V_HIST = range(6)
VICTIM_NAMES = ["triad", "gemm", "gemv", "layernorm", "softmax", "hist"]


class ifr_device_info(C.Structure):
    _fields_ = [
        ("device", C.c_int32), ("num_sms", C.c_int32), ("cc_major", C.c_int32), ("cc_minor", C.c_int32),
        ("l2_bytes", C.c_int64), ("smem_per_sm", C.c_int32), ("smem_per_block_optin", C.c_int32),
        ("regs_per_sm", C.c_int32), ("max_threads_per_sm", C.c_int32), ("max_blocks_per_sm", C.c_int32),
        ("sm_clock_khz", C.c_int32), ("mem_clock_khz", C.c_int32), ("mem_bus_width_bits", C.c_int32),
        ("global_mem_bytes", C.c_int64), ("name", C.c_char * 128),
    ]


class ifr_stressor_cfg(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("sm_count", C.c_int32), ("blocks_per_sm", C.c_int32), ("block", C.c_int32),
        ("ilp", C.c_int32), ("smem_ways", C.c_int32), ("duty", C.c_float), ("period_ns", C.c_int32),
        ("working_set_bytes", C.c_int64), ("buf", C.c_void_p), ("seed", C.c_uint64), ("max_rounds", C.c_int64),
        ("sched_blocks", C.c_int32), ("sched_launches", C.c_int32), ("sched_cycles", C.c_int32),
        ("mask_mode", C.c_int32), ("deadline_ns", C.c_uint64), ("sm_mask", C.c_uint32 * (IFR_MAX_SMS // 32)),
        ("staging", C.c_int32), ("reserved", C.c_int32),
    ]


class ifr_stressor_result(C.Structure):
    _fields_ = [
        ("checksum", C.c_uint32), ("status", C.c_int32), ("rounds", C.c_uint64), ("work", C.c_uint64),
        ("t_start_ns", C.c_uint64), ("t_start_last_ns", C.c_uint64), ("t_end_first_ns", C.c_uint64),
        ("t_end_ns", C.c_uint64), ("blocks_launched", C.c_int32), ("blocks_active", C.c_int32),
        ("sms_used", C.c_int32), ("planned_active", C.c_int32), ("elapsed_ms", C.c_double),
    ]


class ifr_block_log(C.Structure):
    _fields_ = [
        ("t_start_ns", C.c_uint64), ("t_end_ns", C.c_uint64), ("rounds", C.c_uint64), ("work", C.c_uint64),
        ("checksum", C.c_uint32), ("checksum2", C.c_uint32), ("smid", C.c_uint32), ("index", C.c_int32),
        ("status", C.c_int32), ("reserved", C.c_uint32),
    ]


class ifr_victim_cfg(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("repeats", C.c_int32), ("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int64),
        ("scalar", C.c_float), ("eps", C.c_float), ("in0", C.c_void_p), ("in1", C.c_void_p), ("out", C.c_void_p),
        ("grid", C.c_int32), ("block", C.c_int32), ("variant", C.c_int32), ("reserved", C.c_int32),
    ]


class ifr_timing(C.Structure):
    _fields_ = [
        ("t_start_ns", C.c_uint64), ("t_end_ns", C.c_uint64), ("event_ms", C.c_double), ("status", C.c_int32),
        ("sms_touched", C.c_int32), ("blocks", C.c_int32), ("repeats", C.c_int32),
    ]


class ifr_sweep_plan(C.Structure):
    _fields_ = [
        ("n_victims", C.c_int32), ("victims", C.POINTER(ifr_victim_cfg)), ("n_stressors", C.c_int32),
        ("n_levels", C.c_int32), ("levels", C.POINTER(ifr_stressor_cfg)), ("repeats", C.c_int32),
        ("batched", C.c_int32),
    ]


class ifr_cell_result(C.Structure):
    _fields_ = [
        ("victim", C.c_int32), ("stressor", C.c_int32), ("level", C.c_int32), ("repeat", C.c_int32),
        ("timing", ifr_timing), ("stress", ifr_stressor_result), ("valid", C.c_int32), ("status", C.c_int32),
    ]


class ifr_sensitivity_out(C.Structure):
    _fields_ = [
        ("n_stressors", C.c_int32), ("n_levels", C.c_int32), ("t0_ns", C.c_double), ("noise", C.c_double),
        ("slowdown", (C.c_double * (IFR_MAX_LEVELS + 1)) * IFR_MAX_STRESSORS),
        ("S", C.c_double * IFR_MAX_STRESSORS), ("auc", C.c_double * IFR_MAX_STRESSORS),
        ("monotone", C.c_int32 * IFR_MAX_STRESSORS), ("n_valid", C.c_int32), ("n_invalid", C.c_int32),
    ]


class ifr_kernel_profile(C.Structure):
    _fields_ = [
        ("grid", C.c_int32), ("block", C.c_int32), ("regs_per_thread", C.c_int32), ("static_smem", C.c_int32),
        ("dynamic_smem", C.c_int32), ("max_blocks_per_sm", C.c_int32), ("tmem_cols", C.c_int32),
        ("uses_tensor", C.c_int32), ("sm_count", C.c_int32), ("blocks_per_sm", C.c_int32), ("launches", C.c_int32),
        ("reserved", C.c_int32), ("bytes_per_launch", C.c_double), ("flops_per_launch", C.c_double),
    ]


class ifr_pair_result(C.Structure):
    _fields_ = [
        ("solo_a", ifr_stressor_result), ("solo_b", ifr_stressor_result), ("co_a", ifr_stressor_result),
        ("co_b", ifr_stressor_result), ("solo_a_ns", C.c_double), ("solo_b_ns", C.c_double),
        ("co_a_ns", C.c_double), ("co_b_ns", C.c_double), ("seq_ns", C.c_double), ("col_ns", C.c_double),
        ("overlapped", C.c_int32), ("status", C.c_int32),
    ]


class ifr_colocate_result(C.Structure):
    _fields_ = [
        ("victim_solo", ifr_timing), ("victim_co", ifr_timing), ("stress_solo", ifr_stressor_result),
        ("stress_co", ifr_stressor_result), ("victim_solo_ns", C.c_double), ("victim_co_ns", C.c_double),
        ("stress_solo_ns", C.c_double), ("stress_co_ns", C.c_double), ("blocked", C.c_int32), ("status", C.c_int32),
    ]


class ifr_partition_info(C.Structure):
    _fields_ = [("victim_sms", C.c_int32), ("stressor_sms", C.c_int32)]


class ifr_corun_result(C.Structure):
    _fields_ = [
        ("victim_solo", ifr_timing), ("corunner_solo", ifr_timing), ("victim_corun", ifr_timing),
        ("corunner_corun", ifr_timing), ("valid", C.c_int32), ("status", C.c_int32),
        ("corunner_launches", C.c_int32), ("blocked", C.c_int32), ("victim_release_ns", C.c_uint64),
        ("victim_slowdown", C.c_double), ("corunner_slowdown", C.c_double),
    ]


IFR_MLP_MAX_LAYERS = 8


class ifr_mlp(C.Structure):
    _fields_ = [
        ("n_layers", C.c_int32), ("batch", C.c_int32), ("dims", C.c_int32 * (IFR_MLP_MAX_LAYERS + 1)),
        ("W", C.c_void_p * IFR_MLP_MAX_LAYERS), ("b", C.c_void_p * IFR_MLP_MAX_LAYERS),
        ("H", C.c_void_p * IFR_MLP_MAX_LAYERS), ("Z", C.c_void_p * IFR_MLP_MAX_LAYERS),
        ("dW", C.c_void_p * IFR_MLP_MAX_LAYERS), ("db", C.c_void_p * IFR_MLP_MAX_LAYERS),
        ("dZ", C.c_void_p * IFR_MLP_MAX_LAYERS), ("dZh", C.c_void_p * IFR_MLP_MAX_LAYERS), ("dX", C.c_void_p),
    ]


STRUCTS = [ifr_device_info, ifr_stressor_cfg, ifr_stressor_result, ifr_block_log, ifr_victim_cfg, ifr_timing,
           ifr_sweep_plan, ifr_cell_result, ifr_sensitivity_out, ifr_kernel_profile, ifr_mlp, ifr_corun_result,
           ifr_pair_result, ifr_colocate_result, ifr_partition_info]

_lib = None


def load():
    """Load libifr.so (built in-tree by paper_2501_16909_b300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libifr.so is not built: run `python -m paper_2501_16909_b300.build` "
                           "(or __graft_entry__.build()); there is no fallback implementation")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp, i32 = C.c_void_p, C.c_int
    sig = {
        "ifr_init": (i32, [i32, P(vp)]),
        "ifr_shutdown": (None, [vp]),
        "ifr_strerror": (C.c_char_p, [i32]),
        "ifr_abi_version": (i32, []),
        "ifr_device_query": (i32, [vp, P(ifr_device_info)]),
        "ifr_launch_count": (i32, [vp, P(C.c_uint64)]),
        "ifr_stressor_launch": (i32, [vp, P(ifr_stressor_cfg), vp, P(i32)]),
        "ifr_stressor_stop": (i32, [vp, i32, vp]),
        "ifr_stressor_wait": (i32, [vp, i32, i32, P(ifr_stressor_result)]),
        "ifr_stressor_block_logs": (i32, [vp, i32, P(ifr_block_log), i32, P(i32)]),
        "ifr_stressor_release": (i32, [vp, i32]),
        "ifr_stream_stressor_noalloc": (i32, [i32, vp, C.c_int64, i32, i32, i32, C.c_int64, C.c_uint64, vp,
                                               vp, i32]),
        "ifr_victim_launch": (i32, [vp, P(ifr_victim_cfg), vp, P(ifr_timing)]),
        "ifr_sweep": (i32, [vp, P(ifr_sweep_plan), P(ifr_cell_result), C.c_size_t, P(C.c_size_t)]),
        "ifr_sensitivity": (i32, [P(ifr_cell_result), C.c_size_t, i32, i32, i32, P(C.c_double),
                                  P(ifr_sensitivity_out)]),
        "ifr_corun": (i32, [vp, P(ifr_victim_cfg), P(ifr_victim_cfg), i32, P(ifr_corun_result)]),
        "ifr_stressor_pair": (i32, [vp, P(ifr_stressor_cfg), P(ifr_stressor_cfg), P(ifr_pair_result)]),
        "ifr_colocate": (i32, [vp, P(ifr_stressor_cfg), P(ifr_victim_cfg), P(ifr_colocate_result)]),
        "ifr_partition": (i32, [vp, i32, i32, P(ifr_partition_info)]),
        "ifr_partition_release": (i32, [vp]),
        "ifr_victim_profile": (i32, [vp, P(ifr_victim_cfg), P(ifr_kernel_profile)]),
        "ifr_stressor_profile": (i32, [vp, P(ifr_stressor_cfg), P(ifr_kernel_profile)]),
        "ifr_mlp_forward": (i32, [vp, P(ifr_mlp), vp]),
        "ifr_mlp_backward": (i32, [vp, P(ifr_mlp), vp, vp]),
        "ifr_mse_grad": (i32, [vp, vp, vp, i32, vp, vp, vp]),
        "ifr_adam_step": (i32, [vp, vp, vp, vp, vp, vp, C.c_int64, C.c_float, C.c_float, C.c_float, C.c_float, i32,
                                vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class IfrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = load().ifr_strerror(status)
        super().__init__("%s: %s (%d)" % (what, msg.decode() if msg else "?", status))


def check(status: int, what: str) -> int:
    if status != IFR_OK:
        raise IfrError(status, what)
    return status

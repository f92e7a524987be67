"""B300-native interference-sensitivity toolkit (thin Python binding over libifr).

Everything that runs on the GPU runs in libifr's CUDA kernels; this package only
marshals arguments (torch tensors -> device pointers, dicts -> C structs) and
reads results back.  PyTorch supplies device memory and streams.

The method (Elvinger et al., "Understanding GPU Resource Interference One Level
Deeper", SoCC '25, Sec. 4.1): colocate a workload with stressors that each hold
one GPU resource at a constant interference level and measure its slowdown
against isolation, per resource.
"""
from __future__ import annotations

import ctypes as C
import math

from . import _abi
from ._abi import (IFR_OK, STRESSOR_NAMES, VICTIM_NAMES, IfrError, check, ifr_block_log, ifr_cell_result,
                   ifr_device_info, ifr_sensitivity_out, ifr_stressor_cfg, ifr_stressor_result, ifr_sweep_plan,
                   ifr_timing, ifr_victim_cfg)
from ._abi import *  # noqa: F401,F403  (status codes and kind constants)

__all__ = ["Context", "stressor_cfg", "victim_cfg", "ifr_sensitivity", "cells_to_dicts", "IfrError",
           "STRESSOR_NAMES", "VICTIM_NAMES"]


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(int(stream.cuda_stream))
    return C.c_void_p(int(stream))


def stressor_cfg(kind: int, **kw) -> ifr_stressor_cfg:
    """Build an ifr_stressor_cfg; `buf` may be a torch tensor."""
    c = ifr_stressor_cfg()
    c.kind = kind
    for k, v in kw.items():
        if k == "buf":
            c.buf = None if v is None else int(v.data_ptr())
        else:
            setattr(c, k, v)
    return c


def victim_cfg(kind: int, in0=None, in1=None, out=None, **kw) -> ifr_victim_cfg:
    """Build an ifr_victim_cfg from torch tensors and shape keywords."""
    c = ifr_victim_cfg()
    c.kind = kind
    c.in0 = None if in0 is None else int(in0.data_ptr())
    c.in1 = None if in1 is None else int(in1.data_ptr())
    c.out = None if out is None else int(out.data_ptr())
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _struct_dict(s):
    d = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        if isinstance(v, C.Structure):
            v = _struct_dict(v)
        elif isinstance(v, bytes):
            v = v.decode(errors="replace")
        d[name] = v
    return d


def cells_to_dicts(cells):
    """Flatten ifr_cell_result records into plain dicts (raw timestamps kept)."""
    out = []
    for c in cells:
        out.append(dict(
            victim=c.victim, stressor=c.stressor, level=c.level, repeat=c.repeat, k=c.timing.repeats,
            t_start=c.timing.t_start_ns, t_end=c.timing.t_end_ns, status=c.timing.status, valid=c.valid,
            cell_status=c.status, event_ms=c.timing.event_ms, sms_touched=c.timing.sms_touched,
            stress_status=c.stress.status, stress_blocks_active=c.stress.blocks_active,
            stress_t_start_last=c.stress.t_start_last_ns, stress_t_end_first=c.stress.t_end_first_ns,
            stress_t_start=c.stress.t_start_ns, stress_t_end=c.stress.t_end_ns, stress_work=c.stress.work,
            stress_rounds=c.stress.rounds, stress_checksum=c.stress.checksum, stress_sms=c.stress.sms_used,
        ))
    return out


class Context:
    """One libifr context on one CUDA device (ifr_init / ifr_shutdown)."""

    def __init__(self, device: int = 0):
        import torch

        torch.cuda.init()
        self._L = _abi.load()
        self._h = C.c_void_p()
        check(self._L.ifr_init(device, C.byref(self._h)), "ifr_init")
        info = ifr_device_info()
        check(self._L.ifr_device_query(self._h, C.byref(info)), "ifr_device_query")
        self.info = _struct_dict(info)
        self.device = device

    # -- lifecycle
    def close(self):
        if self._h:
            self._L.ifr_shutdown(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _sync():
        import torch

        torch.cuda.synchronize()

    def launch_count(self) -> int:
        n = C.c_uint64(0)
        check(self._L.ifr_launch_count(self._h, C.byref(n)), "ifr_launch_count")
        return int(n.value)

    # -- stressors
    def stressor_launch(self, cfg: ifr_stressor_cfg, stream=None) -> int:
        self._sync()
        h = C.c_int(-1)
        check(self._L.ifr_stressor_launch(self._h, C.byref(cfg), _stream_handle(stream), C.byref(h)),
              "ifr_stressor_launch")
        return h.value

    def stressor_stop(self, handle: int, stream=None):
        check(self._L.ifr_stressor_stop(self._h, handle, _stream_handle(stream)), "ifr_stressor_stop")

    def stressor_wait(self, handle: int, timeout_ms: int = 0, allow_timeout: bool = False) -> dict:
        r = ifr_stressor_result()
        st = self._L.ifr_stressor_wait(self._h, handle, timeout_ms, C.byref(r))
        if not (allow_timeout and st == _abi.IFR_ERR_TIMEOUT):
            check(st, "ifr_stressor_wait")
        d = _struct_dict(r)
        d["wait_status"] = st
        return d

    def stressor_block_logs(self, handle: int) -> list:
        n = C.c_int(0)
        cap = self.info["num_sms"] * 32
        arr = (ifr_block_log * cap)()
        check(self._L.ifr_stressor_block_logs(self._h, handle, arr, cap, C.byref(n)), "ifr_stressor_block_logs")
        return [_struct_dict(arr[i]) for i in range(n.value)]

    def stressor_release(self, handle: int):
        check(self._L.ifr_stressor_release(self._h, handle), "ifr_stressor_release")

    def run_stressor(self, cfg: ifr_stressor_cfg, timeout_ms: int = 0):
        """Launch, wait, collect logs, release: (result, logs)."""
        h = self.stressor_launch(cfg)
        try:
            r = self.stressor_wait(h, timeout_ms)
            logs = self.stressor_block_logs(h)
        finally:
            self.stressor_release(h)
        return r, logs

    # -- solo kernel profiles
    def victim_profile(self, cfg: ifr_victim_cfg) -> dict:
        p = _abi.ifr_kernel_profile()
        check(self._L.ifr_victim_profile(self._h, C.byref(cfg), C.byref(p)), "ifr_victim_profile")
        return _struct_dict(p)

    def stressor_profile(self, cfg: ifr_stressor_cfg) -> dict:
        p = _abi.ifr_kernel_profile()
        check(self._L.ifr_stressor_profile(self._h, C.byref(cfg), C.byref(p)), "ifr_stressor_profile")
        return _struct_dict(p)

    def stressor_pair(self, a: ifr_stressor_cfg, b: ifr_stressor_cfg) -> dict:
        """ifr_stressor_pair: A alone, B alone, then both released together (fixed work)."""
        self._sync()
        r = _abi.ifr_pair_result()
        check(self._L.ifr_stressor_pair(self._h, C.byref(a), C.byref(b), C.byref(r)), "ifr_stressor_pair")
        d = {k: getattr(r, k) for k, _ in r._fields_ if k not in ("solo_a", "solo_b", "co_a", "co_b")}
        for k in ("solo_a", "solo_b", "co_a", "co_b"):
            d[k] = _struct_dict(getattr(r, k))
        return d

    def colocate(self, stressor: ifr_stressor_cfg, victim: ifr_victim_cfg) -> dict:
        """ifr_colocate: victim alone, stressor alone, both released together (latency from release)."""
        self._sync()
        r = _abi.ifr_colocate_result()
        check(self._L.ifr_colocate(self._h, C.byref(stressor), C.byref(victim), C.byref(r)), "ifr_colocate")
        nested = ("victim_solo", "victim_co", "stress_solo", "stress_co")
        d = {k: getattr(r, k) for k, _ in r._fields_ if k not in nested}
        for k in nested:
            d[k] = _struct_dict(getattr(r, k))
        return d

    def partition(self, victim_sms: int, fine: bool = False) -> dict:
        """ifr_partition: green-context split, victims on one SM set, stressors on the other."""
        self._sync()
        info = _abi.ifr_partition_info()
        check(self._L.ifr_partition(self._h, victim_sms, 1 if fine else 0, C.byref(info)), "ifr_partition")
        return _struct_dict(info)

    def partition_release(self):
        check(self._L.ifr_partition_release(self._h), "ifr_partition_release")

    # -- victims
    def victim_launch(self, cfg: ifr_victim_cfg, stream=None) -> dict:
        self._sync()
        t = ifr_timing()
        check(self._L.ifr_victim_launch(self._h, C.byref(cfg), _stream_handle(stream), C.byref(t)),
              "ifr_victim_launch")
        return _struct_dict(t)

    # -- kernel-with-kernel colocation
    def corun(self, victim: ifr_victim_cfg, corunner: ifr_victim_cfg, corunner_launches: int = 0) -> dict:
        """Victim K launches beside a chain of co-runner launches; returns the raw
        timings plus the victim's slowdown and the chain's (reduced by ifr_corun)."""
        self._sync()
        r = _abi.ifr_corun_result()
        check(self._L.ifr_corun(self._h, C.byref(victim), C.byref(corunner), corunner_launches, C.byref(r)),
              "ifr_corun")
        return _struct_dict(r)

    # -- sweep
    def sweep(self, victims, levels, repeats: int = 3, batched: bool = False, grouped: bool = False):
        """victims: list of ifr_victim_cfg; levels: [n_stressors][n_levels] of
        ifr_stressor_cfg; grouped (with batched): grouped persistent victims.
        Returns the list of ifr_cell_result."""
        self._sync()
        nv = len(victims)
        ns = len(levels)
        nl = len(levels[0]) if ns else 0
        V = (ifr_victim_cfg * nv)(*victims)
        flat = [c for row in levels for c in row]
        S = (ifr_stressor_cfg * max(1, len(flat)))(*flat) if flat else (ifr_stressor_cfg * 1)()
        plan = ifr_sweep_plan(nv, V, ns, nl, S, repeats, (2 if grouped else 1) if batched else 0)
        cap = repeats * nv * (1 + ns * (nl + 1))
        cells = (ifr_cell_result * cap)()
        n = C.c_size_t(0)
        check(self._L.ifr_sweep(self._h, C.byref(plan), cells, cap, C.byref(n)), "ifr_sweep")
        return [cells[i] for i in range(n.value)]


def ifr_sensitivity(cells, victim: int, n_stressors: int, n_levels: int, intensity=None) -> dict:
    """Reduce cells (ifr_cell_result list) for one victim; returns a dict."""
    L = _abi.load()
    arr = (ifr_cell_result * max(1, len(cells)))(*cells)
    inten = None
    if intensity is not None:
        flat = [float(x) for row in intensity for x in row]
        inten = (C.c_double * len(flat))(*flat)
    out = ifr_sensitivity_out()
    check(L.ifr_sensitivity(arr, len(cells), victim, n_stressors, n_levels, inten, C.byref(out)), "ifr_sensitivity")
    L_ = n_levels
    return {
        "t0": out.t0_ns,
        "noise": out.noise,
        "slowdown": [[out.slowdown[r][l] for l in range(L_ + 1)] for r in range(n_stressors)],
        "S": [out.S[r] for r in range(n_stressors)],
        "auc": [out.auc[r] for r in range(n_stressors)],
        "monotone": [out.monotone[r] for r in range(n_stressors)],
        "n_valid": out.n_valid,
        "n_invalid": out.n_invalid,
    }


def isclose_nan(a, b, rel=1e-12):
    if isinstance(a, float) and math.isnan(a):
        return isinstance(b, float) and math.isnan(b)
    return math.isclose(a, b, rel_tol=rel, abs_tol=1e-15)

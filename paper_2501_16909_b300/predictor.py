"""Learned slowdown predictor — the kernel-level interference estimator of Sec. 5.1.

The paper proposes an estimator that collects each kernel's metrics and resource
sensitivity and predicts its slowdown under colocation; it gives no model.  Here a
pair (victim, co-runner) is described by 24 measured solo quantities of each side
(a profiler that replays kernels serialises them and cannot observe colocation,
Sec. 5.2, so every quantity comes from the library's own solo and probe runs):

* victim (VICTIM_FEATURES): its achieved fraction of the HBM, L2, tensor and FP32
  peaks (algorithmic bytes and flops over its measured solo time), that time, the
  SMs its blocks ran on, its measured sensitivity — the log slowdown beside each of
  the seven stressor kinds at full intensity (Sec. 5.1's "resource sensitivity") —
  and its launch shape (threads, registers, shared memory, occupancy, waves, TMEM);
* co-runner (CORUNNER_FEATURES): its measured solo fraction of each resource's peak
  (a stressor's rate over the peak of its resource, the HBM stream's rate also over
  the L2 peak since every byte crosses the L2; a kernel's algorithmic rates), its
  measured pressure — the log slowdown of each of six probe kernels run beside it —
  the SMs and blocks it held (from its block logs), and its launch shape.

The pair's 48 features are z-scored with the training statistics; the target is
the log of the measured slowdown.  The network is an MLP 48-256-256-256-1 with exact
GELU, bf16 weights and activations into the tensor cores with fp32 accumulation,
trained with Adam (lr 1e-3, batch 512) by the library's own kernels
(ifr_mlp_forward / backward, ifr_mse_grad, ifr_adam_step) behind a
torch.autograd.Function.  The baseline without the network ("the method without
it") predicts 1 + S_v,r(x): the victim's measured slowdown-minus-one curve for the
co-runner's resource r at the co-runner's solo fraction x of that resource.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _abi as A
from . import check

# kinds whose full-intensity slowdown makes up a victim's sensitivity vector, in order
SENSITIVITY_KINDS = [A.IFR_S_SCHED, A.IFR_S_FMA, A.IFR_S_TENSOR, A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W, A.IFR_S_L2,
                     A.IFR_S_HBM]
PROBES = ["hbm_triad", "l2_triad", "tensor_gemm", "smem_hist", "exp_softmax", "short_gemv"]

VICTIM_FEATURES = (["frac_hbm", "frac_l2", "frac_tensor", "frac_fp32", "log_duration_us", "sm_fraction"] +
                   ["log_sens_" + A.STRESSOR_NAMES[k] for k in SENSITIVITY_KINDS] +
                   ["threads_per_block", "regs_per_thread", "smem_per_block", "occupancy_blocks", "log_waves",
                    "tmem_cols", "uses_tensor", "log_bytes", "log_flops", "log_intensity", "thread_fill"])
CORUNNER_FEATURES = (["frac_hbm", "frac_l2", "frac_tensor", "frac_fp32", "frac_smem", "frac_sched"] +
                     ["log_pressure_" + p for p in PROBES] +
                     ["sm_fraction", "blocks_per_sm", "warps_per_sm", "threads_per_block", "regs_per_thread",
                      "smem_per_block", "tmem_cols", "occupancy_blocks", "log_rate", "log_solo_ms",
                      "pressure_max", "pressure_mean"])
assert len(VICTIM_FEATURES) == 24 and len(CORUNNER_FEATURES) == 24
RESOURCE_OF = {A.IFR_S_HBM: 0, A.IFR_S_L2: 1, A.IFR_S_TENSOR: 2, A.IFR_S_FMA: 3, A.IFR_S_SMEM_CF: 4,
               A.IFR_S_SMEM_32W: 4, A.IFR_S_SCHED: 5}


def _safe_log10(x):
    return math.log10(max(float(x), 1e-12))


def _log_slow(s):
    return math.log(max(float(s), 1e-3)) if s == s else 0.0  # NaN (no valid cell): no evidence


def _shape(prof, S, blocks=None):
    blocks = prof["grid"] if blocks is None else blocks
    occ = max(1, prof["max_blocks_per_sm"])
    return {
        "threads_per_block": prof["block"] / 1024.0,
        "regs_per_thread": prof["regs_per_thread"] / 255.0,
        "smem_per_block": (prof["static_smem"] + prof["dynamic_smem"]) / (228.0 * 1024),
        "occupancy_blocks": occ / 32.0,
        "log_waves": _safe_log10(blocks / (S * occ)),
        "tmem_cols": prof["tmem_cols"] / 512.0,
        "uses_tensor": float(prof["uses_tensor"]),
        "thread_fill": min(1.0, blocks * prof["block"] / (S * 2048.0)),
    }


def kernel_fracs(prof, solo_ns, pk):
    """Achieved fractions of the HBM, L2, tensor and FP32 peaks of one kernel launch:
    its algorithmic bytes and flops over its measured solo time."""
    T = max(solo_ns, 1.0) * 1e-9
    bps = prof["bytes_per_launch"] / T
    fps = prof["flops_per_launch"] / T
    return {"frac_hbm": bps / pk[A.IFR_S_HBM][0], "frac_l2": bps / pk[A.IFR_S_L2][0],
            "frac_tensor": fps / pk[A.IFR_S_TENSOR][0] if prof["uses_tensor"] else 0.0,
            "frac_fp32": 0.0 if prof["uses_tensor"] else fps / pk[A.IFR_S_FMA][0]}


def victim_features(prof, solo_ns, sms_touched, sens, pk, S):
    """24 measured features of a victim: profile, solo time per launch (ns), SMs its
    blocks ran on, and its sensitivity (slowdown beside each SENSITIVITY_KINDS
    stressor at full intensity)."""
    f = dict.fromkeys(VICTIM_FEATURES, 0.0)
    f.update({k: v for k, v in _shape(prof, S).items() if k in f})
    f.update(kernel_fracs(prof, solo_ns, pk))
    f["log_duration_us"] = _safe_log10(max(solo_ns, 1.0) * 1e-3)
    f["sm_fraction"] = min(1.0, sms_touched / S)
    for k, s in zip(SENSITIVITY_KINDS, sens):
        f["log_sens_" + A.STRESSOR_NAMES[k]] = _log_slow(s)
    f["log_bytes"] = _safe_log10(prof["bytes_per_launch"] + 1.0)
    f["log_flops"] = _safe_log10(prof["flops_per_launch"] + 1.0)
    f["log_intensity"] = _safe_log10(prof["flops_per_launch"] / max(prof["bytes_per_launch"], 1.0) + 1e-3)
    return np.array([f[k] for k in VICTIM_FEATURES], np.float64)


def _pressure(f, pressure):
    logs = [_log_slow(s) for s in pressure]
    for p, v in zip(PROBES, logs):
        f["log_pressure_" + p] = v
    f["pressure_max"] = max(logs)
    f["pressure_mean"] = sum(logs) / len(logs)


def stressor_corunner_features(prof, cfg, rate, frac_of_peak, pk, solo, pressure, S):
    """24 measured features of a stressor configuration as a co-runner: its solo rate
    and fraction of its resource's peak, `solo` (the fixed-work solo run's result:
    SMs used, active blocks, elapsed ms) and its pressure on the PROBES."""
    f = dict.fromkeys(CORUNNER_FEATURES, 0.0)
    slot = ["frac_hbm", "frac_l2", "frac_tensor", "frac_fp32", "frac_smem", "frac_sched"][RESOURCE_OF[cfg.kind]]
    f[slot] = frac_of_peak
    if cfg.kind == A.IFR_S_HBM:
        f["frac_l2"] = rate / pk[A.IFR_S_L2][0]  # every byte read from DRAM crosses the L2
    _pressure(f, pressure)
    f["sm_fraction"] = solo["sms_used"] / S
    f["blocks_per_sm"] = solo["blocks_active"] / S / 8.0
    f["warps_per_sm"] = solo["blocks_active"] * prof["block"] / 32.0 / S / 64.0
    f.update({k: v for k, v in _shape(prof, S).items() if k in f})
    f["log_rate"] = _safe_log10(rate)
    f["log_solo_ms"] = _safe_log10(solo["elapsed_ms"])
    return np.array([f[k] for k in CORUNNER_FEATURES], np.float64)


def kernel_corunner_features(prof, solo_ns, sms_touched, pressure, pk, S):
    """24 measured features of a kernel (a victim configuration) as a co-runner."""
    f = dict.fromkeys(CORUNNER_FEATURES, 0.0)
    f.update(kernel_fracs(prof, solo_ns, pk))
    f["frac_sched"] = prof["grid"] / (max(solo_ns, 1.0) * 1e-9) / pk[A.IFR_S_SCHED][0]
    _pressure(f, pressure)
    f["sm_fraction"] = min(1.0, sms_touched / S)
    blocks = min(prof["grid"], S * max(1, prof["max_blocks_per_sm"]))
    f["blocks_per_sm"] = blocks / S / 8.0
    f["warps_per_sm"] = blocks * prof["block"] / 32.0 / S / 64.0
    f.update({k: v for k, v in _shape(prof, S).items() if k in f})
    f["log_rate"] = _safe_log10((prof["bytes_per_launch"] + prof["flops_per_launch"]) / (max(solo_ns, 1.0) * 1e-9))
    f["log_solo_ms"] = _safe_log10(solo_ns * 1e-6)
    return np.array([f[k] for k in CORUNNER_FEATURES], np.float64)


# ----------------------------------------------------------------------------- the network
class PredictorMLP:
    """Flat fp32 master parameters + bf16 copy + gradients + Adam moments on the GPU,
    driven through the library's MLP kernels."""

    def __init__(self, ctx, dims=(48, 256, 256, 256, 1), seed=4, device="cuda"):
        self.ctx = ctx
        self.L = ctx._L
        self.dims = list(dims)
        self.nl = len(dims) - 1
        # PyTorch-style init U(-1/sqrt(fan_in), 1/sqrt(fan_in)) drawn from numpy's
        # default_rng(seed) in the order W0, b0, W1, b1, ...
        rng = np.random.default_rng(seed)
        host, self.offsets = [], []
        off = 0
        for fi, fo in zip(self.dims[:-1], self.dims[1:]):
            bound = 1.0 / math.sqrt(fi)
            W = rng.uniform(-bound, bound, (fo, fi))
            b = rng.uniform(-bound, bound, fo)
            wo = off
            off += fo * fi
            off += (-off) % 8
            bo = off
            off += fo
            off += (-off) % 8
            self.offsets.append((wo, bo))
            host.append((W, b))
        self.n = off
        self.w32 = torch.zeros(off, dtype=torch.float32, device=device)
        for (W, b), (wo, bo) in zip(host, self.offsets):
            self.w32[wo:wo + W.size] = torch.from_numpy(W.ravel()).float()
            self.w32[bo:bo + b.size] = torch.from_numpy(b).float()
        self.wbf = self.w32.to(torch.bfloat16)
        self.g = torch.zeros_like(self.w32)
        self.m = torch.zeros_like(self.w32)
        self.v = torch.zeros_like(self.w32)
        self.step_count = 0
        self.bufs = {}
        self.device = device

    # views
    def weight(self, l, dtype="f32"):
        fi, fo = self.dims[l], self.dims[l + 1]
        wo, _ = self.offsets[l]
        src = self.w32 if dtype == "f32" else self.wbf
        return src[wo:wo + fo * fi].view(fo, fi)

    def bias(self, l):
        _, bo = self.offsets[l]
        return self.w32[bo:bo + self.dims[l + 1]]

    def grad_views(self, l):
        fi, fo = self.dims[l], self.dims[l + 1]
        wo, bo = self.offsets[l]
        return self.g[wo:wo + fo * fi].view(fo, fi), self.g[bo:bo + fo]

    def _buffers(self, B):
        if B not in self.bufs:
            d = self.device
            H = [torch.zeros(B, self.dims[l], dtype=torch.bfloat16, device=d) for l in range(self.nl)]
            Z = [torch.zeros(B, self.dims[l + 1], dtype=torch.float32, device=d) for l in range(self.nl)]
            dZ = [torch.zeros(B, self.dims[l + 1], dtype=torch.float32, device=d) for l in range(self.nl)]
            dZh = [torch.zeros(B, self.dims[l + 1], dtype=torch.bfloat16, device=d) for l in range(self.nl)]
            dX = torch.zeros(B, self.dims[0], dtype=torch.float32, device=d)
            dY = torch.zeros(B, dtype=torch.float32, device=d)
            loss = torch.zeros(1, dtype=torch.float32, device=d)
            s = A.ifr_mlp()
            s.n_layers = self.nl
            s.batch = B
            for l, dim in enumerate(self.dims):
                s.dims[l] = dim
            for l in range(self.nl):
                wo, bo = self.offsets[l]
                s.W[l] = self.wbf.data_ptr() + 2 * wo
                s.b[l] = self.w32.data_ptr() + 4 * bo
                s.H[l] = H[l].data_ptr()
                s.Z[l] = Z[l].data_ptr()
                s.dW[l] = self.g.data_ptr() + 4 * wo
                s.db[l] = self.g.data_ptr() + 4 * bo
                s.dZ[l] = dZ[l].data_ptr()
                s.dZh[l] = dZh[l].data_ptr()
            s.dX = dX.data_ptr()
            self.bufs[B] = dict(H=H, Z=Z, dZ=dZ, dZh=dZh, dX=dX, dY=dY, loss=loss, s=s)
        return self.bufs[B]

    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def forward(self, x):
        """x: [B, dims[0]] (any float dtype) -> prediction [B] (fp32, a view of Z)."""
        B = x.shape[0]
        b = self._buffers(B)
        b["H"][0].copy_(x.to(torch.bfloat16))
        check(self.L.ifr_mlp_forward(self.ctx._h, C.byref(b["s"]), self._stream()), "ifr_mlp_forward")
        return b["Z"][-1].view(B)

    def backward(self, dY):
        """dY: [B] fp32 = dLoss/dprediction; fills self.g and the dX buffer."""
        B = dY.shape[0]
        b = self._buffers(B)
        b["dY"].copy_(dY)
        check(self.L.ifr_mlp_backward(self.ctx._h, C.byref(b["s"]), C.c_void_p(b["dY"].data_ptr()), self._stream()),
              "ifr_mlp_backward")
        return b["dX"]

    def mse_grad(self, target):
        B = target.shape[0]
        b = self._buffers(B)
        check(self.L.ifr_mse_grad(self.ctx._h, C.c_void_p(b["Z"][-1].data_ptr()), C.c_void_p(target.data_ptr()), B,
                                  C.c_void_p(b["dY"].data_ptr()), C.c_void_p(b["loss"].data_ptr()), self._stream()),
              "ifr_mse_grad")
        return b["dY"], b["loss"]

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        check(self.L.ifr_adam_step(self.ctx._h, C.c_void_p(self.w32.data_ptr()), C.c_void_p(self.g.data_ptr()),
                                   C.c_void_p(self.m.data_ptr()), C.c_void_p(self.v.data_ptr()),
                                   C.c_void_p(self.wbf.data_ptr()), self.n, lr, beta1, beta2, eps, self.step_count,
                                   self._stream()), "ifr_adam_step")


class MLPFunction(torch.autograd.Function):
    """y = MLP(x; w) with the library's forward and backward kernels.  `w` is the
    flat fp32 master parameter tensor of the model (its bf16 copy feeds the
    kernels), so autograd returns d(loss)/dw in the same flat layout."""

    @staticmethod
    def forward(fctx, x, w, model):
        model.wbf.copy_(w.detach().to(torch.bfloat16))
        y = model.forward(x)
        fctx.model = model
        return y.clone()

    @staticmethod
    def backward(fctx, gy):
        model = fctx.model
        dx = model.backward(gy.contiguous().float())
        return dx.clone(), model.g.clone(), None


# ----------------------------------------------------------------------------- training
def mape(pred, y):
    pred = np.asarray(pred, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.abs(pred - y) / y))


class Standardizer:
    """z-scores with the training statistics, clipped to +-Z_CLIP: a held-out kernel
    whose feature lies far outside the training range enters the network at the edge
    of that range instead of at a z-score of thousands.  A feature that is constant
    over the training rows (the fraction of a resource only the held-out stressor kind
    uses, say) taught the network nothing, so it enters as 0 for every row instead of
    as an input direction the network never saw vary."""

    Z_CLIP = 8.0

    def __init__(self, X):
        self.mu = X.mean(axis=0)
        sd = X.std(axis=0)
        self.live = sd >= 1e-9
        self.sd = np.where(self.live, sd, 1.0)

    def __call__(self, X):
        z = np.clip((X - self.mu) / self.sd, -self.Z_CLIP, self.Z_CLIP)
        return np.where(self.live, z, 0.0)


def train(model, Xtr, ytr, Xva, yva, lr=1e-3, batch=512, max_epochs=500, patience=20, seed=5, log=None):
    """Adam on MSE of log slowdown; early stop when validation MAPE stalls.
    X*: z-scored float arrays; y*: slowdowns (> 0).  Returns the history."""
    dev = model.device
    Xt = torch.tensor(Xtr, dtype=torch.float32, device=dev)
    yt = torch.tensor(np.log(ytr), dtype=torch.float32, device=dev)
    Xv = torch.tensor(Xva, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed)
    best, best_w, since, hist = math.inf, model.w32.clone(), 0, []
    n = Xt.shape[0]
    for ep in range(max_epochs):
        perm = torch.tensor(rng.permutation(n), device=dev)
        tot = 0.0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            model.forward(Xt[idx])
            _, loss = model.mse_grad(yt[idx].contiguous())
            model.backward(model._buffers(batch)["dY"])
            model.adam(lr)
            tot += float(loss.item()) if s == 0 else 0.0
        pv = predict(model, Xv)
        m = mape(pv, yva)
        hist.append((ep, m))
        if log:
            log(ep, m)
        if m < best - 1e-5:
            best, best_w, since = m, model.w32.clone(), 0
        else:
            since += 1
            if since >= patience:
                break
    model.w32.copy_(best_w)
    model.wbf.copy_(best_w.to(torch.bfloat16))
    return hist


def train_ensemble(ctx, Xtr, ytr, Xva, yva, members=5, seed=4, **kw):
    """`members` MLPs that differ only in their initial weights and batch order
    (seeds seed, seed + 1, ...), each trained like `train`."""
    models = []
    for i in range(members):
        m = PredictorMLP(ctx, seed=seed + i)
        train(m, Xtr, ytr, Xva, yva, seed=5 + i, **kw)
        models.append(m)
    return models


def predict_ensemble(models, X):
    """Geometric mean of the members' predicted slowdowns (the mean of their log)."""
    logs = np.stack([np.log(predict(m, X)) for m in models])
    return np.exp(logs.mean(axis=0))


# predicted log slowdowns are clamped to slowdowns in [1/4, 1000]: the measured ones
# lie within about 0.9 .. 60
LOG_SLOWDOWN_RANGE = (math.log(0.25), math.log(1000.0))


def predict(model, X, batch=512):
    X = torch.as_tensor(X, dtype=torch.float32, device=model.device)
    out = []
    for s in range(0, X.shape[0], batch):
        xb = X[s:s + batch]
        out.append(model.forward(xb).clone())
    return np.exp(np.clip(torch.cat(out).double().cpu().numpy(), *LOG_SLOWDOWN_RANGE))


# ----------------------------------------------------------------------------- baseline
def baseline_predict(curves, victim, resource, x):
    """1 + S_v,r(x): linear interpolation of the victim's measured slowdown-minus-one
    curve for resource r at the co-runner's solo fraction x (flat beyond the ends)."""
    xs, ss = curves[(victim, resource)]
    return 1.0 + float(np.interp(x, xs, ss))

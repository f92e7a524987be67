"""Learned slowdown predictor — the kernel-level interference estimator of Sec. 5.1.

The paper proposes an estimator that collects each kernel's metrics and resource
sensitivity and predicts its slowdown under colocation; it gives no model.  Here:

* every kernel (victim, or co-runner = a stressor configuration) gets a solo
  profile of 24 features (FEATURES): its achieved fraction of each resource's peak
  (HBM, L2, tensor pipe, FP32 pipe, shared-memory wavefronts, block dispatch) and
  its launch shape (threads, registers, shared memory, occupancy, waves, TMEM,
  SMs used, duty, ILP, bank-conflict degree, work and duration);
* a pair is the concatenation victim || co-runner (48 features, z-scored with the
  training statistics); the target is the log of the measured slowdown;
* the network is an MLP 48-256-256-256-1 with exact GELU, bf16 weights and
  activations into the tensor cores with fp32 accumulation, trained with Adam
  (lr 1e-3, batch 512) by the library's own kernels (ifr_mlp_forward / backward,
  ifr_mse_grad, ifr_adam_step) behind a torch.autograd.Function;
* the baseline without the network ("the method without it") predicts
  1 + S_v,r(x): the victim's measured slowdown-minus-one curve for the co-runner's
  resource r, interpolated at the co-runner's solo fraction x of that resource.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _abi as A
from . import check

FEATURES = [
    "frac_hbm", "frac_l2", "frac_tensor", "frac_fp32", "frac_smem", "frac_sched", "conflict_degree",
    "sm_fraction", "threads_per_block", "regs_per_thread", "smem_per_block", "occupancy_blocks",
    "warps_per_sm", "log_waves", "tmem_cols", "uses_tensor", "log_intensity", "log_duration_us", "duty", "ilp",
    "log_bytes", "log_flops", "is_stressor", "thread_fill",
]
RESOURCE_OF = {A.IFR_S_HBM: 0, A.IFR_S_L2: 1, A.IFR_S_TENSOR: 2, A.IFR_S_FMA: 3, A.IFR_S_SMEM_CF: 4,
               A.IFR_S_SMEM_32W: 4, A.IFR_S_SCHED: 5}


def _safe_log10(x):
    return math.log10(max(float(x), 1e-12))


def _shape_features(prof, S, grid_blocks_active=None):
    blocks = prof["grid"] if grid_blocks_active is None else grid_blocks_active
    occ = max(1, prof["max_blocks_per_sm"])
    resident = min(occ, max(1, math.ceil(blocks / S)))
    return {
        "threads_per_block": prof["block"] / 1024.0,
        "regs_per_thread": prof["regs_per_thread"] / 255.0,
        "smem_per_block": (prof["static_smem"] + prof["dynamic_smem"]) / (228.0 * 1024),
        "occupancy_blocks": occ / 32.0,
        "warps_per_sm": resident * prof["block"] / 32.0 / 64.0,
        "log_waves": _safe_log10(blocks / (S * occ)),
        "tmem_cols": prof["tmem_cols"] / 512.0,
        "uses_tensor": float(prof["uses_tensor"]),
        "thread_fill": min(1.0, blocks * prof["block"] / (S * 2048.0)),
    }


def victim_features(prof, solo_ns, pk, S):
    """24 features of a victim from its profile and solo duration per launch (ns)."""
    T = max(solo_ns, 1.0) * 1e-9
    bps = prof["bytes_per_launch"] / T
    fps = prof["flops_per_launch"] / T
    f = dict.fromkeys(FEATURES, 0.0)
    f.update(_shape_features(prof, S))
    f["frac_hbm"] = bps / pk[A.IFR_S_HBM][0]
    f["frac_l2"] = bps / pk[A.IFR_S_L2][0]
    if prof["uses_tensor"]:
        f["frac_tensor"] = fps / pk[A.IFR_S_TENSOR][0]
    else:
        f["frac_fp32"] = fps / pk[A.IFR_S_FMA][0]
    f["frac_sched"] = prof["grid"] / T / pk[A.IFR_S_SCHED][0]
    f["sm_fraction"] = min(1.0, prof["grid"] / S)
    f["log_intensity"] = _safe_log10(prof["flops_per_launch"] / max(prof["bytes_per_launch"], 1.0) + 1e-3)
    f["log_duration_us"] = _safe_log10(T * 1e6)
    f["log_bytes"] = _safe_log10(prof["bytes_per_launch"] + 1.0)
    f["log_flops"] = _safe_log10(prof["flops_per_launch"] + 1.0)
    return np.array([f[k] for k in FEATURES], np.float64)


def stressor_features(prof, cfg, frac_of_peak, S):
    """24 features of a stressor configuration from its profile and solo fraction of peak."""
    f = dict.fromkeys(FEATURES, 0.0)
    active = cfg.sm_count * max(1, prof["blocks_per_sm"])
    f.update(_shape_features(prof, S, active if cfg.kind != A.IFR_S_SCHED else None))
    slot = ["frac_hbm", "frac_l2", "frac_tensor", "frac_fp32", "frac_smem", "frac_sched"][RESOURCE_OF[cfg.kind]]
    f[slot] = frac_of_peak
    if cfg.kind == A.IFR_S_HBM:
        f["frac_l2"] = frac_of_peak * 0.4  # every DRAM byte also crosses L2
    if cfg.kind in (A.IFR_S_SMEM_CF, A.IFR_S_SMEM_32W):
        f["conflict_degree"] = (cfg.smem_ways or (1 if cfg.kind == A.IFR_S_SMEM_CF else 32)) / 32.0
    f["sm_fraction"] = cfg.sm_count / S
    f["duty"] = cfg.duty if 0.0 < cfg.duty < 1.0 else 1.0
    f["ilp"] = (cfg.ilp or 4) / 8.0 if cfg.kind == A.IFR_S_FMA else 0.0
    f["is_stressor"] = 1.0
    return np.array([f[k] for k in FEATURES], np.float64)


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
    def __init__(self, X):
        self.mu = X.mean(axis=0)
        self.sd = X.std(axis=0)
        self.sd[self.sd < 1e-9] = 1.0

    def __call__(self, X):
        return (X - self.mu) / self.sd


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


def predict(model, X, batch=512):
    X = torch.as_tensor(X, dtype=torch.float32, device=model.device)
    out = []
    for s in range(0, X.shape[0], batch):
        xb = X[s:s + batch]
        out.append(model.forward(xb).clone())
    return np.exp(torch.cat(out).double().cpu().numpy())


# ----------------------------------------------------------------------------- baseline
def baseline_predict(curves, victim, resource, x):
    """1 + S_v,r(x): linear interpolation of the victim's measured slowdown-minus-one
    curve for resource r at the co-runner's solo fraction x (flat beyond the ends)."""
    xs, ss = curves[(victim, resource)]
    return 1.0 + float(np.interp(x, xs, ss))

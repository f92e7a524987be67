"""Slowdown-predictor MLP in fp64 numpy — oracle (test infrastructure).

The paper proposes (Sec. 5.1) a kernel-level interference estimator that
collects each kernel's metrics and resource sensitivity and predicts its
slowdown under colocation; it gives no model.  The reading used here is a
multilayer perceptron on the concatenated solo profiles of a victim and a
co-runner:

    h_0 = x                                  (48 features)
    z_l = h_l W_l^T + b_l,  h_{l+1} = GELU(z_l)   for hidden layers
    y_hat = z_last[:, 0]                      (predicted log slowdown)
    loss = mean((y_hat - log slowdown)^2)

GELU is the exact form 0.5 x (1 + erf(x / sqrt 2)).  Adam follows Kingma & Ba
(2015) with PyTorch's defaults (beta 0.9 / 0.999, eps 1e-8 added after the
square root, no weight decay).  Weights are stored [out][in] as in a linear
layer.

With ``bf16=True`` every GEMM operand is first rounded to bf16 (round to
nearest even), the way the tensor-core kernels consume them: the layer input
and weight in the forward pass, and the pre-activation gradient, weight and
layer input in the backward pass.  With ``bf16=False`` the network is a smooth
fp64 function, which is what the finite-difference pins check.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to fp32 and then to the nearest bf16 value (ties to even), as a
    kernel holding fp32 values does; returned as float64."""
    b = np.ascontiguousarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    rnd = ((b >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    r = ((b + rnd) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def _q(a, bf16):
    return round_bf16(a) if bf16 else np.asarray(a, np.float64)


def forward(params, x, bf16=False):
    """params: list of (W [out,in], b [out]).  Returns (y_hat, cache)."""
    h = np.asarray(x, np.float64)
    cache = []
    n = len(params)
    for l, (W, b) in enumerate(params):
        hin = _q(h, bf16)
        Wq = _q(W, bf16)
        z = hin @ Wq.T + np.asarray(b, np.float64)
        cache.append((hin, Wq, z))
        h = gelu(z) if l < n - 1 else z
    return h[:, 0], cache


def loss(y_hat, target):
    d = y_hat - target
    return float(np.mean(d * d))


def backward(params, cache, y_hat, target, bf16=False):
    """Gradients of the mean-squared loss; returns [(dW, db)] per layer and dX."""
    B = y_hat.shape[0]
    n = len(params)
    dz = (2.0 / B) * (y_hat - target)[:, None]
    grads = [None] * n
    dx = None
    for l in range(n - 1, -1, -1):
        hin, Wq, z = cache[l]
        if l < n - 1:
            dz = dz * gelu_grad(z)
        dzq = _q(dz, bf16)
        dW = dzq.T @ hin
        db = dz.sum(axis=0)
        grads[l] = (dW, db)
        dx = dzq @ Wq
        dz = dx
    return grads, dx


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based).  Returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(dims, seed=4):
    """PyTorch-style linear init U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a numpy RNG."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(dims[:-1], dims[1:]):
        bound = 1.0 / np.sqrt(fi)
        params.append((rng.uniform(-bound, bound, (fo, fi)), rng.uniform(-bound, bound, fo)))
    return params

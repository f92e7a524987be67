"""GPU tests of the slowdown-predictor kernels (forward, backward, MSE gradient,
Adam) and of their torch.autograd.Function wrapper.

Tolerances.  The kernels feed bf16 operands (weights, activations, dZ) to the
tensor cores with fp32 accumulation; the oracle in bf16 mode, and a PyTorch
reference that rounds at the same points, round the same operands, so the
remaining differences are fp32 accumulation order and erff vs erf, which can flip
the bf16 rounding of an occasional activation (one bf16 ulp, 2^-8 relative).
Forward outputs: 1e-2 x max(|r|, rms r).  Gradients: relative Frobenius error
1e-3 against the bf16-mode oracle and the bf16-rounding PyTorch reference; 1e-2
against central finite differences of the smooth fp64 network; 5e-2 against
PyTorch autograd of the smooth network, where the activations' bf16 rounding
itself (2^-9 relative per activation, on every layer) is the difference.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as OM
import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import predictor as PR
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
DIMS = (48, 256, 256, 256, 1)


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ifr.Context(0)
    yield c
    c.close()


def _oracle_params(model):
    return [(model.weight(l).double().cpu().numpy(), model.bias(l).double().cpu().numpy())
            for l in range(model.nl)]


def _data(B, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, DIMS[0]))
    t = rng.standard_normal(B) * 0.3
    return x, t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [512, 37])
def test_forward_matches_oracle_bf16(ctx, B):
    model = PR.PredictorMLP(ctx, DIMS, seed=4)
    x, _ = _data(B)
    y = model.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    r, _ = OM.forward(_oracle_params(model), x, bf16=True)
    rms = np.sqrt(np.mean(r * r))
    assert np.all(np.abs(y - r) <= 1e-2 * np.maximum(np.abs(r), rms))


def test_backward_matches_oracle_bf16(ctx):
    B = 512
    model = PR.PredictorMLP(ctx, DIMS, seed=4)
    x, t = _data(B, 1)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    model.forward(xt)
    dY, loss = model.mse_grad(tt)
    dX = model.backward(dY).double().cpu().numpy()
    P = _oracle_params(model)
    yr, cache = OM.forward(P, x, bf16=True)
    assert abs(float(loss.item()) - OM.loss(yr, t)) <= 1e-2 * OM.loss(yr, t)
    grads, dx_r = OM.backward(P, cache, yr, t, bf16=True)
    for l in range(model.nl):
        gW, gb = model.grad_views(l)
        assert _rel(gW.double().cpu().numpy(), grads[l][0]) <= 1e-3, (l, _rel(gW.double().cpu().numpy(), grads[l][0]))
        assert _rel(gb.double().cpu().numpy(), grads[l][1]) <= 1e-3, (l, _rel(gb.double().cpu().numpy(), grads[l][1]))
    assert _rel(dX, dx_r) <= 1e-3, _rel(dX, dx_r)


def test_autograd_function_vs_torch_reference(ctx):
    B = 256
    model = PR.PredictorMLP(ctx, DIMS, seed=7)
    x, t = _data(B, 2)
    w = model.w32.clone().requires_grad_(True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    y = PR.MLPFunction.apply(xt, w, model)
    loss = ((y - torch.tensor(t, dtype=torch.float32, device="cuda")) ** 2).mean()
    loss.backward()
    # PyTorch reference in fp64 on the CPU, weights and input rounded to bf16 once
    h = torch.tensor(x).to(torch.bfloat16).double().requires_grad_(True)
    params = []
    a = h
    for l in range(model.nl):
        W = model.weight(l).detach().cpu().to(torch.bfloat16).double().requires_grad_(True)
        b = model.bias(l).detach().cpu().double().requires_grad_(True)
        params.append((W, b))
        z = a @ W.T + b
        a = torch.nn.functional.gelu(z) if l < model.nl - 1 else z
    ref = ((a[:, 0] - torch.tensor(t)) ** 2).mean()
    ref.backward()
    assert abs(float(loss.detach()) - float(ref.detach())) <= 2e-2 * float(ref.detach())
    g = w.grad.double().cpu()
    for l, (W, b) in enumerate(params):
        wo, bo = model.offsets[l]
        gw = g[wo:wo + W.numel()].view_as(W)
        gb = g[bo:bo + b.numel()]
        assert _rel(gw.numpy(), W.grad.numpy()) <= 5e-2, l
        assert _rel(gb.numpy(), b.grad.numpy()) <= 5e-2, l
    assert _rel(xt.grad.double().cpu().numpy(), h.grad.numpy()) <= 5e-2


def _q_bf16(t):
    """Round fp64 values to fp32 and then to bf16 (nearest even), as a kernel holding
    fp32 values does before feeding them to the tensor cores."""
    return t.float().to(torch.bfloat16).double()


class _RoundFwd(torch.autograd.Function):
    """bf16 rounding of an operand in the forward pass; the gradient passes through."""

    @staticmethod
    def forward(fctx, x):
        return _q_bf16(x)

    @staticmethod
    def backward(fctx, g):
        return g


class _Linear(torch.autograd.Function):
    """z = h W^T + b with bf16 operands h, W (already rounded) whose backward rounds
    dZ to bf16 for the two GEMMs (dW = dZ^T h, dh = dZ W) and sums the unrounded dZ
    for the bias, as the library's backward kernels do."""

    @staticmethod
    def forward(fctx, h, W, b):
        fctx.save_for_backward(h, W)
        return h @ W.T + b

    @staticmethod
    def backward(fctx, dz):
        h, W = fctx.saved_tensors
        dzq = _q_bf16(dz)
        return dzq @ W, dzq.T @ h, dz.sum(dim=0)


def test_autograd_function_vs_bf16_rounding_torch_reference(ctx):
    """PyTorch autograd in fp64 through a network that rounds to bf16 exactly where
    the kernels do (layer inputs, weights and dZ), held to 1e-3."""
    B = 512
    model = PR.PredictorMLP(ctx, DIMS, seed=8)
    x, t = _data(B, 4)
    w = model.w32.clone().requires_grad_(True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    y = PR.MLPFunction.apply(xt, w, model)
    loss = ((y - torch.tensor(t, dtype=torch.float32, device="cuda")) ** 2).mean()
    loss.backward()
    h = torch.tensor(x).float().double().requires_grad_(True)
    a = h
    params = []
    for l in range(model.nl):
        W = model.weight(l).detach().cpu().double().requires_grad_(True)
        b = model.bias(l).detach().cpu().double().requires_grad_(True)
        params.append((W, b))
        z = _Linear.apply(_RoundFwd.apply(a), _RoundFwd.apply(W), b)
        a = torch.nn.functional.gelu(z) if l < model.nl - 1 else z
    ref = ((a[:, 0] - torch.tensor(t)) ** 2).mean()
    ref.backward()
    assert abs(float(loss.detach()) - float(ref.detach())) <= 1e-3 * float(ref.detach())
    g = w.grad.double().cpu()
    for l, (W, b) in enumerate(params):
        wo, bo = model.offsets[l]
        gw = g[wo:wo + W.numel()].view_as(W)
        gb = g[bo:bo + b.numel()]
        assert _rel(gw.numpy(), W.grad.numpy()) <= 1e-3, (l, _rel(gw.numpy(), W.grad.numpy()))
        assert _rel(gb.numpy(), b.grad.numpy()) <= 1e-3, (l, _rel(gb.numpy(), b.grad.numpy()))
    assert _rel(xt.grad.double().cpu().numpy(), h.grad.numpy()) <= 1e-3


def test_directional_finite_differences_1k(ctx):
    """Central differences (h = 1e-3 along random unit directions of the fp32
    master weights) of the smooth fp64 network on 1000 samples, against the
    kernels' gradient projected on the same directions."""
    B = 1000
    model = PR.PredictorMLP(ctx, DIMS, seed=9)
    x, t = _data(B, 3)
    model.forward(torch.tensor(x, dtype=torch.float32, device="cuda"))
    dY, _ = model.mse_grad(torch.tensor(t, dtype=torch.float32, device="cuda"))
    model.backward(dY)
    g = model.g.double().cpu().numpy()
    w0 = model.w32.double().cpu().numpy()
    rng = np.random.default_rng(0)

    def loss_at(w):
        P = []
        for l in range(model.nl):
            wo, bo = model.offsets[l]
            fi, fo = DIMS[l], DIMS[l + 1]
            P.append((w[wo:wo + fo * fi].reshape(fo, fi), w[bo:bo + fo]))
        return OM.loss(OM.forward(P, x)[0], t)

    h = 1e-3
    fd, an = [], []
    for _ in range(6):
        d = rng.standard_normal(w0.size)
        d /= np.linalg.norm(d)
        fd.append((loss_at(w0 + h * d) - loss_at(w0 - h * d)) / (2 * h))
        an.append(float(g @ d))
    fd, an = np.array(fd), np.array(an)
    assert _rel(an, fd) <= 1e-2, (_rel(an, fd), an, fd)


def test_adam_matches_oracle(ctx):
    model = PR.PredictorMLP(ctx, DIMS, seed=1)
    rng = np.random.default_rng(3)
    w = model.w32.double().cpu().numpy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for step in range(1, 4):
        g = rng.standard_normal(w.size) * 0.01
        model.g.copy_(torch.tensor(g, dtype=torch.float32))
        model.adam(1e-3)
        w, m, v = OM.adam_step(w, g.astype(np.float32).astype(np.float64), m, v, step)
    got = model.w32.double().cpu().numpy()
    assert np.max(np.abs(got - w)) <= 1e-6
    assert torch.equal(model.wbf, model.w32.to(torch.bfloat16))


def test_training_reduces_error(ctx):
    rng = np.random.default_rng(11)
    n = 4096
    X = rng.standard_normal((n, 48))
    y = np.exp(0.3 * np.tanh(X[:, 0] + 0.5 * X[:, 1] * X[:, 2]) + 0.2)
    model = PR.PredictorMLP(ctx, DIMS, seed=4)
    before = PR.mape(PR.predict(model, X[3500:]), y[3500:])
    hist = PR.train(model, X[:3000], y[:3000], X[3000:3500], y[3000:3500], max_epochs=40, patience=10)
    after = PR.mape(PR.predict(model, X[3500:]), y[3500:])
    assert after < 0.4 * before, (before, after, hist[-3:])


def test_ensemble_is_geometric_mean_of_members(ctx):
    rng = np.random.default_rng(12)
    n = 2048
    X = rng.standard_normal((n, 48))
    y = np.exp(0.3 * np.tanh(X[:, 0] - X[:, 3]) + 0.1)
    models = PR.train_ensemble(ctx, X[:1500], y[:1500], X[1500:1800], y[1500:1800], members=2, max_epochs=10,
                               patience=5)
    assert len(models) == 2
    p0, p1 = PR.predict(models[0], X[1800:]), PR.predict(models[1], X[1800:])
    assert not np.allclose(p0, p1)  # members start from different weights
    pe = PR.predict_ensemble(models, X[1800:])
    np.testing.assert_allclose(pe, np.sqrt(p0 * p1), rtol=1e-12)

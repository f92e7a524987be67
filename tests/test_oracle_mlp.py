"""Pins for the fp64 MLP oracle: finite differences, closed forms, and PyTorch's
autograd as an independent implementation."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _data(B=16, dims=(48, 32, 32, 1), seed=1):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(list(dims), seed=seed)
    x = rng.standard_normal((B, dims[0]))
    t = rng.standard_normal(B) * 0.3
    return params, x, t


def test_gelu_closed_forms():
    # GELU(x) = x * Phi(x): Phi(0) = 1/2, Phi(1) = 0.8413447460685429
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert mlp.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert mlp.gelu(np.array(-1.0)) == pytest.approx(-(1 - 0.8413447460685429), abs=1e-15)
    assert mlp.gelu_grad(np.array(0.0)) == 0.5
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, rtol=0, atol=1e-8)


def test_backward_matches_finite_differences():
    params, x, t = _data()
    y, cache = mlp.forward(params, x)
    grads, dx = mlp.backward(params, cache, y, t)
    h = 1e-6
    rng = np.random.default_rng(0)
    for l, (W, b) in enumerate(params):
        for _ in range(4):
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            Wp = [(w.copy(), bb.copy()) for w, bb in params]
            Wm = [(w.copy(), bb.copy()) for w, bb in params]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (mlp.loss(mlp.forward(Wp, x)[0], t) - mlp.loss(mlp.forward(Wm, x)[0], t)) / (2 * h)
            assert grads[l][0][i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        i = rng.integers(b.shape[0])
        Pp = [(w.copy(), bb.copy()) for w, bb in params]
        Pm = [(w.copy(), bb.copy()) for w, bb in params]
        Pp[l][1][i] += h
        Pm[l][1][i] -= h
        fd = (mlp.loss(mlp.forward(Pp, x)[0], t) - mlp.loss(mlp.forward(Pm, x)[0], t)) / (2 * h)
        assert grads[l][1][i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # input gradient
    xp, xm = x.copy(), x.copy()
    xp[3, 5] += h
    xm[3, 5] -= h
    fd = (mlp.loss(mlp.forward(params, xp)[0], t) - mlp.loss(mlp.forward(params, xm)[0], t)) / (2 * h)
    assert dx[3, 5] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_forward_backward_match_torch_autograd():
    params, x, t = _data(B=32)
    y, cache = mlp.forward(params, x)
    grads, _ = mlp.backward(params, cache, y, t)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    h = torch.tensor(x)
    for l, (W, b) in enumerate(tp):
        z = h @ W.T + b
        h = torch.nn.functional.gelu(z) if l < len(tp) - 1 else z
    L = ((h[:, 0] - torch.tensor(t)) ** 2).mean()
    L.backward()
    assert np.allclose(y, h[:, 0].detach().numpy(), rtol=1e-12, atol=1e-14)
    for (dW, db), (W, b) in zip(grads, tp):
        assert np.allclose(dW, W.grad.numpy(), rtol=1e-10, atol=1e-14)
        assert np.allclose(db, b.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_bf16_rounding_is_applied_and_matches_torch():
    v = np.random.default_rng(3).standard_normal(1000)
    ours = mlp.round_bf16(v)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(ours, ref)
    params, x, t = _data()
    y0, _ = mlp.forward(params, x)
    y1, _ = mlp.forward(params, x, bf16=True)
    assert not np.array_equal(y0, y1)
    assert np.allclose(y0, y1, rtol=0.05, atol=0.05)


def test_adam_first_step_closed_form_and_torch():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    w1, m1, v1 = mlp.adam_step(w, g, m, v, 1, lr=1e-3)
    # step 1: mhat = g, vhat = g^2, update = lr * g / (|g| + eps)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-16)
    tw = torch.tensor(w, requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-3)
    wn, mn, vn = w.copy(), m, v
    for step in range(1, 6):
        gg = g * step
        tw.grad = torch.tensor(gg)
        opt.step()
        wn, mn, vn = mlp.adam_step(wn, gg, mn, vn, step, lr=1e-3)
    assert np.allclose(wn, tw.detach().numpy(), rtol=1e-12, atol=1e-15)

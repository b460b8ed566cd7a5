"""Pins of the network oracle (oracle/cnn.py): library routines (torch conv2d
with circular padding, torch GELU, torch Adam, all FP64 on the CPU) and finite
differences of the full network."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import cnn


def test_conv_matches_torch_circular():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 9, 7))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = F.conv2d(F.pad(torch.from_numpy(x), (1, 1, 1, 1), mode="circular"),
                   torch.from_numpy(W), torch.from_numpy(b)).numpy()
    assert np.allclose(cnn.conv(x, W, b), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_dilated_conv_matches_torch_circular(d):
    rng = np.random.default_rng(d)
    x = rng.standard_normal((2, 3, 16, 13))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = F.conv2d(F.pad(torch.from_numpy(x), (d, d, d, d), mode="circular"),
                   torch.from_numpy(W), torch.from_numpy(b), dilation=d).numpy()
    assert np.allclose(cnn.conv(x, W, b, d), ref, rtol=0, atol=1e-12)


def test_dilated_backward_matches_autograd():
    rng = np.random.default_rng(4)
    widths, dil = (1, 3, 3, 1), (1, 3, 2)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in cnn.init_params(rng, widths)]
    x = rng.standard_normal((2, 1, 12, 12))
    t = rng.standard_normal((2, 1, 12, 12))
    y, cache = cnn.forward(params, x, dil)
    L, dy = cnn.mse(y, t)
    grads = cnn.backward(params, cache, dy, dil)
    tp = [(torch.from_numpy(W).requires_grad_(True), torch.from_numpy(b).requires_grad_(True))
          for W, b in params]
    h = torch.from_numpy(x)
    for li, (W, b) in enumerate(tp):
        d = dil[li]
        h = F.conv2d(F.pad(h, (d, d, d, d), mode="circular"), W, b, dilation=d)
        if li < len(tp) - 1:
            h = F.gelu(h)
    ((h - torch.from_numpy(t)) ** 2).mean().backward()
    for (dW, db), (W, b) in zip(grads, tp):
        assert np.allclose(dW, W.grad.numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(db, b.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_gelu_matches_torch():
    z = np.linspace(-6, 6, 1001)
    ref = F.gelu(torch.from_numpy(z)).numpy()
    assert np.allclose(cnn.gelu(z), ref, rtol=0, atol=1e-14)
    zt = torch.from_numpy(z).requires_grad_(True)
    F.gelu(zt).sum().backward()
    assert np.allclose(cnn.gelu_grad(z), zt.grad.numpy(), rtol=0, atol=1e-14)


def test_backward_matches_autograd_and_finite_differences():
    rng = np.random.default_rng(1)
    widths = (1, 4, 4, 1)
    params = cnn.init_params(rng, widths)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    x = rng.standard_normal((2, 1, 8, 8))
    t = rng.standard_normal((2, 1, 8, 8))
    y, cache = cnn.forward(params, x)
    L, dy = cnn.mse(y, t)
    grads = cnn.backward(params, cache, dy)
    # autograd on the same definition built from torch ops (library routine)
    tp = [(torch.from_numpy(W).requires_grad_(True), torch.from_numpy(b).requires_grad_(True))
          for W, b in params]
    h = torch.from_numpy(x)
    for li, (W, b) in enumerate(tp):
        h = F.conv2d(F.pad(h, (1, 1, 1, 1), mode="circular"), W, b)
        if li < len(tp) - 1:
            h = F.gelu(h)
    Lt = ((h - torch.from_numpy(t)) ** 2).mean()
    Lt.backward()
    assert abs(float(Lt) - L) < 1e-12
    for (dW, db), (W, b) in zip(grads, tp):
        assert np.allclose(dW, W.grad.numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(db, b.grad.numpy(), rtol=1e-10, atol=1e-12)
    # central finite differences on a few weights of each layer
    for li in range(len(params)):
        W, b = params[li]
        for idx in [(0, 0, 1, 1), (W.shape[0] - 1, W.shape[1] - 1, 2, 0)]:
            Wp, Wm = W.copy(), W.copy()
            eps = 1e-6
            Wp[idx] += eps
            Wm[idx] -= eps
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            Lp, _ = cnn.mse(cnn.forward(pp, x)[0], t)
            Lm, _ = cnn.mse(cnn.forward(pm, x)[0], t)
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_matches_torch():
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(10)
    gs = [rng.standard_normal(10) for _ in range(5)]
    tp = torch.from_numpy(p0.copy()).requires_grad_(True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(10), np.zeros(10)
    for k, g in enumerate(gs, start=1):
        opt.zero_grad()
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = cnn.adam_step(p, g, m, v, k, 1e-2)
    assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", ["tap", "gelu_prime", "weight_grad_shift"])
def test_pins_catch_planted_mistakes(name, monkeypatch):
    """Plant a mistake in the oracle (CPU) and check a pin fails."""
    if name == "tap":
        orig = cnn.conv
        monkeypatch.setattr(cnn, "conv", lambda x, W, b, d=1: orig(x, W[:, :, ::-1, :].copy(), b, d))
        with pytest.raises(AssertionError):
            test_conv_matches_torch_circular()
    elif name == "gelu_prime":
        monkeypatch.setattr(cnn, "gelu_grad", lambda z: 0.5 * (1.0 + np.tanh(z)))
        with pytest.raises(AssertionError):
            test_backward_matches_autograd_and_finite_differences()
    else:
        orig = cnn.conv_weight_grad
        def bad(g, x, d=1):
            dW, db = orig(g, x, d)
            return dW[:, :, ::-1, ::-1].copy(), db
        monkeypatch.setattr(cnn, "conv_weight_grad", bad)
        with pytest.raises(AssertionError):
            test_backward_matches_autograd_and_finite_differences()

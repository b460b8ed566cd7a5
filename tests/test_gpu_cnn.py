"""GPU parity of the learned-guess network kernels (px_cnn_*) against the FP64
network oracle (oracle/cnn.py), through the C ABI.

Tolerances come from BF16: weights and activations are rounded to 8-bit
mantissas (unit roundoff 2^-9 = 2.0e-3) at every layer and accumulated in
FP32. A layer's output then carries a relative error of a few 2^-9 of its
scale, and six layers give a few percent of the output scale:
  forward y:    max|y - y_oracle| <= 3e-2 max|y_oracle|
  gradients:    per layer, max|dW - dW_oracle| <= 5e-2 max|dW_oracle|
  loss:         relative 2e-2
Adam runs in FP32 on FP32 master weights: the update matches the oracle's
FP64 Adam applied to the same gradients to 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import cnn as ocnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def oracle_params(px, net):
    return [(w.astype(np.float64), b.astype(np.float64)) for w, b in px.cnn_unflatten(net.params())]


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)


DIL = (1, 3, 9, 27, 81, 1)


@pytest.mark.parametrize("B,H,W,dil", [(2, 8, 64, None), (1, 12, 128, None), (1, 256, 256, None),
                                       (2, 8, 64, DIL), (1, 256, 256, DIL), (1, 32, 192, (1, 2, 5, 7, 3, 2))])
def test_forward_matches_oracle(px, B, H, W, dil):
    net = px.Cnn(seed=3, dilations=dil)
    rng = np.random.default_rng(B * 1000 + H)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    net.forward(xt, y)
    torch.cuda.synchronize()
    ref, _ = ocnn.forward(oracle_params(px, net), x.astype(np.float64)[:, None], dil)
    ref = ref[:, 0]
    got = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 3e-2 * np.max(np.abs(ref))
    net.close()


@pytest.mark.parametrize("dil", [None, DIL])
def test_gradients_match_oracle(px, dil):
    B, H, W = 2, 8, 64
    net = px.Cnn(seed=5, dilations=dil)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = rng.standard_normal((B, H, W)).astype(np.float32)
    g, loss = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    P = oracle_params(px, net)
    y, cache = ocnn.forward(P, x.astype(np.float64)[:, None], dil)
    L, dy = ocnn.mse(y, t.astype(np.float64)[:, None])
    ref = ocnn.backward(P, cache, dy, dil)
    assert abs(loss - L) <= 2e-2 * L
    gl = px.cnn_unflatten(g)
    for li, ((dW, db), (gw, gb)) in enumerate(zip(ref, gl)):
        assert np.max(np.abs(gw - dW)) <= 5e-2 * np.max(np.abs(dW)), li
        assert np.max(np.abs(gb - db)) <= 5e-2 * max(np.max(np.abs(db)), 1e-3 * np.max(np.abs(dW))), li
    net.close()


def test_adam_step_matches_oracle(px):
    B, H, W = 2, 8, 64
    net = px.Cnn(seed=11)
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    p0 = net.params().astype(np.float64)
    g, _ = net.grads(x, t)
    net.train_step(x, t, 1e-3)
    p1 = net.params().astype(np.float64)
    ref, _, _ = ocnn.adam_step(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.max(np.abs(p1 - ref)) <= 1e-5 * np.max(np.abs(p0))
    net.close()


def test_training_reduces_loss(px):
    B, H, W = 4, 32, 64
    net = px.Cnn(seed=1)
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(0.1 * rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    l0 = net.train_step(x, t, 1e-3)
    for _ in range(40):
        l1 = net.train_step(x, t, 1e-3)
    assert l1 < 0.5 * l0
    net.close()


def test_prepare_and_guess_scaling(px):
    """x = rho h^2 / s, t = phi 4 pi^2 h^2 / s with s = max|rho h^2| per image,
    and guess = s / (4 pi^2 h^2) (y - mean y); the scaling arithmetic is checked
    in FP64 numpy."""
    B, H, W = 2, 16, 64
    h = 1.0 / W
    net = px.Cnn(seed=4)
    rng = np.random.default_rng(6)
    rho = rng.standard_normal((B, H, W))
    phi = rng.standard_normal((B, H, W))
    r_t, p_t = torch.from_numpy(rho).cuda(), torch.from_numpy(phi).cuda()
    x = torch.empty(B, H, W, dtype=torch.float32, device="cuda")
    t = torch.empty_like(x)
    sc = net.prepare(r_t, p_t, x, t, h)
    s_ref = np.max(np.abs(rho * h * h), axis=(1, 2))
    assert np.array_equal(sc, s_ref)
    # one FP32 ulp: the kernel multiplies by 1/s where numpy divides by s
    assert np.allclose(x.cpu().numpy(), (rho * h * h / s_ref[:, None, None]).astype(np.float32), rtol=2.4e-7, atol=0)
    ts = 4 * np.pi**2 * h * h
    assert np.allclose(t.cpu().numpy(), (phi * ts / s_ref[:, None, None]).astype(np.float32), rtol=2.4e-7, atol=0)
    y = torch.empty_like(x)
    net.forward(x, y)
    g = torch.empty_like(r_t)
    net.guess(r_t, g, h)
    torch.cuda.synchronize()
    yy = y.cpu().numpy().astype(np.float64)
    ref = (s_ref / ts)[:, None, None] * (yy - yy.mean(axis=(1, 2), keepdims=True))
    assert np.max(np.abs(g.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    net.close()


def test_unsupported_shapes(px):
    with pytest.raises(px.PxError) as ei:
        px.Cnn(seed=0, dilations=(1, 0, 1, 1, 1, 1))
    assert ei.value.status == px.PX_EINVAL
    net = px.Cnn(seed=0)
    x = torch.zeros(1, 8, 100, device="cuda")
    with pytest.raises(px.PxError) as ei:
        net.forward(x, torch.empty_like(x))
    assert ei.value.status == px.PX_EUNSUPPORTED
    net.close()


def test_checkpoint_resume_is_bitwise(px, tmp_path):
    """Training interrupted after 3 of 6 steps and resumed from its checkpoint
    (parameters, Adam moments, step, data-order RNG) ends in exactly the state
    of an uninterrupted 6-step run."""
    from paper_2307_07931_b300 import learned
    rng = np.random.default_rng(31)
    X = torch.from_numpy(rng.standard_normal((8, 64, 64)).astype(np.float32)).cuda()
    T = torch.from_numpy(0.1 * rng.standard_normal((8, 64, 64)).astype(np.float32)).cuda()
    dil = (1, 2, 3, 2, 1, 1)
    ck = str(tmp_path / "ck.npz")
    log = lambda m: None
    a = px.Cnn(seed=1, dilations=dil)
    learned.train(px, torch, a, X, T, 6, 4, 1e-3, 5, log, ckpt=ck, ckpt_every=3, stop_at=3)
    a.close()
    b = px.Cnn(seed=99, dilations=dil)  # different init: everything comes from the checkpoint
    learned.train(px, torch, b, X, T, 6, 4, 1e-3, 5, log, ckpt=ck, ckpt_every=3)
    c = px.Cnn(seed=1, dilations=dil)
    learned.train(px, torch, c, X, T, 6, 4, 1e-3, 5, log)
    sb, stb = b.state()
    sc, stc = c.state()
    assert stb == stc == 6
    assert np.array_equal(sb, sc)
    b.close()
    c.close()

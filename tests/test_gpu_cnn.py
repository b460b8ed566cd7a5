"""GPU parity of the learned-guess network kernels (px_cnn_*) against the FP64
network oracle (oracle/cnn.py), through the C ABI.

Tolerances come from BF16 storage. BF16 keeps 8 significant bits, so one
rounding has a relative error of at most u = 2^-8 = 3.9e-3. The hidden
weights W2..W5 are BF16 on the GPU; the oracle gets the same BF16-rounded
weights (W1, W6 and the biases stay FP32 on both sides), so what is left is
the rounding of the five hidden activations (and, backwards, of the
activation gradients) plus FP32 accumulation. A CPU emulation of that
storage (FP64 arithmetic, BF16 rounding where the GPU stores BF16) against
the plain oracle gives, over 15 seeded cases of the shapes below:
  forward y:   max|y - y_oracle| / max|y_oracle| <= 6.5e-3  -> bound 1.25e-2
  gradients:   per layer, err / max|dW_oracle| <= 4e-3 on 8-row images,
               <= 1.6e-4 on 256^2 images (many pixels per sum)
                                                             -> 1e-2 and 2e-3
  loss:        relative <= 2.2e-4                            -> 2e-3
One layer at a time the bound is tight and rigorous: with the GPU's own BF16
input of a layer, z = bf16(fp32 sum) differs from the FP64 oracle's z by at
most u |z| (the rounding) plus the FP32 accumulation error of 289 terms,
289 * 2^-24 * sum|w x| <= 2e-5 S (S bounded by max|x| sum|w| per output
channel; 5e-5 S is allowed for the tensor cores' accumulation order).
The GPU's GELU is erf from Abramowitz and Stegun 7.1.26 (|error| <= 1.5e-7)
with the hardware reciprocal and exponential: within 4.2e-7 of the oracle's
erf-GELU, and within 1e-6 |z| + 0.01 u |GELU(z)| (the slack of the activation
bound below) at every FP32 z in [-12, 12] (tests/test_cnn_gelu.py).
Adam runs in FP32 on FP32 master weights: the update matches the oracle's
FP64 Adam applied to the same gradients to 1e-5 relative.

The multi-tile cases run the persistent kernels with several tiles per CTA:
the 4 x 64 output tiles are dealt to min(tiles, 2 x SMs) CTAs (296 on
B300), so B = 8 images of 256^2 (2048 tiles) give each CTA about seven
tiles, alternating its two tensor-memory accumulator sets and flipping every
barrier phase many times; the weight gradient's 2 x 64-pixel tiles at B = 2,
256^2 (1024 tiles) make each CTA accumulate about 3.5 tiles in tensor memory
before the fixed-order reduction of the 296 partials.
"""
import numpy as np
import pytest

from oracle import cnn as ocnn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)


def oracle_params(px, net, bf16_hidden=True):
    """The network's FP32 master parameters in FP64; with bf16_hidden the
    weights of the four 32 -> 32 layers rounded to BF16, as the GPU uses them."""
    out = []
    for li, (w, b) in enumerate(px.cnn_unflatten(net.params())):
        w = w.astype(np.float64)
        if bf16_hidden and 1 <= li <= 4:
            w = bf16_round(w)
        out.append((w, b.astype(np.float64)))
    return out


DIL = (1, 3, 9, 27, 81, 1)
FWD_TOL, GRAD_TOL_SMALL, GRAD_TOL_LARGE, LOSS_TOL = 1.25e-2, 1e-2, 2e-3, 2e-3


@pytest.mark.parametrize("relabel", [1, 0])
@pytest.mark.parametrize("B,H,W,dil", [(2, 8, 64, None), (1, 12, 128, None), (1, 256, 256, None),
                                       (2, 8, 64, DIL), (1, 256, 256, DIL), (1, 32, 192, (1, 2, 5, 7, 3, 2)),
                                       (1, 12, 192, (1, 5, 3, 7, 9, 1))])
def test_forward_matches_oracle(px, B, H, W, dil, relabel):
    """relabel 1: dilated layers whose dilation is invertible modulo H and W
    run over relabelled activations (at 32 x 192, d = 2 and 3 are not, d = 5
    and 7 are, so relabelled and natural-order layers alternate; at 12 x 192
    only d = 5 and 7 are); relabel 0: natural order everywhere."""
    net = px.Cnn(seed=3, dilations=dil)
    net.set_relabel(relabel)
    rng = np.random.default_rng(B * 1000 + H)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    net.forward(xt, y)
    torch.cuda.synchronize()
    ref, _ = ocnn.forward(oracle_params(px, net), x.astype(np.float64)[:, None], dil)
    ref = ref[:, 0]
    got = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= FWD_TOL * np.max(np.abs(ref))
    net.close()


@pytest.mark.parametrize("relabel", [1, 0])
@pytest.mark.parametrize("dil", [None, DIL, (1, 2, 5, 7, 3, 2)])
def test_gradients_match_oracle(px, dil, relabel):
    B, H, W = 2, 8, 64
    net = px.Cnn(seed=5, dilations=dil)
    net.set_relabel(relabel)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = rng.standard_normal((B, H, W)).astype(np.float32)
    g, loss = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    P = oracle_params(px, net)
    y, cache = ocnn.forward(P, x.astype(np.float64)[:, None], dil)
    L, dy = ocnn.mse(y, t.astype(np.float64)[:, None])
    ref = ocnn.backward(P, cache, dy, dil)
    assert abs(loss - L) <= LOSS_TOL * L
    check_grads(px, g, ref, GRAD_TOL_SMALL)
    net.close()


def check_grads(px, g, ref, tol):
    gl = px.cnn_unflatten(g)
    for li, ((dW, db), (gw, gb)) in enumerate(zip(ref, gl)):
        assert np.max(np.abs(gw - dW)) <= tol * np.max(np.abs(dW)), li
        assert np.max(np.abs(gb - db)) <= tol * max(np.max(np.abs(db)), 1e-3 * np.max(np.abs(dW))), li


def _layer_bound(h, w, b, d):
    """Per-element FP32 accumulation scale S of one conv: max|h| over the
    image times sum |w| over (c, tap) of the output channel, plus |b|."""
    amax = np.max(np.abs(h), axis=(1, 2, 3))                     # per image
    wsum = np.sum(np.abs(w), axis=(1, 2, 3))                    # per output channel
    return amax[:, None, None, None] * wsum[None, :, None, None] + np.abs(b)[None, :, None, None]


@pytest.mark.parametrize("dil", [None, DIL])
def test_forward_multitile_matches_oracle(px, dil):
    """B = 8 images of 256^2: about seven tiles per CTA of every tensor-core
    layer. The output is compared element by element with the FP64 oracle
    (bound FWD_TOL), and every hidden layer of images 0, 3, 6 and 7 (the
    first and the later tiles of the CTAs, both accumulator sets) with the
    oracle's conv of the GPU's own BF16 input (rigorous per-element bound)."""
    B, H, W = 8, 256, 256
    d = dil or (1,) * 6
    net = px.Cnn(seed=13, dilations=dil)
    rng = np.random.default_rng(17)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = rng.standard_normal((B, H, W)).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    net.forward(xt, y)
    torch.cuda.synchronize()
    P = oracle_params(px, net)
    ref, _ = ocnn.forward(P, x.astype(np.float64)[:, None], dil)
    got = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref[:, 0])) <= FWD_TOL * np.max(np.abs(ref))
    # training forward keeps z; its activations equal the inference ones
    net.grads(xt, torch.from_numpy(t).cuda())
    imgs = [0, 3, 6, 7]

    def hidden(layer, which):
        return net.hidden(layer, which, (B, H, W))[imgs].transpose(0, 3, 1, 2).astype(np.float64)
    hin = x.astype(np.float64)[imgs][:, None]
    for li in range(5):                                          # layers 1..5 (index li)
        w, b = P[li]
        zr = ocnn.conv(hin, w, b, d[li])
        S = _layer_bound(hin, w, b, d[li])
        zg = hidden(li + 1, "z")
        assert np.all(np.abs(zg - zr) <= 1.01 * U_BF16 * np.abs(zr) + 5e-5 * S), li
        del zg
        ar = ocnn.gelu(zr)
        ag = hidden(li + 1, "a")
        assert np.all(np.abs(ag - ar) <= 1.01 * U_BF16 * np.abs(ar) + 1.13 * 5e-5 * S
                      + 1e-6 * np.abs(zr)), li
        hin = ag
        del zr, ar, S
    w6, b6 = P[5]
    yr = ocnn.conv(hin, w6, b6, d[5])[:, 0]
    S6 = _layer_bound(hin, w6, b6, d[5])[:, 0]
    assert np.all(np.abs(got[imgs] - yr) <= 5e-5 * S6)
    # inference output unchanged by the training forward's bookkeeping
    y2 = torch.empty_like(xt)
    net.forward(xt, y2)
    torch.cuda.synchronize()
    assert torch.equal(y, y2)
    net.close()


@pytest.mark.parametrize("dil,relabel", [(None, 1), (DIL, 1), (DIL, 0)])
def test_gradients_multitile_match_oracle(px, dil, relabel):
    """B = 2 images of 256^2: the weight-gradient kernel accumulates about 3.5
    tiles per CTA in tensor memory and reduces 296 partials; the input-gradient
    convolution runs about 1.7 tiles per CTA. Every layer's dW and db against
    the oracle's analytic backward, the loss against the oracle's MSE."""
    B, H, W = 2, 256, 256
    net = px.Cnn(seed=21, dilations=dil)
    net.set_relabel(relabel)
    rng = np.random.default_rng(23)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = rng.standard_normal((B, H, W)).astype(np.float32)
    g, loss = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    P = oracle_params(px, net)
    y, cache = ocnn.forward(P, x.astype(np.float64)[:, None], dil)
    L, dy = ocnn.mse(y, t.astype(np.float64)[:, None])
    ref = ocnn.backward(P, cache, dy, dil)
    assert abs(loss - L) <= LOSS_TOL * L
    check_grads(px, g, ref, GRAD_TOL_LARGE)
    # deterministic: the same call gives bitwise the same gradients
    g2, loss2 = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    assert np.array_equal(g, g2) and loss == loss2
    net.close()


@pytest.mark.parametrize("dil,relabel", [(None, 1), (DIL, 1), (DIL, 0), ((1, 2, 5, 64, 7, 1), 1),
                                         ((1, 2, 5, 64, 7, 1), 0)])
def test_tma_staging_bitwise_equals_copies(px, dil, relabel):
    """Tiles and patches staged by the tensor memory accelerator (in-image
    ones) and by per-pixel copies (every one) are the same bytes: the forward
    output, the hidden tensors and all gradients agree bitwise, at several
    tiles per CTA (B = 4, 256^2), for the unit-offset patches (relabelled or
    d = 1) and the nine offset tap tiles (natural order, or d = 2 and 64,
    which are not invertible modulo 256), with boxes that cross the edge."""
    B, H, W = 4, 256, 256
    rng = np.random.default_rng(41)
    x = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    out = {}
    for mode in (0, 1):
        net = px.Cnn(seed=43, dilations=dil)
        net.set_staging(mode)
        net.set_relabel(relabel)
        y = torch.empty_like(x)
        net.forward(x, y)
        g, loss = net.grads(x, t)
        hid = [net.hidden(l, w, (B, H, W)) for l in (2, 5) for w in ("a", "z")]
        torch.cuda.synchronize()
        out[mode] = (y.cpu().numpy(), g, loss, hid)
        net.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
    for a, b in zip(out[0][3], out[1][3]):
        assert np.array_equal(a, b)
    with pytest.raises(px.PxError):
        px.Cnn(seed=1).set_staging(2)
    with pytest.raises(px.PxError):
        px.Cnn(seed=1).set_relabel(2)


def test_bounded_wait_times_out_and_recovers(px):
    """With one poll per handshake wait the tensor-core kernels give up (no
    phase completes that fast everywhere), drain their issued MMAs, free
    their tensor memory and raise the fault word: the call returns
    PX_ETIMEOUT. With the default limit restored, the next call on the same
    context gives bitwise the gradients of a call made before the timeout."""
    B, H, W = 4, 64, 256
    net = px.Cnn(seed=29, dilations=DIL)
    rng = np.random.default_rng(31)
    x = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, H, W)).astype(np.float32)).cuda()
    g0, l0 = net.grads(x, t)
    net.set_wait_limit(1)
    with pytest.raises(px.PxError) as ei:
        net.grads(x, t)
    assert ei.value.status == px.PX_ETIMEOUT
    net.set_wait_limit(0)
    g1, l1 = net.grads(x, t)
    assert np.array_equal(g0, g1) and l0 == l1
    y = torch.empty_like(x)
    net.forward(x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
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

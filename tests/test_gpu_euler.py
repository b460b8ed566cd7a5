"""GPU parity of the fused 2D Euler finite-volume step (px_euler_step)
against the FP64 oracle (oracle/euler.py), through the C ABI, element by
element.

Tolerances, from the arithmetic. Both sides evaluate the same formulas; the
GPU multiplies by reciprocals where the oracle divides and contracts
products into FMAs, so each flux differs by a few ulps of its magnitude |F|.
A step changes U by dt times flux differences over the cell size, and
dt (|u| + c) / dx <= cfl, so the per-step difference is a few ulps of
cfl |U| per flux evaluation; minmod and max are Lipschitz (a rounding-level
change of their arguments changes their value by as much), so no branch of
the limiter amplifies it. Allowed per step, relative to the component's
max |U|: FP64 1e-12 (about 4500 ulps), FP32 storage and arithmetic 2e-5
(about 170 FP32 ulps; the FP32 input is the oracle's input rounded to
FP32, and the oracle then works in FP64). Over n steps n times that (the
scheme is stable at cfl 0.4, so differences grow at most additively at
these sizes). The time steps: FP64 1e-13, FP32 1e-6 relative.
"""
import numpy as np
import pytest

import synth
from oracle import euler as E

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-5}
DT_TOL = {torch.float64: 1e-13, torch.float32: 1e-6}


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def random_state(rng, ny, nx, amp=0.3):
    rho = 1.0 + amp * rng.uniform(-1, 1, (ny, nx))
    p = 1.0 + amp * rng.uniform(-1, 1, (ny, nx))
    u = amp * rng.uniform(-1, 1, (ny, nx))
    v = amp * rng.uniform(-1, 1, (ny, nx))
    return E.conserved(np.stack([rho, u, v, p]))


def blocky_state(rng, ny, nx):
    """Piecewise-constant blocks of random states: discontinuities everywhere,
    so every limiter branch is taken."""
    by, bx = max(1, ny // 5), max(1, nx // 7)
    W = np.empty((4, ny, nx))
    for j0 in range(0, ny, by):
        for i0 in range(0, nx, bx):
            W[:, j0:j0 + by, i0:i0 + bx] = np.array(
                [rng.uniform(0.2, 2.0), rng.uniform(-1, 1), rng.uniform(-1, 1),
                 rng.uniform(0.2, 3.0)])[:, None, None]
    return E.conserved(W)


def rel_err(got, ref):
    return max(float(np.max(np.abs(got[m] - ref[m])) / np.max(np.abs(ref[m]))) for m in range(4))


SHAPES = [(64, 48), (130, 70), (33, 17), (8, 8), (1, 5), (200, 3), (36, 20), (35, 19), (97, 161),
          (256, 96)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_steps_match_oracle(px, nx, ny, dtype):
    rng = np.random.default_rng(nx * 1000 + ny)
    dx, dy = 1.0 / nx, 0.8 / ny
    for make in (random_state, blocky_state):
        U0 = make(rng, ny, nx)
        if dtype == torch.float32:
            U0 = U0.astype(np.float32).astype(np.float64)
        nsteps = 3 if dtype == torch.float64 else 1
        ref, dts = E.run(U0, dx, dy, nsteps, cfl=0.4)
        u = torch.from_numpy(U0).to(dtype).cuda()
        out = torch.empty_like(u)
        dt = torch.zeros(nsteps, dtype=torch.float64, device="cuda")
        px.euler_step(u, out, dx, dy, nsteps, cfl=0.4, dt=dt)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert rel_err(got, ref) <= nsteps * TOL[dtype], (make.__name__, rel_err(got, ref))
        g = dt.cpu().numpy()
        assert np.all(np.abs(g - np.array(dts)) <= DT_TOL[dtype] * np.array(dts)), (g, dts)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pressureless_static_state_is_steady(px, dtype):
    """p = 0 and u = v = 0 with varying density: the sound speed is 0 and every
    flux vanishes (no pressure, no transport, a zero Rusanov coefficient), so
    steps with a fixed dt leave the state unchanged bitwise, with no NaN (the
    sound speed's product form g p rsqrt(g p rho) must not become 0 * inf)."""
    rng = np.random.default_rng(3)
    ny, nx = 40, 70
    z = np.zeros((ny, nx))
    U0 = E.conserved(np.stack([rng.uniform(0.5, 2.0, (ny, nx)), z, z, z]))
    u = torch.from_numpy(U0).to(dtype).cuda()
    out = torch.empty_like(u)
    px.euler_step(u, out, 1.0 / nx, 1.0 / ny, 2, dt_fixed=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(out, u)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_fixed_dt_and_in_place(px, dtype):
    rng = np.random.default_rng(5)
    nx, ny = 96, 64
    dx = dy = 1.0 / 96
    U0 = blocky_state(rng, ny, nx)
    if dtype == torch.float32:
        U0 = U0.astype(np.float32).astype(np.float64)
    dts = [2e-3, 1e-3, 3e-3]
    ref, _ = E.run(U0, dx, dy, 3, dts=dts)
    u = torch.from_numpy(U0).to(dtype).cuda()
    out = torch.empty_like(u)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    # three calls of one step each with fixed dt, then in place
    a = u.clone()
    for k in range(3):
        px.euler_step(a if k else u, out, dx, dy, 1, dt_fixed=dts[k], dt=dt)
        torch.cuda.synchronize()
        assert float(dt[0]) == dts[k]
        a = out.clone()
    got = out.double().cpu().numpy()
    assert rel_err(got, ref) <= 3 * TOL[dtype]
    b = u.clone()
    for k in range(3):
        px.euler_step(b, b, dx, dy, 1, dt_fixed=dts[k])
    torch.cuda.synchronize()
    assert torch.equal(b, out)


def test_adaptive_multistep_in_place_equals_out_of_place(px):
    rng = np.random.default_rng(6)
    U0 = torch.from_numpy(random_state(rng, 70, 130)).cuda()
    a = torch.empty_like(U0)
    px.euler_step(U0, a, 1 / 130, 1 / 70, 5)
    b = U0.clone()
    px.euler_step(b, b, 1 / 130, 1 / 70, 5)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_uniform_state_preserved_and_conservation(px, dtype):
    W = np.stack([np.full((40, 50), 1.3), np.full((40, 50), 0.7), np.full((40, 50), -0.2),
                  np.full((40, 50), 2.1)])
    u = torch.from_numpy(E.conserved(W)).to(dtype).cuda()
    out = torch.empty_like(u)
    px.euler_step(u, out, 0.1, 0.2, 4)
    torch.cuda.synchronize()
    assert torch.equal(out, u)
    rng = np.random.default_rng(8)
    U0 = blocky_state(rng, 64, 96)
    u = torch.from_numpy(U0).to(dtype).cuda()
    out = torch.empty_like(u)
    px.euler_step(u, out, 1 / 96, 1 / 64, 10)
    torch.cuda.synchronize()
    s0 = u.double().sum(dim=(1, 2)).cpu().numpy()
    s1 = out.double().sum(dim=(1, 2)).cpu().numpy()
    scale = u.double().abs().sum(dim=(1, 2)).cpu().numpy()
    eps = 1e-13 if dtype == torch.float64 else 2e-6
    assert np.all(np.abs(s1 - s0) <= eps * scale), (s1 - s0) / scale


def test_pitched_layout_bitwise(px):
    """Row pitch > nx and plane pitch > ny * ld give bitwise the results of the
    packed layout (the vectorless kernel indexes through both pitches)."""
    rng = np.random.default_rng(9)
    U0 = torch.from_numpy(blocky_state(rng, 37, 75)).cuda()
    big = torch.full((4, 40, 80), float("nan"), dtype=torch.float64, device="cuda")
    p_in = big[:, :37, :75]
    p_in.copy_(U0)
    p_out = torch.full((4, 40, 80), float("nan"), dtype=torch.float64, device="cuda")[:, :37, :75]
    px.euler_step(p_in, p_out, 1 / 75, 1 / 37, 3)
    packed = torch.empty_like(U0)
    px.euler_step(U0, packed, 1 / 75, 1 / 37, 3)
    torch.cuda.synchronize()
    assert torch.equal(p_out, packed)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_box_and_per_cell_staging_bitwise(px, dtype):
    """Tiles whose halo lies inside the field arrive as one tensor-memory-
    accelerator box when the row and plane pitches are multiples of 16 bytes;
    a row pitch of nx + 1 elements forces the per-cell copies everywhere. The
    staged values are the same, so the states and time steps are bitwise equal."""
    rng = np.random.default_rng(10)
    nx, ny = 256, 200
    U0 = torch.from_numpy(blocky_state(rng, ny, nx)).to(dtype).cuda()
    a = torch.empty_like(U0)
    da = torch.zeros(3, dtype=torch.float64, device="cuda")
    px.euler_step(U0, a, 1 / nx, 1 / ny, 3, dt=da)
    big = torch.zeros(4, ny, nx + 1, dtype=dtype, device="cuda")
    p_in = big[:, :, :nx]
    p_in.copy_(U0)
    p_out = torch.zeros(4, ny, nx + 1, dtype=dtype, device="cuda")[:, :, :nx]
    db = torch.zeros(3, dtype=torch.float64, device="cuda")
    px.euler_step(p_in, p_out, 1 / nx, 1 / ny, 3, dt=db)
    torch.cuda.synchronize()
    assert torch.equal(a, p_out) and torch.equal(da, db)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_conserved_conversion(px, dtype):
    W = synth.euler_kh_primitives(128, 96, seed=3)
    w = torch.from_numpy(W).to(dtype).cuda()
    u = torch.empty_like(w)
    px.euler_conserved(w, u)
    torch.cuda.synchronize()
    ref = E.conserved(W.astype(np.float32).astype(np.float64) if dtype == torch.float32 else W)
    got = u.double().cpu().numpy()
    eps = 2.3e-16 if dtype == torch.float64 else 1.2e-7
    assert np.all(np.abs(got - ref) <= 4 * eps * np.abs(ref))


def test_argument_errors(px):
    u = torch.zeros(4, 8, 8, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    for kw in ({"gamma": 1.0}, {"cfl": 0.0}, {"nsteps": -1}, {"dt_fixed": -1.0}):
        args = dict(nsteps=1, gamma=1.4, cfl=0.4, dt_fixed=0.0)
        args.update(kw)
        with pytest.raises(px.PxError) as ei:
            px.euler_step(u, out, 0.1, 0.1, **args)
        assert ei.value.status == px.PX_EINVAL
    with pytest.raises(px.PxError) as ei:
        px.euler_step(u, out, 0.0, 0.1)
    assert ei.value.status == px.PX_EINVAL
    # nsteps = 0 copies; an empty grid is a no-op
    u.fill_(1.0)
    px.euler_step(u, out, 0.1, 0.1, 0)
    torch.cuda.synchronize()
    assert torch.equal(out, u)
    e = torch.zeros(4, 0, 8, dtype=torch.float64, device="cuda")
    px.euler_step(e, e.clone(), 0.1, 0.1, 3)


def _window(a, j0, i0, size):
    ny, nx = a.shape[-2:]
    rows = (np.arange(j0, j0 + size) % ny)[:, None]
    cols = (np.arange(i0, i0 + size) % nx)[None, :]
    return a[..., rows, cols]


def test_full_size_sampled(px):
    """The benchmark's workload: 8192^2 double shear layer in FP32, two
    adaptive steps in one call. 24 windows of 48^2 cells (periodic) are
    recomputed by the oracle from the FP32 input with the GPU's time steps;
    their centres (margin 8 = two steps x two stages x two cells of halo)
    must match, and the first dt must match the oracle's CFL step of the
    whole field."""
    n = 8192
    W = synth.euler_kh_primitives(n, n)
    w = torch.from_numpy(W).float().cuda()
    del W
    u = torch.empty_like(w)
    px.euler_conserved(w, u)
    del w
    out = torch.empty_like(u)
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    px.euler_step(u, out, 1.0 / n, 1.0 / n, 2, dt=dt)
    torch.cuda.synchronize()
    U0 = u.cpu().numpy().astype(np.float64)
    got = out.cpu().numpy()
    del u, out
    dts = dt.cpu().numpy()
    smax = E.max_wave(U0, 1.0 / n, 1.0 / n)
    assert abs(dts[0] - 0.4 / smax) <= DT_TOL[torch.float32] * dts[0]
    rng = np.random.default_rng(12)
    size, m = 48, 8
    starts = [(0, 0), (n - 20, n - 20), (n // 4 - 24, 100), (3 * n // 4 - 24, n - 30)]
    starts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(20)]
    scale = [float(np.max(np.abs(U0[c]))) for c in range(4)]
    for (j0, i0) in starts:
        ref, _ = E.run(_window(U0, j0, i0, size), 1.0 / n, 1.0 / n, 2, dts=list(dts))
        g = _window(got, j0, i0, size)
        c = slice(m, size - m)
        for comp in range(4):
            err = float(np.max(np.abs(g[comp, c, c] - ref[comp, c, c])))
            assert err <= 2 * TOL[torch.float32] * scale[comp], (j0, i0, comp, err)

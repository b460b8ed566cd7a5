"""GPU parity of the multigrid V-cycle (px_mg_solve) against the FP64 oracle
(oracle/mg.py), through the C ABI.

Tolerances (max-norm of the difference over ||phi||, the larger of the
starting and the final state; the arithmetic behind them):
  * FP64: every step of a cycle rounds a few times at 1.1e-16 on either side
    (FMA form on the GPU, plain order in the oracle). The smoothers are
    non-expansive for omega <= 1 and the coarse correction is a projection,
    so differences grow at most linearly: 1e-11 per cycle, times the
    coarsest level's sweeps in thousands when that is larger than one.
  * FP32 (inputs rounded to FP32 on both sides): the residual is formed in
    FP32 from terms of size 8 ||phi|| / h^2, so its rounding noise is about
    eps_32 * 8 ||phi|| / h^2 per cell; the coarse correction applies L^-1,
    whose gain on the lowest mode is n^2 h^2 / (4 pi^2) (n the larger extent),
    and N = nx ny independent roundings reach one mode with weight
    1 / sqrt(N). Per cycle that is eps_32 * 8 n^2 / (4 pi^2 sqrt(N)) of
    ||phi||, about 0.2 eps_32 n for square grids; the test allows 4 eps_32 n
    per cycle (20 times that), accumulated linearly.
  * Residual reports: the same factors times the scale of the summed terms,
    8 ||phi|| / h^2 + ||rho||.
"""

import numpy as np
import pytest

import oracle
import synth
from oracle import mg as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def fields(nx, ny, seed, dtype):
    rng = np.random.default_rng(seed)
    rho = synth.random_field(rng, nx, ny)
    phi = synth.random_field(rng, nx, ny, zero_mean=False)
    return host(dev(phi, dtype)), host(dev(rho, dtype))


def tolerance(dtype, nx, ny, ncycles, coarse_sweeps):
    if dtype == torch.float64:
        return max(1, ncycles) * 1e-11 * max(1.0, coarse_sweeps / 1000.0)
    return max(1, ncycles) * 4 * EPS32 * max(nx, ny)


def run(px, phi, rho, h, ncycles, dtype, layout="plain", **kw):
    ny, nx = phi.shape
    if layout == "plain":
        a, r = dev(phi, dtype), dev(rho, dtype)
    else:  # pitch nx + 1: the finest level takes the two-pass kernels
        def place(x):
            buf = torch.full((ny, nx + 1), float("nan"), dtype=dtype, device="cuda")
            v = buf[:, :nx]
            v.copy_(torch.from_numpy(np.ascontiguousarray(x)).to(dtype))
            return v
        a, r = place(phi), place(rho)
    res = torch.full((ncycles + 1,), -1.0, dtype=torch.float64, device="cuda")
    px.mg_solve(a, r, h, ncycles, resid=res, **kw)
    torch.cuda.synchronize()
    return host(a), res.cpu().numpy()


def check(got, R, phi0, rho, h, ref, Rref, tol):
    # ||phi|| of the tolerances: the largest state the cycles round (a random
    # phi0 can be far larger than the smooth state a cycle leaves)
    scale = max(np.max(np.abs(phi0)), np.max(np.abs(ref)))
    err = np.max(np.abs(got - ref)) / scale
    assert err <= tol, err
    sc = 8.0 * scale / h**2 + np.max(np.abs(rho))
    assert np.max(np.abs(R - Rref)) <= tol * sc, (R, Rref)


CASES = [
    # (nx, ny, ncycles, nu1, nu2, omega, max_levels)
    (64, 64, 3, 2, 2, 1.0, 0),        # down to 2 x 2
    (96, 96, 2, 2, 2, 1.0, 0),        # coarsest 6 x 6 (72 sweeps)
    (256, 128, 3, 1, 1, 1.0, 0),      # rectangular, down to 4 x 2
    (128, 256, 2, 0, 2, 1.0, 0),      # no pre-smoothing: report from the restriction
    (132, 68, 2, 2, 1, 0.9, 0),       # coarsest 66 x 34
    (512, 512, 2, 3, 3, 1.0, 4),      # capped at 4 levels (coarsest 64 x 64)
    (1024, 1024, 2, 2, 2, 1.0, 0),    # several tiles per level
    (8, 4, 3, 1, 1, 1.0, 0),
    (2, 2, 2, 1, 1, 1.0, 0),          # a single 2 x 2 level
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ny,ncycles,nu1,nu2,omega,max_levels", CASES)
def test_cycles_match_oracle(px, nx, ny, ncycles, nu1, nu2, omega, max_levels, dtype):
    h = 1.0 / nx
    phi, rho = fields(nx, ny, nx + 3 * ny, dtype)
    shapes = omg.level_shapes(nx, ny, max_levels)
    cs = omg.auto_coarse_sweeps(*shapes[-1])
    got, R = run(px, phi, rho, h, ncycles, dtype, nu1=nu1, nu2=nu2, omega=omega,
                 max_levels=max_levels)
    ref, Rref = omg.mg_solve(phi, rho, h, ncycles, nu1, nu2, omega, 0, max_levels)
    check(got, R, phi, rho, h, ref, Rref, tolerance(dtype, nx, ny, ncycles, cs))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pitched_finest_level(px, dtype):
    nx, ny = 128, 64
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 4, dtype)
    ref, Rref = omg.mg_solve(phi, rho, h, 2)
    got, R = run(px, phi, rho, h, 2, dtype, layout="pitched")
    check(got, R, phi, rho, h, ref, Rref, tolerance(dtype, nx, ny, 2, 1))


def test_explicit_coarse_sweeps_and_zero_cycles(px):
    nx, ny = 64, 32
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 8, torch.float64)
    got, R = run(px, phi, rho, h, 2, torch.float64, coarse_sweeps=5, max_levels=3)
    ref, Rref = omg.mg_solve(phi, rho, h, 2, coarse_sweeps=5, max_levels=3)
    check(got, R, phi, rho, h, ref, Rref, 2e-11)
    got0, R0 = run(px, phi, rho, h, 0, torch.float64)
    assert np.array_equal(got0, phi)
    sc = 8 * np.max(np.abs(phi)) / h**2
    assert R0.shape == (1,) and abs(R0[0] - oracle.residual_norm(phi, rho, h)[0]) <= 1e-12 * sc


def test_rejects_bad_arguments(px):
    a = torch.zeros((64, 62), dtype=torch.float32, device="cuda")
    px.mg_solve(a, torch.zeros_like(a), 1 / 62, 1)  # even extents are fine
    b = torch.zeros((64, 63), dtype=torch.float32, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.mg_solve(b, torch.zeros_like(b), 1 / 63, 1)
    assert ei.value.status == px.PX_EINVAL
    with pytest.raises(px.PxError) as ei:
        px.mg_solve(a, a, 1 / 62, 1)  # rho overlaps phi
    assert ei.value.status == px.PX_EINVAL
    with pytest.raises(px.PxError) as ei:
        px.mg_solve(a, torch.zeros_like(a), 1 / 62, 1, nu1=-1)
    assert ei.value.status == px.PX_EINVAL
    e = torch.zeros(0, 6, dtype=torch.float32, device="cuda")
    px.mg_solve(e, e.clone(), 1.0, 3)


def exact_modes_solution(n, modes):
    """The discrete solution of L phi = sum of modes: each mode is an
    eigenvector of L with eigenvalue -(4/h^2)(sin^2(pi k/n) + sin^2(pi l/n))."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    phi = np.zeros((n, n))
    for (k, l, a, b) in modes:
        lam = -(4 / h**2) * (np.sin(np.pi * k / n) ** 2 + np.sin(np.pi * l / n) ** 2)
        cx, sx = np.cos(2 * np.pi * k * x), np.sin(2 * np.pi * k * x)
        cy, sy = np.cos(2 * np.pi * l * x), np.sin(2 * np.pi * l * x)
        # a cos(2 pi (k x + l y)) + b sin(2 pi (k x + l y)), separably
        phi += (a * (np.outer(cy, cx) - np.outer(sy, sx))
                + b * (np.outer(cy, sx) + np.outer(sy, cx))) / lam
    return phi


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_full_size_convergence(px, dtype):
    """16384 x 16384 (14 levels, down to 2 x 2) with rho a sum of 12 modes
    (k up to 512), whose discrete solution is known in closed form. From
    phi = 0, V(2,2) cycles reduce the residual by a factor of at most 0.15
    per cycle over the first three and keep reducing it until the storage
    precision's floor, and the state approaches the closed-form solution;
    the state-0 report is max|rho| exactly."""
    n = 16384
    h = 1.0 / n
    rng = np.random.default_rng(12)
    modes = [(int(rng.integers(1, 513)), int(rng.integers(0, 513)), float(rng.normal()),
              float(rng.normal())) for _ in range(12)]
    sol = exact_modes_solution(n, modes)
    rho = oracle.apply_stencil(sol, h)   # the exact right-hand side of sol (FP64)
    rho_t = dev(rho, dtype)
    rho_s = host(rho_t)
    del rho
    phi = torch.zeros_like(rho_t)
    nc = 6 if dtype == torch.float32 else 9
    res = torch.zeros(nc + 1, dtype=torch.float64, device="cuda")
    px.mg_solve(phi, rho_t, h, nc, resid=res)
    torch.cuda.synchronize()
    R = res.cpu().numpy()
    assert R[0] == np.max(np.abs(rho_s))
    floor = (8 * np.max(np.abs(sol)) / h**2) * (1e-6 if dtype == torch.float32 else 1e-13)
    # the first cycle's factor depends on the starting error's mix of modes;
    # over three cycles the textbook rate holds, and every cycle reduces the
    # residual until the precision's floor
    assert (R[3] / R[0]) ** (1.0 / 3.0) <= 0.15, R
    for k in range(nc):
        assert R[k + 1] <= max(0.5 * R[k], floor), (k, R)
    got = host(phi)
    got -= got.mean()
    err = np.max(np.abs(got - (sol - sol.mean()))) / np.max(np.abs(sol))
    # FP32: the solution of the FP32-rounded problem is within about
    # eps_32 n^2 / (4 pi^2) of the exact one on the lowest modes present
    assert err <= (1e-3 if dtype == torch.float32 else 1e-8), err


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_smoother_paths_bitwise(sweeps):
    """On FP32 the finest level's smoother runs on the register wavefront
    (aligned rows) or on the two-pass kernels (pitch nx + 1); both evaluate
    the same per-cell expressions, so whole cycles agree bitwise, at every
    depth of the wavefront (selected per context with
    PX_OPT_RB_SWEEPS_PER_LAUNCH)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_RB_SWEEPS_PER_LAUNCH, sweeps)
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        for (nx, ny) in [(1024, 512), (256, 256), (132, 68)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            rho -= rho.mean()
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)

            def pitched(a):
                b = torch.zeros(ny, nx + 1, device="cuda", dtype=torch.float32)[:, :nx]
                b.copy_(a)
                return b
            a, ra = phi.clone(), torch.zeros(4, dtype=torch.float64, device="cuda")
            px.mg_solve(a, rho, h, 3, resid=ra, ctx=ctx)
            b, rb = pitched(phi), torch.zeros_like(ra)
            px.mg_solve(b, pitched(rho), h, 3, resid=rb, ctx=ctx)
            torch.cuda.synchronize()
            assert torch.equal(a, b) and torch.equal(ra, rb), (nx, ny)
    finally:
        ctx.close()


def test_fp64_smoother_fused_bitwise():
    """On FP64 every level's smoother runs one fused launch per red-black sweep
    (16-byte aligned levels) or a red and a black pass
    (PX_OPT_RB_FP64_PASSES = 2); both evaluate the same per-cell expressions,
    so whole cycles agree bitwise."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctxs = [px.Context(torch.cuda.current_device()) for _ in range(2)]
    try:
        ctxs[1].set_option(px.PX_OPT_RB_FP64_PASSES, 2)
        g = torch.Generator(device="cuda")
        g.manual_seed(9)
        for (nx, ny) in [(1024, 512), (256, 256), (132, 68)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
            rho -= rho.mean()
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
            got = []
            for ctx in ctxs:
                a, ra = phi.clone(), torch.zeros(4, dtype=torch.float64, device="cuda")
                px.mg_solve(a, rho, h, 3, resid=ra, ctx=ctx)
                torch.cuda.synchronize()
                got.append((a, ra))
            assert torch.equal(got[0][0], got[1][0]) and torch.equal(got[0][1], got[1][1]), (nx, ny)
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("nu2", [1, 2, 3, 4])
def test_interpolation_in_smoother_bitwise(nu2):
    """On FP32 levels that the register wavefront smooths, the interpolation and
    correction run inside the first post-smoothing launch (each input row gets
    its correction as it is loaded), with the operations of the separate pass
    (PX_OPT_MG_PROLONG = 1): whole cycles and their reports agree bitwise, for
    one to four post-smoothing sweeps (one or two launches), on grids whose
    levels cover several strips, ragged strips and row ranges of one pair."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctxs = [px.Context(torch.cuda.current_device()) for _ in range(2)]
    try:
        ctxs[1].set_option(px.PX_OPT_MG_PROLONG, 1)
        assert ctxs[1].get_option(px.PX_OPT_MG_PROLONG) == 1
        g = torch.Generator(device="cuda")
        g.manual_seed(11)
        for (nx, ny) in [(4096, 2048), (1024, 512), (520, 264), (132, 68), (16, 8)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            rho -= rho.mean()
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            got = []
            for ctx in ctxs:
                a, ra = phi.clone(), torch.zeros(4, dtype=torch.float64, device="cuda")
                px.mg_solve(a, rho, h, 3, nu1=2, nu2=nu2, resid=ra, ctx=ctx)
                torch.cuda.synchronize()
                got.append((a, ra))
            assert torch.equal(got[0][0], got[1][0]) and torch.equal(got[0][1], got[1][1]), (nx, ny)
    finally:
        for c in ctxs:
            c.close()

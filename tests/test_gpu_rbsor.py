"""GPU parity of the red-black SOR sweeps (px_rbsor_n) against the FP64
oracle (oracle.rbsor_n), through the C ABI.

Tolerances (relative max-norm; the arithmetic behind them):
  * One sweep from the same state: the kernel rounds the tap sum and the
    update a handful of times (FMA form), the oracle in FP64. A red update
    differs from the oracle's by a few ulps of |phi|; a black update reads four
    red values, each off by that much, and scales them by omega / 4 each, plus
    |1 - omega| times its own value, so one sweep is off by at most
    (|1 - omega| + omega) + 1 = 2 omega (omega >= 1) or 2 (omega <= 1) times
    the per-update figure. Per update: 1e-12 (FP64), 2e-6 (FP32, about 30 ulps).
  * n sweeps at omega <= 1: the sweep operator is a convex combination of
    old values (plus the rho term) for each colour, so it is non-expansive in
    the max-norm and per-sweep differences add up at most linearly: n times.
  * Over-relaxation (omega > 1) is checked one sweep at a time from the same
    state (the max-norm of the sweep operator exceeds one there, so no linear
    bound holds over many sweeps).
  * Residual reports (the input state of each reported sweep): against the
    scale of the summed terms, 8 ||phi|| / h^2 + ||rho||, with the factors of phi.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def per_update(dtype):
    return 2e-6 if dtype == torch.float32 else 1e-12


def fields(nx, ny, seed, dtype):
    """Seeded phi/rho, rounded to the storage type so both sides start equal."""
    rng = np.random.default_rng(seed)
    rho = synth.random_field(rng, nx, ny)
    phi = synth.random_field(rng, nx, ny, zero_mean=False)
    return host(dev(phi, dtype)), host(dev(rho, dtype))


def place(x, dtype, layout):
    """Device copy of x: 'plain' (aligned, vector path), 'pitched' (odd pitch)
    or 'offset' (base one element past a 16-byte boundary)."""
    ny, nx = x.shape
    if layout == "plain":
        return dev(x, dtype)
    extra = 1 if layout == "pitched" else 0
    shift = 1 if layout == "offset" else 0
    buf = torch.full((ny, nx + extra + shift), float("nan"), dtype=dtype, device="cuda")
    v = buf[:, shift:shift + nx]
    v.copy_(torch.from_numpy(np.ascontiguousarray(x)).to(dtype))
    return v


def run(px, phi, rho, h, omega, nsweeps, dtype, every=1, layout="plain", inplace=False):
    a, r = place(phi, dtype, layout), place(rho, dtype, layout)
    out = a if inplace else place(np.zeros_like(phi), dtype, layout)
    nrep = (nsweeps + every - 1) // every if every > 0 else 0
    resid = torch.full((max(nrep, 1),), -1.0, dtype=torch.float64, device="cuda")
    px.rbsor_n(a, out, r, h, omega, nsweeps, resid if nrep else None, every)
    torch.cuda.synchronize()
    return host(out), resid.cpu().numpy()[:nrep], host(a)


def check(got, ref, tol):
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= tol, err


def check_reports(R_got, R_ref, phi_scale, rho, h, tol):
    assert R_got.shape == R_ref.shape
    sc = 8.0 * phi_scale / h**2 + np.max(np.abs(rho))
    assert np.max(np.abs(R_got - R_ref)) <= tol * sc, (R_got, R_ref)


SIZES = [(64, 64), (130, 66), (256, 198), (1030, 514), (2, 2), (2, 130), (4098, 6)]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("omega", [2.0 / 3.0, 1.0])
def test_sweeps_match_oracle(px, nx, ny, dtype, omega):
    h = 1.0 / nx
    phi, rho = fields(nx, ny, nx * 7 + ny, dtype)
    n, every = 9, 2
    got, R, a = run(px, phi, rho, h, omega, n, dtype, every)
    ref, Rref = oracle.rbsor_n(phi, rho, h, omega, n, every)
    tol = 2 * n * per_update(dtype)
    check(got, ref, tol)
    check_reports(R, Rref, max(np.max(np.abs(phi)), np.max(np.abs(ref))), rho, h, tol)
    assert np.array_equal(a, phi)  # phi_in is not written out of place


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("omega", [1.25, 1.5, 1.9])
def test_over_relaxed_sweep_by_sweep(px, dtype, omega):
    """Each sweep from the oracle's own previous state (rounded to storage)."""
    nx, ny = 258, 132
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 31, dtype)
    state = phi
    for k in range(4):
        got, R, _ = run(px, state, rho, h, omega, 1, dtype)
        ref, Rref = oracle.rbsor_n(state, rho, h, omega, 1, 1)
        tol = 2 * omega * per_update(dtype)
        check(got, ref, tol)
        check_reports(R, Rref, np.max(np.abs(state)), rho, h, per_update(dtype))
        state = host(dev(ref, dtype))


@pytest.mark.parametrize("layout", ["pitched", "offset"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_general_layouts(px, layout, dtype):
    """Pitched rows and a misaligned base take the scalar path; same results."""
    nx, ny = 132, 70
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 5, dtype)
    got, R, _ = run(px, phi, rho, h, 1.0, 5, dtype, 1, layout)
    ref, Rref = oracle.rbsor_n(phi, rho, h, 1.0, 5, 1)
    tol = 10 * per_update(dtype)
    check(got, ref, tol)
    check_reports(R, Rref, np.max(np.abs(phi)), rho, h, tol)


@pytest.mark.parametrize("nsweeps", [1, 2, 5, 6])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_in_place_equals_out_of_place(px, nsweeps, dtype):
    """In place (odd and even counts) gives bitwise the out-of-place result."""
    nx, ny = 160, 96
    phi, rho = fields(nx, ny, 9, dtype)
    a, R_a, _ = run(px, phi, rho, 1.0 / nx, 1.0, nsweeps, dtype, 1)
    b, R_b, _ = run(px, phi, rho, 1.0 / nx, 1.0, nsweeps, dtype, 1, inplace=True)
    assert np.array_equal(a, b)
    assert np.array_equal(R_a, R_b)


def test_vector_and_scalar_paths_bitwise(px):
    """The 16-byte vector path and the scalar path evaluate the same
    expressions per cell, so they agree bitwise."""
    nx, ny = 256, 64
    for dtype in (torch.float32, torch.float64):
        phi, rho = fields(nx, ny, 3, dtype)
        a, Ra, _ = run(px, phi, rho, 1.0 / nx, 1.3, 4, dtype, 1, "plain")
        b, Rb, _ = run(px, phi, rho, 1.0 / nx, 1.3, 4, dtype, 1, "pitched")
        assert np.array_equal(a, b) and np.array_equal(Ra, Rb)


def test_zero_sweeps_and_empty(px):
    nx, ny = 64, 32
    phi, rho = fields(nx, ny, 1, torch.float32)
    got, R, _ = run(px, phi, rho, 1 / nx, 1.0, 0, torch.float32, 1)
    assert np.array_equal(got, phi) and R.size == 0
    e = torch.zeros(0, 6, dtype=torch.float32, device="cuda")
    px.rbsor_n(e, e.clone(), e.clone(), 1.0, 1.0, 3)


def test_rejects_odd_extents(px):
    a = torch.zeros((64, 63), dtype=torch.float32, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.rbsor_n(a, torch.zeros_like(a), torch.zeros_like(a), 1 / 63, 1.0, 2)
    assert ei.value.status == px.PX_EINVAL
    a = torch.zeros((63, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.rbsor_n(a, torch.zeros_like(a), torch.zeros_like(a), 1 / 64, 1.0, 2)
    assert ei.value.status == px.PX_EINVAL


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_discrete_solution_is_a_fixed_point(px, omega):
    """A property that holds at any size: the exact solution of the periodic
    discrete Poisson problem (spectral division by the 5-point symbol) is left
    in place by a sweep, and its report is round-off."""
    n = 512
    h = 1.0 / n
    rho, _ = synth.modes_rho(n, n, 8, 16, 11, noise_sigma=0.1)
    k = 2 * np.pi * np.fft.fftfreq(n)
    sym = (2 * np.cos(k)[None, :] + 2 * np.cos(k)[:, None] - 4) / h**2
    sym[0, 0] = 1.0
    R = np.fft.fft2(rho)
    R[0, 0] = 0.0
    phi = np.real(np.fft.ifft2(R / sym))
    got, rep, _ = run(px, phi, rho, h, omega, 3, torch.float64, 1)
    check(got, phi, 3 * 2 * omega * 1e-12)
    sc = 8.0 * np.max(np.abs(phi)) / h**2 + np.max(np.abs(rho))
    assert np.all(rep <= 1e-12 * sc), rep


def _window(a, j0, i0, size):
    ny, nx = a.shape
    jj = (np.arange(j0, j0 + size) % ny)[:, None]
    ii = (np.arange(i0, i0 + size) % nx)[None, :]
    return a[jj, ii]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_full_size_sampled(px, dtype):
    """16384 x 16384, the large-field workload (64 modes k,l in 1..512 plus
    sigma = 0.1 noise), Gauss-Seidel in the benchmark's launch configuration
    (a report every sweep). Four sweeps from phi0 = 0; 40 windows sampled over
    the grid (edges and corners included; each origin has x + y even, so the
    window keeps the colouring) are recomputed by the oracle on a periodic
    window. A sweep carries information two cells (red one, black two), so
    cells 2n + 2 away from the window's edges are unaffected by its own wrap.
    The state-0 report is max|rho| exactly."""
    n = 16384
    h = 1.0 / n
    rho_t = dev(synth.large_field_rho(n), dtype)
    rho = host(rho_t)
    phi = torch.zeros_like(rho_t)
    out = torch.empty_like(rho_t)
    nsw = 4
    resid = torch.zeros(nsw, dtype=torch.float64, device="cuda")
    px.rbsor_n(phi, out, rho_t, h, 1.0, nsw, resid, 1)
    torch.cuda.synchronize()
    rep = resid.cpu().numpy()
    assert rep[0] == np.max(np.abs(rho))
    assert np.all(np.isfinite(rep))
    o = host(out)
    tol = 2 * nsw * per_update(dtype)
    rng = np.random.default_rng(91)
    size, m = 48, 2 * nsw + 2
    starts = [(-m, -m), (n - size + m, n - size + m), (-m, n // 2), (n // 2, -m)]
    for _ in range(36):
        j0, i0 = (int(v) for v in rng.integers(0, n, 2))
        starts.append((j0, i0 - ((i0 + j0) & 1)))
    scale = np.max(np.abs(o))
    for (j0, i0) in starts:
        assert (j0 + i0) % 2 == 0
        w_rho = _window(rho, j0, i0, size)
        ref, _ = oracle.rbsor_n(np.zeros_like(w_rho), w_rho, h, 1.0, nsw, 0)
        got = _window(o, j0, i0, size)
        c = slice(m, size - m)
        assert np.max(np.abs(got[c, c] - ref[c, c])) <= tol * scale, (j0, i0)


@pytest.mark.parametrize("sweeps", [1, 2, 3, 4])
def test_register_wavefront_depths_bitwise(sweeps):
    """The FP32 register wavefront at 1..4 red-black sweeps per launch gives
    bitwise the states and reports of the two-pass kernels (the oracle tests
    pin those); the depth is selected on a context of its own
    (PX_OPT_RB_SWEEPS_PER_LAUNCH). Sizes cover several strips and ranges,
    ragged strips, strips wider than the grid and launches of dynamic balance."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_RB_SWEEPS_PER_LAUNCH, sweeps)
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        for (nx, ny) in [(4096, 4096), (1000, 1002), (260, 150), (16, 8), (4, 4), (124, 64),
                         (8, 300)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)

            # the pitched copies take the two-pass kernels (row pitch nx + 1)
            def pitched(a):
                b = torch.zeros(ny, nx + 1, device="cuda", dtype=torch.float32)[:, :nx]
                b.copy_(a)
                return b
            pp, rp, op = pitched(phi), pitched(rho), pitched(torch.zeros_like(phi))
            out = torch.empty_like(phi)
            r1 = torch.zeros(11, dtype=torch.float64, device="cuda")
            r2 = torch.zeros_like(r1)
            for omega in (1.0, 1.6):
                px.rbsor_n(pp, op, rp, h, omega, 11, r1, 1, ctx=ctx)
                px.rbsor_n(phi, out, rho, h, omega, 11, r2, 1, ctx=ctx)
                torch.cuda.synchronize()
                assert torch.equal(op, out) and torch.equal(r1, r2), (nx, ny, omega)
    finally:
        ctx.close()


def test_fp64_fused_sweep_bitwise():
    """FP64 vector layouts run one fused launch per sweep (new red values of
    the rows and columns next to a warp's block recomputed from the input);
    the red pass + black pass form, selected with PX_OPT_RB_FP64_PASSES = 2,
    evaluates the same expressions per cell, so states and reports agree
    bitwise (the oracle tests above pin the fused form). Sizes cover several
    strips of 30 column pairs and row segments, ragged strips, strips wider
    than the grid and the smallest even extents; in place and out of place."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    fused, passes = px.Context(torch.cuda.current_device()), px.Context(torch.cuda.current_device())
    try:
        passes.set_option(px.PX_OPT_RB_FP64_PASSES, 2)
        fused.set_option(px.PX_OPT_RB_FP64_PASSES, 1)
        assert passes.get_option(px.PX_OPT_RB_FP64_PASSES) == 2
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        for (nx, ny) in [(4096, 2048), (1030, 514), (122, 66), (60, 64), (62, 6), (2, 2), (2, 130),
                         (4, 300), (16384, 8)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
            for omega, every in ((1.0, 1), (1.7, 2), (0.9, 0)):
                outs = []
                for ctx in (passes, fused):
                    out = torch.empty_like(phi)
                    r = torch.zeros(7, dtype=torch.float64, device="cuda")
                    px.rbsor_n(phi, out, rho, h, omega, 7, r if every else None, every, ctx=ctx)
                    ip = phi.clone()
                    px.rbsor_n(ip, ip, rho, h, omega, 3, None, 0, ctx=ctx)
                    torch.cuda.synchronize()
                    outs.append((out, r, ip))
                (a, ra, ia), (b, rb, ib) = outs
                assert torch.equal(a, b) and torch.equal(ra, rb) and torch.equal(ia, ib), (nx, ny, omega)
    finally:
        fused.close()
        passes.close()

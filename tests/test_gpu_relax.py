"""GPU parity of the fused relaxation path (px_relax_n, px_apply_stencil,
px_residual_norm) against the FP64 CPU oracle, through the C ABI.

Tolerances (relative max-norm; the arithmetic behind them):
  * FP64 phi, one sweep: 1e-12. The kernel evaluates C + c (s/h^2 - rho)
    with FMAs where the oracle evaluates (C + w s) - lambda rho; both round
    a handful of times at 1.1e-16, so they differ by a few ulps of |phi|.
  * FP64 phi after n sweeps: 1e-10 at n = 1000. Jacobi with omega <= 1 is
    non-expansive, so per-sweep differences add up at most linearly.
  * FP32 storage, one sweep from the oracle's state rounded to FP32: 2e-6
    (about 30 ulps of FP32); n sweeps: n * 2e-6 by the same linear growth.
  * Residual reports: measured against the scale of the summed terms,
    8 ||phi||/h^2 + ||rho||, with the same factors as phi (the residual is a
    difference of two large terms near convergence).
  * px_residual_norm and px_apply_stencil on FP64 fields evaluate in the
    oracle's exact operation order, so they are compared bitwise.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 2.0 / 3.0


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


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def scale_of(phi, rho, h):
    return 8.0 * np.max(np.abs(phi)) / h**2 + np.max(np.abs(rho))


def fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    rho = synth.random_field(rng, nx, ny)
    phi = synth.random_field(rng, nx, ny, zero_mean=False)
    return phi, rho


def run_gpu(px, phi, rho, h, nsweeps, dtype, tblock=0, every=1, layout="plain"):
    """Runs px.relax_n on copies of phi/rho; layout 'plain' (aligned, vector path),
    'pitched' (odd pitch -> general path) or 'offset' (misaligned base)."""
    ny, nx = phi.shape
    if layout == "plain":
        a, r = dev(phi, dtype), dev(rho, dtype)
        out = torch.empty_like(a)
    else:
        extra = 1 if layout == "pitched" else 0
        shift = 1 if layout == "offset" else 0
        def place(x):
            buf = torch.full((ny, nx + extra + shift), float("nan"), dtype=dtype, device="cuda")
            v = buf[:, shift:shift + nx]
            v.copy_(torch.from_numpy(np.ascontiguousarray(x)).to(dtype))
            return v
        a, r = place(phi), place(rho)
        out = place(np.zeros_like(phi))
    nrep = (nsweeps + every - 1) // every if every > 0 else 0
    resid = torch.zeros(max(nrep, 1), dtype=torch.float64, device="cuda")
    px.relax_n(a, out, r, h, OMEGA, nsweeps, tblock, resid if every > 0 else None, every)
    torch.cuda.synchronize()
    return host(out), resid.cpu().numpy()[:nrep]


# ------------------------------------------------------------ one sweep, FP64
@pytest.mark.parametrize("nx,ny", [(64, 64), (33, 47), (128, 96), (260, 150), (3, 5), (1, 1),
                                   (2, 7), (8, 1), (1000, 3)])
@pytest.mark.parametrize("layout", ["plain", "pitched", "offset"])
def test_one_sweep_f64(px, nx, ny, layout):
    h = 1.0 / max(nx, ny)
    phi, rho = fields(nx, ny, 10 * nx + ny)
    ref, R = oracle.sweep(phi, rho, h, OMEGA)
    got, rep = run_gpu(px, phi, rho, h, 1, torch.float64, tblock=1, layout=layout)
    assert relerr(got, ref) <= 1e-12
    assert abs(rep[0] - R) <= 1e-12 * scale_of(phi, rho, h)


# ------------------------------------------------------------ one sweep, FP32
@pytest.mark.parametrize("nx,ny", [(64, 64), (33, 47), (128, 96), (260, 150), (4, 4), (5, 3)])
@pytest.mark.parametrize("layout", ["plain", "pitched"])
def test_one_sweep_f32(px, nx, ny, layout):
    """Input = the oracle's FP64 state rounded to FP32; oracle sweeps the
    widened FP32 values in FP64 (the FP32-storage reading of the method)."""
    h = 1.0 / max(nx, ny)
    phi, rho = fields(nx, ny, 7 * nx + ny)
    phi32 = phi.astype(np.float32).astype(np.float64)
    rho32 = rho.astype(np.float32).astype(np.float64)
    ref, R = oracle.sweep(phi32, rho32, h, OMEGA)
    got, rep = run_gpu(px, phi32, rho32, h, 1, torch.float32, tblock=1, layout=layout)
    assert relerr(got, ref) <= 2e-6
    assert abs(rep[0] - R) <= 2e-6 * scale_of(phi32, rho32, h)


# ------------------------------------------------------------ temporal blocking
@pytest.mark.parametrize("tb", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("nx,ny", [(128, 128), (260, 150), (16, 8), (400, 260)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_temporal_blocking(px, tb, nx, ny, dtype):
    """tb sweeps fused in one launch, and 2 tb + 1 sweeps (two full blocks and
    a remainder), each against the oracle with per-sweep residual reports."""
    h = 1.0 / max(nx, ny)
    phi, rho = fields(nx, ny, 100 * tb + nx)
    if dtype == torch.float32:
        phi = phi.astype(np.float32).astype(np.float64)
        rho = rho.astype(np.float32).astype(np.float64)
        tol = 2e-6
    else:
        tol = 1e-12
    for n in (tb, 2 * tb + 1):
        ref, R = oracle.relax_n(phi, rho, h, OMEGA, n, 1)
        got, rep = run_gpu(px, phi, rho, h, n, dtype, tblock=tb)
        assert relerr(got, ref) <= n * tol, n
        sc = scale_of(ref, rho, h) + scale_of(phi, rho, h)
        assert np.max(np.abs(rep - R)) <= n * tol * sc, n


# ------------------------------------------------------------ small-field workload
@pytest.mark.parametrize("tblock", [1, 4])
def test_small_field_1000_sweeps(px, tblock):
    """64x64, 8 modes, FP64, omega = 2/3, phi0 = 0, 1000 sweeps, residual every
    10 sweeps: 1e-10 after 1000 sweeps."""
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    ref, R = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 1000, 10)
    got, rep = run_gpu(px, np.zeros_like(rho), rho, h, 1000, torch.float64, tblock=tblock,
                       every=10)
    assert rep.shape == (100,)
    assert relerr(got, ref) <= 1e-10
    assert np.max(np.abs(rep - R)) <= 1e-10 * scale_of(ref, rho, h)


# ------------------------------------------------------------ in place, reports
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 5, 8, 9])
@pytest.mark.parametrize("tblock", [1, 2, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_in_place(px, nsweeps, tblock, dtype):
    nx, ny = 136, 96
    h = 1.0 / nx
    phi, rho = fields(nx, ny, nsweeps * 3 + tblock)
    phi = phi.astype(np.float32).astype(np.float64)
    rho = rho.astype(np.float32).astype(np.float64)
    ref, R = oracle.relax_n(phi, rho, h, OMEGA, nsweeps, 2)
    a, r = dev(phi, dtype), dev(rho, dtype)
    resid = torch.zeros(len(R), dtype=torch.float64, device="cuda")
    px.relax_n(a, a, r, h, OMEGA, nsweeps, tblock, resid, 2)
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert relerr(host(a), ref) <= nsweeps * tol
    assert np.max(np.abs(resid.cpu().numpy() - R)) <= nsweeps * tol * scale_of(ref, rho, h) * 2


def test_report_indexing(px):
    """report_every = 3 over 10 sweeps reports states 0, 3, 6, 9."""
    nx = ny = 48
    h = 1.0 / 48
    phi, rho = fields(nx, ny, 3)
    ref, R = oracle.relax_n(phi, rho, h, OMEGA, 10, 3)
    assert len(R) == 4
    for tb in (1, 2, 4, 8):
        got, rep = run_gpu(px, phi, rho, h, 10, torch.float64, tblock=tb, every=3)
        assert rep.shape == (4,)
        assert np.max(np.abs(rep - R)) <= 1e-11 * scale_of(phi, rho, h)


def test_zero_sweeps_copies_and_empty_grid(px):
    phi, rho = fields(40, 24, 1)
    got, _ = run_gpu(px, phi, rho, 1 / 40, 0, torch.float64, every=0)
    assert np.array_equal(got, phi)
    e = torch.zeros(0, 5, dtype=torch.float64, device="cuda")
    px.relax_n(e, e.clone(), e.clone(), 0.1, OMEGA, 3)


# ------------------------------------------------------------ ghosted layout
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ghost_layout(px, dtype):
    """Box of 64 x 64 stored as 66 x 66 (interior at offset 67). Input ghosts
    hold NaN and must be ignored; output ghosts are periodic images."""
    n, h = 64, 1.0 / 64
    phi, rho = fields(n, n, 21)
    phi = phi.astype(np.float32).astype(np.float64)
    rho = rho.astype(np.float32).astype(np.float64)
    ref, R = oracle.relax_n(phi, rho, h, OMEGA, 3, 1)
    def ghosted(x):
        g = np.full((n + 2, n + 2), np.nan)
        g[1:-1, 1:-1] = x
        return dev(g, dtype)
    a, r = ghosted(phi), ghosted(rho)
    out = ghosted(np.zeros_like(phi))
    resid = torch.zeros(3, dtype=torch.float64, device="cuda")
    px.relax_n(a, out, r, h, OMEGA, 3, 0, resid, 1, ghost=1)
    o = host(out)
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert relerr(o[1:-1, 1:-1], ref) <= 3 * tol
    assert np.array_equal(o, oracle.fill_ghosts(o))
    assert np.max(np.abs(resid.cpu().numpy() - R)) <= 3 * tol * scale_of(ref, rho, h)
    # stencil on the ghosted layout
    lp = ghosted(np.zeros_like(phi))
    px.apply_stencil(a, lp, h, ghost=1)
    L = host(lp)
    assert np.array_equal(L, oracle.fill_ghosts(L))
    Lref = oracle.apply_stencil(phi, h)
    assert relerr(L[1:-1, 1:-1], Lref) <= (0 if dtype == torch.float64 else 1e-5)


# ------------------------------------------------------------ stencil, residual norm
@pytest.mark.parametrize("nx,ny", [(64, 64), (33, 47), (5, 3)])
def test_apply_stencil_and_residual_norm_bitwise_f64(px, nx, ny):
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 5)
    a, r = dev(phi, torch.float64), dev(rho, torch.float64)
    out = torch.empty_like(a)
    px.apply_stencil(a, out, h)
    assert np.array_equal(host(out), oracle.apply_stencil(phi, h))
    R, P = px.residual_norm(a, r, h)
    Ro, Po = oracle.residual_norm(phi, rho, h)
    assert R == Ro and P == Po


def test_residual_norm_f32_is_widened_f64(px):
    nx, ny = 96, 80
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 8)
    a, r = dev(phi, torch.float32), dev(rho, torch.float32)
    R, P = px.residual_norm(a, r, h)
    Ro, Po = oracle.residual_norm(host(a), host(r), h)
    assert R == Ro and P == Po


def test_nan_propagates(px):
    nx = ny = 64
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 9)
    phi[10, 20] = np.nan
    for dtype in (torch.float64, torch.float32):
        for tb in (1, 4):
            _, rep = run_gpu(px, phi, rho, h, 4, dtype, tblock=tb)
            assert np.isnan(rep[0])
        R, _ = px.residual_norm(dev(phi, dtype), dev(rho, dtype), h)
        assert np.isnan(R)


def test_residual_report_equals_residual_norm_of_state(px):
    """The report of state k equals px_residual_norm of that state (FP64)."""
    nx = ny = 128
    h = 1.0 / nx
    phi, rho = fields(nx, ny, 12)
    a, r = dev(phi, torch.float64), dev(rho, torch.float64)
    out = torch.empty_like(a)
    resid = torch.zeros(5, dtype=torch.float64, device="cuda")
    px.relax_n(a, out, r, h, OMEGA, 5, 1, resid, 1)
    mid = torch.empty_like(a)
    px.relax_n(a, mid, r, h, OMEGA, 3, 1)
    R3, _ = px.residual_norm(mid, r, h)
    assert abs(resid[3].item() - R3) <= 1e-13 * scale_of(host(mid), rho, h)


# ------------------------------------------------------------ argument checks
def test_invalid_arguments(px):
    a = torch.zeros(32, 32, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    r = torch.zeros_like(a)
    bad = [
        dict(tblock=9), dict(tblock=-1), dict(nsweeps=-1), dict(h=0.0), dict(h=float("nan")),
        dict(omega=float("nan")), dict(report_every=-2),
    ]
    for kw in bad:
        args = dict(h=1 / 32, omega=OMEGA, nsweeps=2, tblock=0, report_every=0)
        args.update(kw)
        with pytest.raises(px.PxError) as ei:
            px.relax_n(a, b, r, args["h"], args["omega"], args["nsweeps"], args["tblock"],
                       None, args["report_every"])
        assert ei.value.status == px.PX_EINVAL, kw
    # partial overlap of phi_in and phi_out, rho aliasing phi_out
    big = torch.zeros(40, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(px.PxError):
        px.relax_n(big[0:32], big[4:36], r, 1 / 32, OMEGA, 1)
    with pytest.raises(px.PxError):
        px.relax_n(a, b, b, 1 / 32, OMEGA, 1)
    # raw ABI: ld smaller than nx, bad dtype, NULL pointer
    lib = px.load_library()
    ctx = px.context()
    for g in (px.Grid(32, 32, 16, 0, 0, 1 / 32), px.Grid(32, 32, 32, 0, 5, 1 / 32),
              px.Grid(32, 32, 32, 2, 0, 1 / 32), px.Grid(-1, 32, 32, 0, 0, 1 / 32)):
        s = lib.px_relax_n(ctx.handle, ctypes.byref(g), a.data_ptr(), b.data_ptr(),
                           r.data_ptr(), OMEGA, 1, 0, None, 0, None)
        assert s == px.PX_EINVAL
        assert len(lib.px_last_error(ctx.handle)) > 0
    g = px.Grid(32, 32, 32, 0, 0, 1 / 32)
    assert lib.px_relax_n(ctx.handle, ctypes.byref(g), None, b.data_ptr(), r.data_ptr(),
                          OMEGA, 1, 0, None, 0, None) == px.PX_EINVAL


def test_report_buffer_next_to_field(px):
    """A report buffer directly below phi_out in one allocation is accepted
    (the check measures each range by its own length); one that overlaps
    phi_out is rejected before anything is written. Both entry points."""
    nx = ny = 64
    phi, rho = fields(nx, ny, 21)
    for entry in ("relax_n", "relax_n_static"):
        fn = getattr(px, entry)
        buf = torch.zeros(256 + nx * ny * 4, dtype=torch.uint8, device="cuda")
        resid = buf[0:32].view(torch.float64)              # 4 reports, then a gap
        out = buf[256:].view(torch.float32).view(ny, nx)   # phi_out right after
        a, r = dev(phi, torch.float32), dev(rho, torch.float32)
        fn(a, out, r, 1.0 / nx, OMEGA, 4, 4, resid, 1)
        torch.cuda.synchronize()
        ref, R = oracle.relax_n(host(a), host(r), 1.0 / nx, OMEGA, 4, 1)
        assert np.max(np.abs(host(out) - ref)) <= 4 * 2e-6 * np.max(np.abs(ref))
        assert np.all(host(resid) > 0)
        # a report buffer inside phi_out: rejected, phi_out untouched
        before = out.clone()
        bad = buf[256 + 64:256 + 96].view(torch.float64)
        with pytest.raises(px.PxError) as ei:
            fn(a, out, r, 1.0 / nx, OMEGA, 4, 4, bad, 1)
        assert ei.value.status == px.PX_EINVAL
        torch.cuda.synchronize()
        assert torch.equal(out, before)


# ------------------------------------------------------------ full size, sampled
def _window(a, j0, i0, size):
    ny, nx = a.shape
    jj = (np.arange(j0, j0 + size) % ny)[:, None]
    ii = (np.arange(i0, i0 + size) % nx)[None, :]
    return a[jj, ii]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_full_size_sampled(px, dtype):
    """16384 x 16384, the large-field workload (64 modes k,l in 1..512 plus
    sigma = 0.1 noise), in the benchmark's launch configuration (automatic
    depth, a report every sweep). Eight sweeps from phi0 = 0; 48 windows
    sampled over the grid (edges and corners included) are recomputed by the
    oracle on a periodic window whose centre is unaffected by the window's
    own wrap after 8 sweeps. The state-0 report is max|rho| exactly."""
    n = 16384
    h = 1.0 / n
    rho64 = synth.large_field_rho(n)
    rho_t = dev(rho64, dtype)
    rho = host(rho_t)  # values as stored
    phi = torch.zeros_like(rho_t)
    out = torch.empty_like(rho_t)
    nsw = 8
    resid = torch.zeros(nsw, dtype=torch.float64, device="cuda")
    px.relax_n(phi, out, rho_t, h, OMEGA, nsw, 0, resid, 1)
    torch.cuda.synchronize()
    rep = resid.cpu().numpy()
    assert rep[0] == np.max(np.abs(rho))
    o = out.cpu().numpy().astype(np.float64)
    tol = (2e-6 if dtype == torch.float32 else 1e-12) * nsw
    rng = np.random.default_rng(77)
    size, m = 48, nsw + 2
    starts = [(-m, -m), (n - size + m, n - size + m), (-m, n // 2), (n // 2, -m)]
    starts += [tuple(rng.integers(0, n, 2)) for _ in range(44)]
    scale = np.max(np.abs(o))
    for (j0, i0) in starts:
        w_rho = _window(rho, j0, i0, size)
        ref, _ = oracle.relax_n(np.zeros_like(w_rho), w_rho, h, OMEGA, nsw, 0)
        got = _window(o, j0, i0, size)
        c = slice(m, size - m)
        assert np.max(np.abs(got[c, c] - ref[c, c])) <= tol * scale, (j0, i0)
    del o, rho64


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_full_size_every_report_and_state(px, dtype):
    """The same 16384^2 workload and launch configuration (automatic depth:
    the FP32 register wavefront at depth 8 with run-time row balancing, or
    the FP64 streaming kernel), eight sweeps with a report every sweep,
    against the serial FP64 oracle run on the whole field: every report
    (states 0..7, not only state 0) and every cell of the final state."""
    n = 16384
    h = 1.0 / n
    rho64 = synth.large_field_rho(n)
    rho_t = dev(rho64, dtype)
    rho = host(rho_t)
    del rho64
    phi = torch.zeros_like(rho_t)
    out = torch.empty_like(rho_t)
    nsw = 8
    resid = torch.zeros(nsw, dtype=torch.float64, device="cuda")
    px.relax_n(phi, out, rho_t, h, OMEGA, nsw, 0, resid, 1)
    torch.cuda.synchronize()
    got_rep = resid.cpu().numpy()
    del phi, rho_t
    ref, ref_rep = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, nsw, 1)
    got = out.cpu().numpy().astype(np.float64)
    del out
    tol = (2e-6 if dtype == torch.float32 else 1e-12) * nsw
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= tol * scale
    sc = 8 * scale / h**2 + np.max(np.abs(rho))
    assert np.all(np.abs(got_rep - ref_rep) <= tol * sc), (got_rep, ref_rep)
    assert got_rep[0] == np.max(np.abs(rho))

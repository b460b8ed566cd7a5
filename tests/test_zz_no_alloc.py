"""px_relax_n_static, the relax entry point that allocates nothing.

Some callers cannot call cudaMalloc: a loop that must not block on the
allocator, applications whose own memory pool owns the device, plug-ins that
may not create library contexts. For them the
library keeps its ping-pong field in a fixed 16 MiB device array. These tests
call that entry point through the C ABI and check it against px_relax_n on
the same inputs, within the parity tolerances of the relax tests (1e-12
relative for FP64, 2e-6 per sweep for FP32), on two calls in a row that both
pass through the shared array. The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 2.0 / 3.0


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    m.load_library()
    return m


def _static(px, g, a, out, r, nsweeps, tblock, resid, every):
    lib = px.load_library()
    return lib.px_relax_n_static(ctypes.byref(g), a.data_ptr(), out.data_ptr(), r.data_ptr(),
                                 OMEGA, nsweeps, tblock,
                                 resid.data_ptr() if resid is not None else None, every,
                                 torch.cuda.current_stream().cuda_stream)


def _relerr(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_static_entry_point_matches_relax_n_two_calls_in_a_row(px):
    rng = np.random.default_rng(2024)
    cases = [
        # (nx, ny, dtype, nsweeps, tblock, in_place, every, tol per sweep)
        (1024, 512, torch.float32, 9, 0, False, 1, 2e-6),   # automatic depth 8: launches 8, 1
        (300, 200, torch.float64, 5, 1, True, 2, 1e-12),    # in place, odd: staged copy
    ]
    for (nx, ny, dt, n, tb, inplace, every, tol) in cases:
        _compare(px, rng, nx, ny, dt, n, tb, inplace, every, tol, ghost=0)


def _compare(px, rng, nx, ny, dt, n, tb, inplace, every, tol, ghost):
    h = 1.0 / nx
    rho = torch.from_numpy(synth.random_field(rng, nx, ny)).to(dt)
    phi0 = torch.from_numpy(synth.random_field(rng, nx, ny, zero_mean=False)).to(dt)
    if ghost:  # interior at (1, 1) of an (ny + 2) x (nx + 2) array; input ghosts are ignored
        rho = torch.nn.functional.pad(rho, (1, 1, 1, 1), value=float("nan"))
        phi0 = torch.nn.functional.pad(phi0, (1, 1, 1, 1), value=float("nan"))
    rho, phi0 = rho.cuda(), phi0.cuda()
    nrep = (n + every - 1) // every
    # existing entry point
    ref_out = phi0.clone() if inplace else torch.empty_like(phi0)
    ref_res = torch.zeros(nrep, dtype=torch.float64, device="cuda")
    px.relax_n(ref_out if inplace else phi0, ref_out, rho, h, OMEGA, n, tb, ref_res, every,
               ghost=ghost)
    # allocation-free entry point
    a = phi0.clone()
    out = a if inplace else torch.empty_like(phi0)
    res = torch.full((nrep,), -1.0, dtype=torch.float64, device="cuda")
    g = px.grid_of(a, h, ghost)
    st = _static(px, g, a, out, rho, n, tb, res, every)
    assert st == px.PX_OK, px.load_library().px_last_error(None)
    assert px.load_library().px_last_error(None) == b""
    torch.cuda.synchronize()
    assert _relerr(out, ref_out) <= n * tol
    inner = (slice(1, -1), slice(1, -1)) if ghost else (slice(None), slice(None))
    sc = 8 * float(ref_out[inner].abs().max()) / h**2 + float(rho[inner].abs().max())
    sc = max(sc, 8 * float(phi0[inner].abs().max()) / h**2)
    assert float((res - ref_res).abs().max()) <= n * tol * sc
    if not inplace:
        assert torch.equal(a[inner], phi0[inner])  # input untouched


def test_static_entry_point_ghosted_fp64(px):
    """The ghosted layout (one ghost layer, NaN in the input ghosts, which the
    sweeps ignore): FP64 at 1e-12 per sweep, out of place and in place."""
    rng = np.random.default_rng(77)
    _compare(px, rng, 130, 97, torch.float64, 6, 1, False, 1, 1e-12, ghost=1)
    _compare(px, rng, 130, 97, torch.float64, 5, 1, True, 2, 1e-12, ghost=1)


def test_static_entry_point_allocates_nothing(px):
    """After a first call (which may look up the array's address), further
    calls leave the device's free memory unchanged: nothing is allocated."""
    nx = ny = 1024
    rng = np.random.default_rng(5)
    rho = torch.from_numpy(synth.random_field(rng, nx, ny)).float().cuda()
    a = torch.zeros_like(rho)
    b = torch.empty_like(rho)
    res = torch.zeros(17, dtype=torch.float64, device="cuda")
    g = px.grid_of(a, 1.0 / nx)
    assert _static(px, g, a, b, rho, 17, 0, res, 1) == px.PX_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _static(px, g, a, b, rho, 17, 0, res, 1) == px.PX_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_entry_point_rejects_fields_beyond_its_limit(px):
    nx, ny = 2048, 2049  # 16 MiB + one row of FP32
    a = torch.zeros(ny, nx, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    r = torch.zeros_like(a)
    g = px.grid_of(a, 1.0 / nx)
    st = _static(px, g, a, b, r, 3, 0, None, 0)
    assert st == px.PX_EINVAL
    msg = px.load_library().px_last_error(None).decode()
    assert "static scratch" in msg and "16 MiB" in msg
    # the largest square FP32 field that fits still runs
    a2 = a[:2048]
    b2 = torch.zeros_like(a2)
    r2 = torch.zeros_like(a2)
    assert _static(px, px.grid_of(a2, 1.0 / nx), a2, b2, r2, 2, 0, None, 0) == px.PX_OK
    assert px.load_library().px_last_error(None) == b""  # the failed call's message is cleared
    torch.cuda.synchronize()

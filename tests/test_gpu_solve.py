"""GPU parity of px_solve: plain sweeps to a tolerance, and FP32-storage sweeps
inside FP64 iterative refinement, against the FP64 oracle and the refinement
oracle (oracle/refine.py), through the C ABI.

The bar for a refined result is the one of the mixed-precision pattern: the
FP64 oracle's max-norm residual of the returned phi is <= 1e-10 relative. The
FP64 residual evaluation of px_residual_norm is bitwise equal to the oracle's,
so the reported rel_resid must equal the oracle's value exactly.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import refine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 2.0 / 3.0


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def oracle_rel(phi, rho, h):
    R, P = oracle.residual_norm(phi, rho, h)
    return R / P


def test_plain_fp64_to_1e8(px):
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    phi = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    info = px.solve(phi, dev(rho), h, "plain", rtol=1e-8, check_every=50)
    got = phi.cpu().numpy()
    rel = oracle_rel(got, rho, h)
    assert rel <= 1e-8 and rel == info["rel_resid"]
    # the oracle crosses 1e-8 at the same check (blocks of 50 sweeps), +-1 block
    p = np.zeros_like(rho)
    k = 0
    while oracle_rel(p, rho, h) > 1e-8:
        p, _ = oracle.relax_n(p, rho, h, OMEGA, 50, 0)
        k += 50
    assert abs(info["sweeps"] - k) <= 50
    assert info["checks"] == info["sweeps"] // 50 + 1


@pytest.mark.parametrize("shape,ghost", [((64, 64), 0), ((45, 33), 0), ((96, 72), 1)])
def test_refine_to_1e10(px, shape, ghost):
    nx, ny = shape
    h = 1.0 / nx
    rho, _ = synth.modes_rho(nx, ny, 8, 8, 31 + nx)
    if ghost:
        g = np.zeros((ny + 2, nx + 2))
        g[1:-1, 1:-1] = rho
        r_t = dev(g)
        phi = torch.zeros_like(r_t)
    else:
        r_t = dev(rho)
        phi = torch.zeros_like(r_t)
    info = px.solve(phi, r_t, h, "refine", rtol=1e-10, inner_sweeps=500, ghost=ghost)
    got = phi.cpu().numpy()
    if ghost:
        assert np.array_equal(got, oracle.fill_ghosts(got))
        got = got[1:-1, 1:-1]
    rel = oracle_rel(got, rho, h)
    assert rel <= 1e-10
    assert rel == info["rel_resid"]
    _, hist = refine.refine_solve(rho, h, OMEGA, 1e-10, 500, 400, fp32=True)
    assert abs(info["cycles"] - (len(hist) - 1)) <= 1
    assert info["sweeps"] == 500 * info["cycles"]


def test_refine_first_cycle_matches_oracle(px):
    """One cycle: the scaled FP32 residual is bitwise the oracle's; after 500 FP32
    sweeps the corrected phi agrees with the refinement oracle to FP32 accuracy
    of the correction (500 sweeps x 2e-6)."""
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    phi = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.solve(phi, dev(rho), h, "refine", rtol=0.0, inner_sweeps=500, max_sweeps=500)
    assert ei.value.status == px.PX_ENOCONV and ei.value.info["cycles"] == 1
    ref, _ = refine.refine_solve(rho, h, OMEGA, 0.0, 500, 1, fp32=True)
    got = phi.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 500 * 2e-6 * np.max(np.abs(ref))


def test_plain_fp32_solve(px):
    n, h = 128, 1.0 / 128
    rho, _ = synth.modes_rho(n, n, 8, 12, 5)
    phi = torch.zeros(n, n, dtype=torch.float32, device="cuda")
    info = px.solve(phi, dev(rho, torch.float32), h, "plain", rtol=1e-4, check_every=200)
    rel = oracle_rel(phi.double().cpu().numpy(), rho.astype(np.float32).astype(np.float64), h)
    assert rel <= 1e-4 and rel == info["rel_resid"]


def test_solve_errors(px):
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    phi = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.solve(phi, dev(rho + 1e-6), h, "plain", check_mean=True)
    assert ei.value.status == px.PX_EMEAN
    px.solve(phi.zero_(), dev(rho), h, "plain", rtol=1e-3, check_mean=True)
    with pytest.raises(px.PxError) as ei:
        px.solve(phi.zero_(), dev(rho), h, "plain", rtol=1e-12, max_sweeps=10, check_every=5)
    assert ei.value.status == px.PX_ENOCONV and ei.value.info["sweeps"] == 10
    bad = rho.copy()
    bad[3, 3] = np.nan
    with pytest.raises(px.PxError) as ei:
        px.solve(phi.zero_(), dev(bad), h, "plain")
    assert ei.value.status == px.PX_ENAN
    with pytest.raises(px.PxError) as ei:
        px.solve(phi.float(), dev(rho, torch.float32), h, "refine")
    assert ei.value.status == px.PX_EINVAL
    with pytest.raises(px.PxError) as ei:
        px.solve(phi.zero_(), dev(rho), h, "plain", check_every=0)
    assert ei.value.status == px.PX_EINVAL
    big = 2048
    rb, _ = synth.modes_rho(big, big, 4, 4, 9)
    pb = torch.zeros(big, big, dtype=torch.float64, device="cuda")
    with pytest.raises(px.PxError) as ei:
        px.solve(pb, dev(rb), 1.0 / big, "plain", rtol=1e-12, check_every=200, timeout_ms=1)
    assert ei.value.status == px.PX_ETIMEOUT


def test_refinement_workload_full_size_budgeted(px):
    """8192 x 8192 refinement field (64 modes, k,l in 1..256, sigma = 0.1 noise),
    three cycles of 500 FP32 sweeps. Its residual equals the oracle's residual of
    the returned phi bitwise, and matches 1500 plain FP64 sweeps (refinement with
    n inner sweeps is Jacobi in blocks of n) to 1e-3 relative."""
    n = 8192
    h = 1.0 / n
    rho, _ = synth.modes_rho(n, n, 64, 256, synth.workload_seed(2), noise_sigma=0.1)
    r_t = dev(rho)
    phi = torch.zeros_like(r_t)
    with pytest.raises(px.PxError) as ei:
        px.solve(phi, r_t, h, "refine", rtol=1e-10, inner_sweeps=500, max_sweeps=1500)
    info = ei.value.info
    assert ei.value.status == px.PX_ENOCONV and info["cycles"] == 3
    got = phi.cpu().numpy()
    assert oracle_rel(got, rho, h) == info["rel_resid"]
    del got
    p64 = torch.zeros_like(r_t)
    px.relax_n(p64, p64, r_t, h, OMEGA, 1500, 1)
    R64, P64 = px.residual_norm(p64, r_t, h)
    assert abs(info["rel_resid"] - R64 / P64) <= 1e-3 * (R64 / P64)

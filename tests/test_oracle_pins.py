"""Pins of the FP64 oracle against things other than itself.

The paper prints no numeric example, so every pin is mathematical:
closed-form eigenmode trajectories, a dense-matrix Jacobi iteration built from
circulant matrices, library routines (numpy eigvalsh, FFT), and invariants.
Each is chosen so that a plausible slip in the oracle (a dropped or repeated
tap, a sign, a transposed nx/ny, the residual of the output state instead of
the input state, lambda without omega) fails at least one of them.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth

OMEGA = 2.0 / 3.0


def mode_eig(k, l, nx, ny, h):
    """Closed-form discrete eigenvalue of the periodic 5-point Laplacian."""
    return -(4.0 / h**2) * (np.sin(np.pi * k / nx) ** 2 + np.sin(np.pi * l / ny) ** 2)


def mode_gain(k, l, nx, ny, omega):
    """Per-sweep factor of weighted Jacobi on mode (k, l)."""
    return 1.0 - omega * (np.sin(np.pi * k / nx) ** 2 + np.sin(np.pi * l / ny) ** 2)


def mode_field(mode, nx, ny):
    vx, vy = synth.mode_vectors(mode, nx, ny)
    return np.outer(vy, vx)


def dense_laplacian(nx, ny, h):
    """(1/h^2) [I_ny (x) C_nx + C_ny (x) I_nx] with C_n the periodic second
    difference built as a circulant (first column -2, 1, 0, ..., 0, 1)."""
    def circ(n):
        col = np.zeros(n)
        col[0] += -2.0
        col[1 % n] += 1.0
        col[(n - 1) % n] += 1.0
        return scipy.linalg.circulant(col)
    return (np.kron(np.eye(ny), circ(nx)) + np.kron(circ(ny), np.eye(nx))) / h**2


# ---------------------------------------------------------------- P1 closed form
def test_stencil_eigenmodes_closed_form():
    nx, ny, h = 48, 40, 1.0 / 48
    rng = np.random.default_rng(1)
    for _ in range(6):
        m = synth.Mode(1.0, int(rng.integers(1, 24)), int(rng.integers(1, 20)),
                       rng.choice(["sin", "cos"]), rng.choice(["sin", "cos"]))
        v = mode_field(m, nx, ny)
        Lv = oracle.apply_stencil(v, h)
        mu = mode_eig(m.k, m.l, nx, ny, h)
        assert np.max(np.abs(Lv - mu * v)) <= 1e-12 * abs(mu)


def test_small_field_trajectory_matches_closed_form():
    """64x64 8-mode field, 1000 sweeps from 0: phi_n and every reported
    residual follow phi_n = sum A/mu (1 - g^n) v, r_n = sum A g^n v."""
    n, h = 64, 1.0 / 64
    rho, modes = synth.small_field_rho(synth.workload_seed(0))
    fields = [mode_field(m, n, n) for m in modes]
    mus = [mode_eig(m.k, m.l, n, n, h) for m in modes]
    gs = [mode_gain(m.k, m.l, n, n, OMEGA) for m in modes]
    every = 10
    phi, rep = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 1000, every)
    assert rep.shape == (100,)
    for kk in range(100):
        st = kk * every
        r_exact = sum(m.amp * g**st * f for m, g, f in zip(modes, gs, fields))
        R = np.max(np.abs(r_exact))
        assert abs(rep[kk] - R) <= 1e-11 * np.max(np.abs(rho)), kk
    phi_exact = sum(m.amp / mu * (1 - g**1000) * f for m, mu, g, f in zip(modes, mus, gs, fields))
    err = np.max(np.abs(phi - phi_exact)) / np.max(np.abs(phi_exact))
    assert err <= 1e-12


@pytest.mark.parametrize("k,l,g", [(16, 16, 1.0 / 3.0), (32, 32, -1.0 / 3.0)])
def test_special_gain_values(k, l, g):
    """At N=64, omega=2/3 the (16,16) mode decays by exactly 1/3 per sweep and
    the (32,32) mode flips sign with factor -1/3."""
    n, h = 64, 1.0 / 64
    m = synth.Mode(1.0, k, l, "cos", "sin" if k == 16 else "cos")
    rho = mode_field(m, n, n)
    phi = np.zeros_like(rho)
    prev = rho.copy()
    for _ in range(5):
        phi, _ = oracle.sweep(phi, rho, h, OMEGA)
        r = rho - oracle.apply_stencil(phi, h)
        assert np.max(np.abs(r - g * prev)) <= 1e-12
        prev = r


def test_one_one_mode_after_1000():
    """(1,1) mode at N=64: g = 1 - (4/3) sin^2(pi/64) ~ 0.99679, g^1000 ~ 0.0401."""
    n, h = 64, 1.0 / 64
    g = mode_gain(1, 1, n, n, OMEGA)
    assert abs(g - 0.99679) < 5e-6
    m = synth.Mode(1.0, 1, 1, "sin", "cos")
    rho = mode_field(m, n, n)
    _, rep = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 1001, 1000)
    assert abs(rep[1] / rep[0] - g**1000) <= 1e-12
    assert abs(g**1000 - 0.0401) < 1e-4


# ---------------------------------------------------------------- P2 dense matrix
@pytest.mark.parametrize("nx,ny", [(8, 8), (3, 5), (5, 3), (7, 4), (4, 6), (2, 3), (1, 4)])
def test_dense_matrix_jacobi(nx, ny):
    h = 1.0 / max(nx, ny)
    rng = np.random.default_rng(100 + nx * 10 + ny)
    rho = rng.standard_normal((ny, nx))
    phi0 = rng.standard_normal((ny, nx))
    A = dense_laplacian(nx, ny, h)
    # The method's Jacobi divides by the fixed centre tap -4/h^2 (lambda = omega h^2/4),
    # which is diag(A) whenever both sides have at least 2 cells.
    D = np.full(nx * ny, -4.0 / h**2)
    if nx >= 2 and ny >= 2:
        assert np.array_equal(np.diag(A), D)
    for omega in (0.5, OMEGA, 1.0):
        x = phi0.reshape(-1).copy()
        b = rho.reshape(-1)
        ref_res, xs = [], []
        for _ in range(30):
            ref_res.append(np.max(np.abs(b - A @ x)))
            x = x + omega * (b - A @ x) / D
            xs.append(x.copy())
        phi, rep = oracle.relax_n(phi0, rho, h, omega, 30, 1)
        scale = np.max(np.abs(xs[-1]))
        assert np.max(np.abs(phi.reshape(-1) - xs[-1])) <= 1e-13 * scale
        rscale = max(ref_res)
        assert np.max(np.abs(np.array(ref_res) - rep)) <= 1e-13 * rscale
        # apply_stencil and residual_norm against the same matrix
        assert np.allclose(oracle.apply_stencil(phi0, h).reshape(-1), A @ phi0.reshape(-1),
                           rtol=0, atol=1e-13 * np.max(np.abs(A)) * np.max(np.abs(phi0)))
        R, P = oracle.residual_norm(phi0, rho, h)
        assert abs(R - np.max(np.abs(b - A @ phi0.reshape(-1)))) <= 1e-13 * R
        assert P == np.max(np.abs(rho))


# ---------------------------------------------------------------- P3 library routines
def test_spectrum_matches_eigvalsh():
    nx, ny, h = 6, 5, 1.0 / 6
    A = dense_laplacian(nx, ny, h)
    ev = np.sort(np.linalg.eigvalsh(A))
    cf = np.sort([mode_eig(k, l, nx, ny, h) for k in range(nx) for l in range(ny)])
    assert np.max(np.abs(ev - cf)) <= 1e-12 * np.max(np.abs(cf))


def test_stencil_matches_fft_symbol():
    nx, ny, h = 40, 24, 1.0 / 40
    phi = np.random.default_rng(7).standard_normal((ny, nx))
    kx = np.arange(nx)
    ky = np.arange(ny)
    sym = (mode_eig(kx[None, :], 0, nx, ny, h) + mode_eig(0, ky[:, None], nx, ny, h))
    ref = np.real(np.fft.ifft2(np.fft.fft2(phi) * sym))
    out = oracle.apply_stencil(phi, h)
    assert np.max(np.abs(out - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_jacobi_converges_to_fft_solution():
    n, h = 16, 1.0 / 16
    rho = synth.random_field(np.random.default_rng(3), n, n)
    k = np.arange(n)
    sym = mode_eig(k[None, :], 0, n, n, h) + mode_eig(0, k[:, None], n, n, h)
    sym[0, 0] = 1.0
    hat = np.fft.fft2(rho) / sym
    hat[0, 0] = 0.0
    exact = np.real(np.fft.ifft2(hat))
    phi, rep = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 2500, 500)
    phi -= phi.mean()
    assert np.max(np.abs(phi - exact)) <= 1e-10 * np.max(np.abs(exact))
    assert rep[-1] < rep[0]
    # lstsq on the dense matrix gives the same minimum-norm solution
    A = dense_laplacian(n, n, h)
    sol = np.linalg.lstsq(A, rho.reshape(-1), rcond=None)[0].reshape(n, n)
    assert np.max(np.abs(sol - exact)) <= 1e-10 * np.max(np.abs(exact))


# ---------------------------------------------------------------- P4 invariants
def test_mean_is_preserved():
    n, h = 32, 1.0 / 32
    rng = np.random.default_rng(11)
    rho = synth.random_field(rng, n, n)
    phi0 = synth.random_field(rng, n, n, zero_mean=False)
    m0 = phi0.mean()
    phi, _ = oracle.relax_n(phi0, rho, h, OMEGA, 200, 0)
    assert abs(phi.mean() - m0) <= 200 * 1e-15 * max(1.0, np.max(np.abs(phi0)))


def test_residual_reports_are_input_state_norms():
    n, h = 24, 1.0 / 24
    rng = np.random.default_rng(12)
    rho = synth.random_field(rng, n, n)
    phi = synth.random_field(rng, n, n)
    for _ in range(4):
        R_in, _ = oracle.residual_norm(phi, rho, h)
        nxt, R = oracle.sweep(phi, rho, h, OMEGA)
        assert R == R_in
        R_out, _ = oracle.residual_norm(nxt, rho, h)
        assert R != R_out
        phi = nxt


def test_error_energy_never_grows():
    """|g| <= 1 for omega in (0, 1]: the l2 norm of the residual is non-increasing."""
    n, h = 20, 1.0 / 20
    rng = np.random.default_rng(13)
    rho = synth.random_field(rng, n, n)
    phi = np.zeros_like(rho)
    prev = np.inf
    for _ in range(50):
        r = rho - oracle.apply_stencil(phi, h)
        e = np.sqrt(np.sum(r * r))
        assert e <= prev * (1 + 1e-14)
        prev = e
        phi, _ = oracle.sweep(phi, rho, h, OMEGA)


def test_nan_propagates_to_residual():
    n, h = 8, 1.0 / 8
    rho = np.zeros((n, n))
    phi = np.zeros((n, n))
    phi[3, 4] = np.nan
    _, R = oracle.sweep(phi, rho, h, OMEGA)
    assert np.isnan(R)
    R2, _ = oracle.residual_norm(phi, rho, h)
    assert np.isnan(R2)


# ---------------------------------------------------------------- P6 fused vs unfused
def test_unfused_program_equals_fused_bitwise():
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    phi0 = synth.random_field(np.random.default_rng(5), n, n)
    iters = 25
    pu, ru = oracle.relax_unfused(phi0, rho, h, 0.5, iters)
    pf, rf = oracle.relax_n(phi0, rho, h, 0.5, iters + 1, 1)
    pf_n, _ = oracle.relax_n(phi0, rho, h, 0.5, iters, 0)
    assert np.array_equal(pu, pf_n)
    assert np.array_equal(ru, rf[1:])


def test_ghosted_layout_equals_unghosted_bitwise():
    """Box of n x n stored with m = n + 2 (interior at offset m + 1 = 67 for
    n = 64, the paper's box), periodic ghosts refilled before each sweep."""
    n, h = 64, 1.0 / 64
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    phi0 = synth.random_field(np.random.default_rng(6), n, n)
    X = np.zeros((n + 2, n + 2))
    X[1:-1, 1:-1] = phi0
    assert X.reshape(-1)[(n + 2) + 1] == phi0[0, 0]
    G, rg = oracle.relax_ghosted(X, rho, h, OMEGA, 7)
    P, rp = oracle.relax_n(phi0, rho, h, OMEGA, 7, 1)
    assert np.array_equal(G[1:-1, 1:-1], P)
    assert np.array_equal(rg, rp)
    F = oracle.fill_ghosts(G)
    assert np.array_equal(F[0, 1:-1], F[n, 1:-1]) and np.array_equal(F[n + 1, 1:-1], F[1, 1:-1])
    assert np.array_equal(F[1:-1, 0], F[1:-1, n]) and np.array_equal(F[1:-1, n + 1], F[1:-1, 1])


def test_openmp_mode_equals_serial():
    n, h = 96, 1.0 / 96
    rho = synth.random_field(np.random.default_rng(9), n, n)
    phi0 = np.zeros_like(rho)
    p1, rep = oracle.relax_n(phi0, rho, h, OMEGA, 9, 1)
    p2, Rlast, used = oracle.relax_omp(phi0, rho, h, OMEGA, 9, 4)
    assert used >= 1
    assert np.array_equal(p1, p2)
    assert Rlast == rep[-1]

"""Pins of the multigrid V-cycle oracle (oracle/mg.py). Every pin is
mathematical and none compares the oracle with itself:
  - restriction and prolongation of Fourier modes against their closed forms
    (the 2 x 2 mean multiplies a mode by cos(pi k h) cos(pi l h); bilinear
    interpolation between cell centres multiplies it by a per-dimension factor
    that depends on which quarter of the coarse cell the fine centre is in);
  - the two-level cycle against dense matrices built from the definitions by
    geometry (L by its stencil, R as block means, P from bilinear weights of
    periodic centre distances, the red-black smoother cell by cell, the coarse
    problem solved by the pseudo-inverse), up to the constant the periodic
    problem leaves free;
  - the exact discrete solution (FFT) is a fixed point;
  - the full V(2,2) cycle reduces the residual by a factor of at most 0.15
    per cycle on several shapes (textbook red-black Gauss-Seidel V-cycles on
    the 5-point Poisson problem reduce it by about 0.1);
  - planted mistakes (coarse spacing h, no 1/4 in the restriction,
    interpolation towards the wrong neighbour, piecewise-constant
    interpolation, a flipped correction) each fail a pin.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mg


# ----------------------------------------------------------------- closed forms
def mode(nx, ny, h, k, l, phase):
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    return np.cos(2 * np.pi * (k * x[None, :] + l * y[:, None]) + phase)


@pytest.mark.parametrize("nx,ny,k,l", [(16, 16, 1, 0), (16, 8, 3, 2), (32, 12, 5, -4),
                                       (8, 8, 4, 4), (64, 32, 7, 11)])
def test_restriction_of_a_mode(nx, ny, k, l):
    h = 1.0 / nx
    fx, fy = k / (nx * h), l / (ny * h)  # periodic on the grid
    v = mode(nx, ny, h, fx, fy, 0.3)
    got = mg.restrict(v)
    want = (np.cos(np.pi * fx * h) * np.cos(np.pi * fy * h)
            * mode(nx // 2, ny // 2, 2 * h, fx, fy, 0.3))
    assert np.max(np.abs(got - want)) <= 1e-14


def interp_factor(theta, s, H):
    """Bilinear interpolation of exp(i theta X) between centres H apart, read
    at X_I + s H / 4, divided by exp(i theta (X_I + s H / 4))."""
    return 0.75 * np.exp(-1j * s * theta * H / 4) + 0.25 * np.exp(3j * s * theta * H / 4)


@pytest.mark.parametrize("nxc,nyc,k,l", [(8, 8, 1, 0), (8, 4, 3, 1), (6, 10, 2, -3),
                                         (16, 16, 7, 5)])
def test_prolongation_of_a_mode(nxc, nyc, k, l):
    H = 1.0 / nxc
    tx, ty = 2 * np.pi * k / (nxc * H), 2 * np.pi * l / (nyc * H)  # periodic on the grid
    X = (np.arange(nxc) + 0.5) * H
    Y = (np.arange(nyc) + 0.5) * H
    V = np.real(np.exp(1j * (tx * X[None, :] + ty * Y[:, None] + 0.7)))
    got = mg.prolong(V)
    want = np.empty_like(got)
    for j in range(2 * nyc):
        for i in range(2 * nxc):
            sx = -1 if i % 2 == 0 else 1
            sy = -1 if j % 2 == 0 else 1
            xf, yf = (i + 0.5) * H / 2, (j + 0.5) * H / 2
            z = (np.exp(1j * (tx * xf + ty * yf + 0.7))
                 * interp_factor(tx, sx, H) * interp_factor(ty, sy, H))
            want[j, i] = z.real
    assert np.max(np.abs(got - want)) <= 1e-14


# ------------------------------------------------------------------ dense two-grid
def dense_laplacian(nx, ny, h):
    n = nx * ny
    A = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            for (di, dj) in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                A[c, ((j + dj) % ny) * nx + (i + di) % nx] += 1.0 / h**2
            A[c, c] -= 4.0 / h**2
    return A


def dense_restriction(nx, ny):
    """Coarse cell (J, I) is the union of fine cells (2J + b, 2I + a)."""
    R = np.zeros(((nx // 2) * (ny // 2), nx * ny))
    for J in range(ny // 2):
        for I in range(nx // 2):
            for b in (0, 1):
                for a in (0, 1):
                    R[J * (nx // 2) + I, (2 * J + b) * nx + 2 * I + a] = 0.25
    return R


def dense_prolongation(nx, ny):
    """Bilinear weights from periodic centre distances: a coarse centre
    within one coarse width H in x and in y gets (1 - |dx|/H)(1 - |dy|/H)."""
    nxc, nyc = nx // 2, ny // 2
    P = np.zeros((nx * ny, nxc * nyc))
    for j in range(ny):
        for i in range(nx):
            xf, yf = (i + 0.5) / 2, (j + 0.5) / 2      # in coarse widths
            for J in range(nyc):
                for I in range(nxc):
                    dx = (xf - (I + 0.5) + nxc / 2) % nxc - nxc / 2
                    dy = (yf - (J + 0.5) + nyc / 2) % nyc - nyc / 2
                    if abs(dx) < 1 and abs(dy) < 1:
                        P[j * nx + i, J * nxc + I] += (1 - abs(dx)) * (1 - abs(dy))
    return P


def dense_rb_sweep(phi, rho, A, nx, ny, h, omega):
    """Red cells ((x + y) even) then black, each phi_c += (omega h^2 / 4)
    ((A phi)_c - rho_c), in place."""
    phi = phi.copy()
    for colour in (0, 1):
        for j in range(ny):
            for i in range(nx):
                if (i + j) % 2 == colour:
                    c = j * nx + i
                    phi[c] += omega * h * h / 4 * (A[c] @ phi - rho[c])
    return phi


def dense_two_grid(phi, rho, nx, ny, h, nu1, nu2, omega):
    A = dense_laplacian(nx, ny, h)
    Ac = dense_laplacian(nx // 2, ny // 2, 2 * h)
    R, P = dense_restriction(nx, ny), dense_prolongation(nx, ny)
    x = phi.ravel().copy()
    f = rho.ravel()
    for _ in range(nu1):
        x = dense_rb_sweep(x, f, A, nx, ny, h, omega)
    ec = np.linalg.pinv(Ac) @ (R @ (f - A @ x))
    x = x + P @ ec
    for _ in range(nu2):
        x = dense_rb_sweep(x, f, A, nx, ny, h, omega)
    return x.reshape(ny, nx)


def two_level_oracle(phi, rho, h, nu1, nu2, omega):
    ny, nx = phi.shape
    shapes = mg.level_shapes(nx, ny, 2)
    return mg.vcycle(phi, rho, h, shapes, 0, nu1, nu2, omega, 6000)


def check_two_grid(vcycle_fn=two_level_oracle, cases=None):
    rng = np.random.default_rng(5)
    cases = cases or [(8, 8, 2, 2, 1.0), (8, 4, 1, 1, 1.0), (4, 8, 2, 1, 1.2), (12, 8, 1, 2, 0.9)]
    for (nx, ny, nu1, nu2, omega) in cases:
        h = 1.0 / nx
        rho = synth.random_field(rng, nx, ny)
        phi = synth.random_field(rng, nx, ny, zero_mean=False)
        got = vcycle_fn(phi, rho, h, nu1, nu2, omega)
        want = dense_two_grid(phi, rho, nx, ny, h, nu1, nu2, omega)
        d = (got - got.mean()) - (want - want.mean())
        assert np.max(np.abs(d)) <= 1e-9 * np.max(np.abs(want)), (nx, ny, nu1, nu2, omega)


def test_two_level_cycle_matches_dense_matrices():
    check_two_grid()


def test_dense_operators_are_what_they_claim():
    """Sanity of the dense builders themselves: P reproduces constants, R
    averages, and R P is the coarse-to-coarse map of bilinear interpolation
    followed by block means (weights 9/16, 3/16 x 2, 1/16 averaged over the
    four children of a coarse cell: 0.5625 on the cell itself)."""
    P = dense_prolongation(8, 6)
    R = dense_restriction(8, 6)
    assert np.allclose(P.sum(axis=1), 1.0) and np.allclose(R.sum(axis=1), 1.0)
    assert np.allclose(np.diag(R @ P), 0.5625)


# ------------------------------------------------------------------ fixed point
def fft_solution(rho, h):
    ny, nx = rho.shape
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    sym = (2 * np.cos(kx)[None, :] + 2 * np.cos(ky)[:, None] - 4) / h**2
    sym[0, 0] = 1.0
    F = np.fft.fft2(rho)
    F[0, 0] = 0.0
    return np.real(np.fft.ifft2(F / sym))


@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 32), (16, 40)])
def test_exact_solution_is_a_fixed_point(nx, ny):
    h = 1.0 / nx
    rho, _ = synth.modes_rho(nx, ny, 6, 5, 3, noise_sigma=0.1)
    phi = fft_solution(rho, h)
    out, R = mg.mg_solve(phi, rho, h, 2)
    assert np.max(np.abs(out - phi)) <= 1e-11 * np.max(np.abs(phi))
    sc = 8 * np.max(np.abs(phi)) / h**2 + np.max(np.abs(rho))
    assert np.all(R <= 1e-12 * sc)


# ------------------------------------------------------------------ convergence
def check_convergence(solve=mg.mg_solve, shapes=((64, 64), (128, 64), (96, 96), (32, 128)),
                      bound=0.15):
    rng = np.random.default_rng(9)
    for (nx, ny) in shapes:
        h = 1.0 / nx
        rho = synth.random_field(rng, nx, ny)
        _, R = solve(np.zeros_like(rho), rho, h, 6)
        rate = (R[-1] / R[0]) ** (1.0 / 6)
        assert rate <= bound, (nx, ny, rate)


def test_vcycle_convergence_factor():
    check_convergence()


def test_level_shapes():
    assert mg.level_shapes(64, 64) == [(64, 64), (32, 32), (16, 16), (8, 8), (4, 4), (2, 2)]
    assert mg.level_shapes(96, 40) == [(96, 40), (48, 20), (24, 10)]
    assert mg.level_shapes(6, 6) == [(6, 6)]
    assert mg.level_shapes(64, 64, 3) == [(64, 64), (32, 32), (16, 16)]
    assert mg.auto_coarse_sweeps(2, 2) == 1 and mg.auto_coarse_sweeps(10, 6) == 200


# ------------------------------------------------------------------ planted mistakes
def _vcycle_with(restrict=None, prolong=None, coarse_h=2.0, sign=1.0):
    restrict = restrict or mg.restrict
    prolong = prolong or mg.prolong

    def vc(phi, rho, h, shapes, level, nu1, nu2, omega, coarse_sweeps):
        phi = np.array(phi, dtype=np.float64)
        if level == len(shapes) - 1:
            return oracle.rbsor_n(phi, rho, h, omega, coarse_sweeps)[0]
        phi, _ = oracle.rbsor_n(phi, rho, h, omega, nu1)
        rc = restrict(rho - oracle.apply_stencil(phi, h))
        ec = vc(np.zeros_like(rc), rc, coarse_h * h, shapes, level + 1, nu1, nu2, omega,
                coarse_sweeps)
        phi = phi + sign * prolong(ec)
        return oracle.rbsor_n(phi, rho, h, omega, nu2)[0]

    def two_level(phi, rho, h, nu1, nu2, omega):
        ny, nx = phi.shape
        return vc(phi, rho, h, mg.level_shapes(nx, ny, 2), 0, nu1, nu2, omega, 6000)

    def solve(phi0, rho, h, ncycles):
        ny, nx = phi0.shape
        shapes = mg.level_shapes(nx, ny)
        cs = mg.auto_coarse_sweeps(*shapes[-1])
        phi, reps = np.array(phi0), [oracle.residual_norm(phi0, rho, h)[0]]
        for _ in range(ncycles):
            phi = vc(phi, rho, h, shapes, 0, 2, 2, 1.0, cs)
            reps.append(oracle.residual_norm(phi, rho, h)[0])
        return phi, np.array(reps)

    return two_level, solve


def _wrong_neighbour_prolong(e):
    """Interpolates towards I + 1 from fine column 2I and towards I - 1 from
    2I + 1 (likewise in y): the far neighbour instead of the near one."""
    ny, nx = e.shape
    out = np.empty((2 * ny, 2 * nx))
    for b in (0, 1):
        for a in (0, 1):
            sx, sy = (-1 if a == 0 else 1), (-1 if b == 0 else 1)
            x, y = np.roll(e, sx, axis=1), np.roll(e, sy, axis=0)
            out[b::2, a::2] = (0.5625 * e + 0.1875 * (x + y)) + 0.0625 * np.roll(x, sy, axis=0)
    return out


MUTANTS = {
    "coarse spacing h": dict(coarse_h=1.0),
    "restriction without 1/4": dict(restrict=lambda r: 4.0 * mg.restrict(r)),
    "interpolation towards the wrong neighbour": dict(prolong=_wrong_neighbour_prolong),
    "piecewise-constant interpolation": dict(
        prolong=lambda e: np.repeat(np.repeat(e, 2, axis=0), 2, axis=1)),
    "flipped correction": dict(sign=-1.0),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistakes_fail_a_pin(name):
    two_level, solve = _vcycle_with(**MUTANTS[name])
    failed = False
    try:
        check_two_grid(two_level, cases=[(8, 8, 2, 2, 1.0), (12, 8, 1, 2, 0.9)])
    except AssertionError:
        failed = True
    if not failed:
        try:
            check_convergence(solve, shapes=((64, 64),))
        except AssertionError:
            failed = True
    assert failed, name

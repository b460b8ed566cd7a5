"""Pins of the red-black SOR oracle (the relaxation named as Proto's multigrid
smoother, Sec. VI; standard definition: red cells (i + j even) updated in place,
then black cells, each with the Jacobi per-point update). Every pin is
mathematical:
  - a dense-matrix SOR in red-black ordering on small periodic grids;
  - the exact discrete solution (FFT solve) is a fixed point;
  - local Fourier analysis: on a periodic grid with even sides, red-black SOR
    maps each harmonic pair {theta, theta + (pi, pi)} into itself, with
    eigenvalues lambda of Young's relation (lambda + omega - 1)^2 =
    lambda omega^2 mu^2, mu = (cos theta_1 + cos theta_2) / 2 the Jacobi
    symbol; for Gauss-Seidel (omega = 1) the non-zero one is mu^2. From a
    single such mode with rho = 0 the residual ratio per sweep must tend to
    the dominant root (a Jacobi-style mistake gives mu, not mu^2)."""
import numpy as np
import pytest

import oracle


def periodic_laplacian(nx, ny, h):
    n = nx * ny
    A = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            for (di, dj) in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                A[c, ((j + dj) % ny) * nx + (i + di) % nx] += 1.0 / h**2
            A[c, c] -= 4.0 / h**2
    return A


@pytest.mark.parametrize("nx,ny", [(2, 2), (4, 4), (6, 4), (4, 6), (8, 8)])
@pytest.mark.parametrize("omega", [1.0, 1.3, 0.7])
def test_dense_matrix_red_black_sor(nx, ny, omega):
    rng = np.random.default_rng(nx * 10 + ny)
    h = 1.0 / nx
    phi = rng.standard_normal((ny, nx))
    rho = rng.standard_normal((ny, nx))
    rho -= rho.mean()
    A = periodic_laplacian(nx, ny, h)
    D = -4.0 / h**2
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    red = ((ii + jj) % 2 == 0).ravel()
    x, b = phi.ravel().copy(), rho.ravel()
    R = []
    for _ in range(5):
        R.append(np.max(np.abs(b - A @ x)))
        for colour in (red, ~red):  # cells of one colour only see the other colour
            x[colour] += omega / D * (b - A @ x)[colour]
    got, rep = oracle.rbsor_n(phi, rho, h, omega, 5, 1)
    scale = np.max(np.abs(x))
    assert np.max(np.abs(got.ravel() - x)) <= 1e-13 * scale
    assert np.allclose(rep, R, rtol=1e-12, atol=1e-12 * max(R))


def test_exact_solution_is_a_fixed_point():
    nx, ny = 32, 24
    h = 1.0 / nx
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((ny, nx))
    rho -= rho.mean()
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    mu = (2 * np.cos(ky)[:, None] + 2 * np.cos(kx)[None, :] - 4) / h**2
    mu[0, 0] = 1.0
    ph = np.fft.fft2(rho) / mu
    ph[0, 0] = 0.0
    phi = np.real(np.fft.ifft2(ph))
    got, rep = oracle.rbsor_n(phi, rho, h, 1.2, 1, 1)
    assert np.max(np.abs(got - phi)) <= 1e-12 * np.max(np.abs(phi))
    assert rep[0] <= 1e-9 * np.max(np.abs(rho))


def young_roots(omega, mu):
    # (lambda + omega - 1)^2 = lambda omega^2 mu^2, as a quadratic in lambda
    b = 2 * (omega - 1) - omega**2 * mu**2
    c = (omega - 1) ** 2
    disc = b * b - 4 * c
    assert disc >= 0
    return sorted([(-b + np.sqrt(disc)) / 2, (-b - np.sqrt(disc)) / 2], key=abs)


# (omega, k, l) with real Young roots (for complex roots both have modulus
# |omega - 1| and the max-norm ratio oscillates instead of converging)
@pytest.mark.parametrize("omega,k,l", [(1.0, 3, 5), (1.0, 1, 2), (1.0, 7, 1), (1.2, 1, 2),
                                       (1.2, 1, 1), (0.8, 3, 5), (0.8, 7, 1), (0.8, 1, 2)])
def test_local_fourier_rate(omega, k, l):
    nx = ny = 32
    h = 1.0 / nx
    t1, t2 = 2 * np.pi * k / nx, 2 * np.pi * l / ny
    mu = (np.cos(t1) + np.cos(t2)) / 2
    small, big = young_roots(omega, mu)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.cos(t1 * ii + 0.3) * np.cos(t2 * jj - 0.7)
    # only while the seeded pair dominates the round-off seeded into other modes
    ns = 12
    _, rep = oracle.rbsor_n(phi, np.zeros_like(phi), h, omega, ns, 1)
    ratios = rep[1:] / rep[:-1]
    if omega == 1.0:
        assert abs(small) < 1e-12 and abs(big - mu**2) < 1e-12
        # the zero eigenvalue dies in the first sweep: exact from then on
        assert np.max(np.abs(ratios[1:] - mu**2)) <= 1e-9
    else:
        # the smaller root decays relative to the larger one as (small/big)^s
        assert abs(ratios[-1] - abs(big)) <= 1e-9 + 4 * abs(small / big) ** (ns - 3)
    assert abs(abs(big) - abs(mu)) > 1e-3  # a Jacobi-style rate would fail


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        oracle.rbsor_n(np.zeros((4, 5)), np.zeros((4, 5)), 0.2, 1.0, 1)

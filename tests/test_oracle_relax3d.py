"""Pins of the 3D fused sweep oracle (7-point periodic Laplacian, Eq. "jacobi"
with D = 3: phi' = phi + (omega h^2 / 6)(L phi - rho)). Every pin is
mathematical:
  - a single Fourier mode is an eigenvector of L with eigenvalue
    -(4/h^2)(s_x + s_y + s_z), s = sin^2(pi k / n), so from rho = 0 it decays by
    the gain g = 1 - (2 omega / 3)(s_x + s_y + s_z) per sweep and each report
    is (4/h^2)(s_x + s_y + s_z) g^k max|v|;
  - dense-matrix Jacobi with L built cell by cell on small grids;
  - one plane (nz = 1) is the 2D sweep with omega' = 2 omega / 3 (its two z
    neighbours are the cell itself);
  - the mean is preserved for mean-zero rho;
  - planted mistakes (centre tap -4, weight omega / 4, a transposed wrap)
    each fail a pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth


def mode3(nx, ny, nz, k, l, m, phase=0.4):
    x = np.arange(nx)[None, None, :] / nx
    y = np.arange(ny)[None, :, None] / ny
    z = np.arange(nz)[:, None, None] / nz
    return np.cos(2 * np.pi * (k * x + l * y + m * z) + phase)


@pytest.mark.parametrize("dims,kl,omega", [((16, 8, 12), (3, 1, 2), 1.0),
                                           ((10, 10, 10), (1, 0, 0), 0.5),
                                           ((8, 6, 4), (2, 3, 1), 6.0 / 7.0),
                                           ((12, 4, 2), (5, 2, 1), 0.8)])
def test_mode_trajectory_closed_form(dims, kl, omega):
    nx, ny, nz = dims
    k, l, m = kl
    h = 1.0 / nx
    v = mode3(nx, ny, nz, k, l, m)
    S = np.sin(np.pi * k / nx) ** 2 + np.sin(np.pi * l / ny) ** 2 + np.sin(np.pi * m / nz) ** 2
    g = 1 - (2 * omega / 3) * S
    n = 7
    out, R = oracle.relax3_n(v, np.zeros_like(v), h, omega, n, 1)
    assert np.max(np.abs(out - g ** n * v)) <= 1e-12
    want = (4 / h**2) * S * np.abs(g) ** np.arange(n) * np.max(np.abs(v))
    assert np.max(np.abs(R - want)) <= 1e-12 * (8 / h**2)


def dense_laplacian3(nx, ny, nz, h):
    n = nx * ny * nz
    A = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = (k * ny + j) * nx + i
                for (di, dj, dk) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                                     (0, 0, -1), (0, 0, 1)):
                    A[c, (((k + dk) % nz) * ny + (j + dj) % ny) * nx + (i + di) % nx] += 1 / h**2
                A[c, c] -= 6 / h**2
    return A


@pytest.mark.parametrize("dims", [(3, 4, 2), (2, 2, 3), (5, 3, 4), (1, 3, 2), (4, 1, 1)])
@pytest.mark.parametrize("omega", [0.5, 1.0])
def test_dense_matrix_jacobi(dims, omega):
    nx, ny, nz = dims
    h = 1.0 / max(nx, 2)
    rng = np.random.default_rng(sum(dims))
    phi = rng.standard_normal((nz, ny, nx))
    rho = rng.standard_normal((nz, ny, nx))
    A = dense_laplacian3(nx, ny, nz, h)
    x = phi.ravel().copy()
    reps = []
    for _ in range(5):
        r = rho.ravel() - A @ x
        reps.append(np.max(np.abs(r)))
        x = x - omega * h * h / 6 * r
    out, R = oracle.relax3_n(phi, rho, h, omega, 5, 1)
    assert np.max(np.abs(out.ravel() - x)) <= 1e-12 * max(1.0, np.max(np.abs(x)))
    assert np.max(np.abs(R - reps)) <= 1e-12 * max(reps)


@pytest.mark.parametrize("nx,ny,omega", [(16, 12, 1.0), (9, 7, 0.6)])
def test_single_plane_is_the_2d_sweep(nx, ny, omega):
    rng = np.random.default_rng(3)
    rho = synth.random_field(rng, nx, ny)
    phi = synth.random_field(rng, nx, ny, zero_mean=False)
    h = 1.0 / nx
    out3, R3 = oracle.relax3_n(phi[None], rho[None], h, omega, 6, 2)
    out2, R2 = oracle.relax_n(phi, rho, h, 2 * omega / 3, 6, 2)
    assert np.max(np.abs(out3[0] - out2)) <= 1e-13 * np.max(np.abs(out2))
    assert np.max(np.abs(R3 - R2)) <= 1e-13 * 8 * np.max(np.abs(phi)) / h**2


def test_mean_preserved():
    rng = np.random.default_rng(8)
    rho = rng.standard_normal((6, 8, 10))
    rho -= rho.mean()
    phi = rng.standard_normal((6, 8, 10)) + 3.0
    out, _ = oracle.relax3_n(phi, rho, 0.1, 0.9, 11)
    assert abs(out.mean() - phi.mean()) <= 1e-13


MUTANTS = {
    "centre_tap": ("+ (pB + pT)) - 6.0 * pC;", "+ (pB + pT)) - 4.0 * pC;"),
    "weight_quarter": ("double w = omega / 6.0, lam = omega * h * h / 6.0;",
                       "double w = omega / 4.0, lam = omega * h * h / 6.0;"),
    "transposed_wrap": ("kp = wrapi(k + 1, nz);", "kp = wrapi(k + 1, ny);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(c), "-lm"])
    saved = oracle._load()
    oracle._lib = oracle.bind(ctypes.CDLL(str(so)))
    caught = 0
    try:
        for f in (lambda: test_mode_trajectory_closed_form((16, 8, 12), (3, 1, 2), 1.0),
                  lambda: test_dense_matrix_jacobi((3, 4, 2), 1.0),
                  lambda: test_single_plane_is_the_2d_sweep(16, 12, 1.0)):
            try:
                f()
            except AssertionError:
                caught += 1
    finally:
        oracle._lib = saved
    assert caught >= 1, name

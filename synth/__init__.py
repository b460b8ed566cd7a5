"""Seeded synthetic inputs for the periodic 2D Poisson relaxation workloads.

This module builds right-hand sides rho (and initial guesses) only. It holds
none of the relaxation arithmetic, so both the FP64 CPU oracle and the CUDA
path can take their inputs from here without sharing any of the method.

Grid convention (cell-centred, row-major, x fastest): cell (i, j) with
i in [0, nx), j in [0, ny) sits at x_i = (i + 1/2) h, y_j = (j + 1/2) h.
A Fourier mode with integer wavenumbers (k, l) is the product
f(2 pi k (i + 1/2) / nx) * g(2 pi l (j + 1/2) / ny) with f, g in {sin, cos}.
Arrays are returned with shape (ny, nx).

The default seed of workload c is 20230717 + c, with c the workload index:
0 = 64x64 8-mode field, 1 = 16384x16384 64-mode field plus noise,
2 = 8192x8192 refinement field, 3 = 1024 uneven batched instances,
4 = 256x256 learned-guess fields, 5 = 512^3 3D field.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 20230717


def workload_seed(index: int) -> int:
    return BASE_SEED + int(index)


@dataclass(frozen=True)
class Mode:
    """One separable Fourier mode: amp * fx(2 pi k (i+1/2)/nx) * fy(2 pi l (j+1/2)/ny)."""
    amp: float
    k: int
    l: int
    fx: str  # "sin" or "cos"
    fy: str


def draw_modes(rng: np.random.Generator, count: int, kmax: int, kmin: int = 1,
               lmax: int | None = None) -> list[Mode]:
    """Draw `count` modes: k, l uniform in [kmin, kmax], amplitudes N(0, 1),
    sin/cos chosen by a fair coin per axis."""
    lmax = kmax if lmax is None else lmax
    amps = rng.standard_normal(count)
    ks = rng.integers(kmin, kmax + 1, size=count)
    ls = rng.integers(kmin, lmax + 1, size=count)
    fxs = rng.integers(0, 2, size=count)
    fys = rng.integers(0, 2, size=count)
    names = ("sin", "cos")
    return [Mode(float(a), int(k), int(l), names[int(fx)], names[int(fy)])
            for a, k, l, fx, fy in zip(amps, ks, ls, fxs, fys)]


def mode_vectors(mode: Mode, nx: int, ny: int) -> tuple[np.ndarray, np.ndarray]:
    """The 1D factors (along x, along y) of one mode, in float64."""
    tx = 2.0 * np.pi * mode.k * (np.arange(nx, dtype=np.float64) + 0.5) / nx
    ty = 2.0 * np.pi * mode.l * (np.arange(ny, dtype=np.float64) + 0.5) / ny
    vx = np.sin(tx) if mode.fx == "sin" else np.cos(tx)
    vy = np.sin(ty) if mode.fy == "sin" else np.cos(ty)
    return vx, vy


def modes_field(modes: list[Mode], nx: int, ny: int) -> np.ndarray:
    """Sum of separable modes as the rank-<=len(modes) product U diag(A) V^T."""
    if not modes:
        return np.zeros((ny, nx), dtype=np.float64)
    vy = np.empty((ny, len(modes)), dtype=np.float64)
    vx = np.empty((len(modes), nx), dtype=np.float64)
    for m, mode in enumerate(modes):
        fx, fy = mode_vectors(mode, nx, ny)
        vx[m] = fx
        vy[:, m] = fy * mode.amp
    return vy @ vx


def remove_mean(a: np.ndarray) -> np.ndarray:
    """Subtract the float64 mean (numpy's pairwise summation) in place."""
    a -= a.sum(dtype=np.float64) / a.size
    return a


def gaussian_blobs(rng: np.random.Generator, nx: int, ny: int, count: int,
                   sig_lo: float = 2.0, sig_hi: float = 20.0) -> np.ndarray:
    """Sum of periodic Gaussian blobs (in cells): amplitude N(0,1), centre uniform,
    sigma uniform in [sig_lo, sig_hi] cells, summed over the 3x3 nearest images."""
    out = np.zeros((ny, nx), dtype=np.float64)
    ix = np.arange(nx, dtype=np.float64)
    iy = np.arange(ny, dtype=np.float64)
    for _ in range(count):
        amp = rng.standard_normal()
        cx = rng.uniform(0.0, nx)
        cy = rng.uniform(0.0, ny)
        sig = rng.uniform(sig_lo, sig_hi)
        gx = np.zeros(nx)
        gy = np.zeros(ny)
        for img in (-1, 0, 1):
            gx += np.exp(-0.5 * ((ix - cx + img * nx) / sig) ** 2)
            gy += np.exp(-0.5 * ((iy - cy + img * ny) / sig) ** 2)
        out += amp * np.outer(gy, gx)
    return out


def modes_rho(nx: int, ny: int, nmodes: int, kmax: int, seed: int,
              noise_sigma: float = 0.0, lmax: int | None = None
              ) -> tuple[np.ndarray, list[Mode]]:
    """rho = sum of `nmodes` seeded modes (+ N(0, noise_sigma^2) white noise),
    mean-zeroed. Returns (rho, modes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    modes = draw_modes(rng, nmodes, kmax, lmax=lmax)
    rho = modes_field(modes, nx, ny)
    if noise_sigma > 0.0:
        rho += noise_sigma * rng.standard_normal((ny, nx))
    return remove_mean(rho), modes


def small_field_rho(seed: int) -> tuple[np.ndarray, list[Mode]]:
    """64x64 field: 8 modes with k, l in 1..16."""
    return modes_rho(64, 64, 8, 16, seed)


def large_field_rho(n: int = 16384, kmax: int = 512, seed: int | None = None,
                    noise_sigma: float = 0.1) -> np.ndarray:
    """n x n field: 64 modes with k, l in 1..kmax plus sigma=0.1 white noise."""
    seed = workload_seed(1) if seed is None else seed
    rho, _ = modes_rho(n, n, 64, kmax, seed, noise_sigma=noise_sigma)
    return rho


def learned_guess_rho(rng: np.random.Generator, n: int = 256) -> np.ndarray:
    """n x n field with 1..32 sine/cosine modes (k, l in 1..32) plus 0..4
    periodic Gaussian blobs (sigma 2..20 cells), mean-zeroed."""
    nm = int(rng.integers(1, 33))
    modes = draw_modes(rng, nm, 32)
    rho = modes_field(modes, n, n)
    nb = int(rng.integers(0, 5))
    if nb:
        rho += gaussian_blobs(rng, n, n, nb)
    return remove_mean(rho)


def batch_sizes(count: int = 1024, seed: int | None = None
                ) -> tuple[np.ndarray, np.ndarray]:
    """Uneven batch: N = 16 j, j = 2..64 (32..1024), P(N) proportional to 1/N
    (log-uniform), dtype per instance a fair coin (0 = FP64, 1 = FP32)."""
    seed = workload_seed(3) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = 16 * np.arange(2, 65)
    p = 1.0 / sizes
    p /= p.sum()
    ns = rng.choice(sizes, size=count, p=p)
    dts = rng.integers(0, 2, size=count)
    return ns.astype(np.int64), dts.astype(np.int32)


def batch_rho(n: int, instance: int, seed: int | None = None) -> np.ndarray:
    """rho of one batched instance: 8 modes with k, l in 1..min(16, n/4)."""
    seed = workload_seed(3) if seed is None else seed
    rho, _ = modes_rho(n, n, 8, max(1, min(16, n // 4)), seed * 7919 + instance)
    return rho


def random_field(rng: np.random.Generator, nx: int, ny: int,
                 zero_mean: bool = True) -> np.ndarray:
    """Uniform(-1, 1) white field (tests only)."""
    a = rng.uniform(-1.0, 1.0, size=(ny, nx))
    return remove_mean(a) if zero_mean else a


def field3_rho(n: int = 512, nmodes: int = 8, kmax: int = 64, noise_sigma: float = 0.1,
               seed: int | None = None) -> np.ndarray:
    """The 3D workload's right-hand side on an n^3 periodic grid (shape
    (n, n, n), z slowest): nmodes seeded plane waves cos(2 pi (k x + l y + m z)
    + phase) with integer wavenumbers in [-kmax, kmax] (not all zero) and
    N(0, 1) amplitudes, plus N(0, noise_sigma^2) white noise, mean-zeroed.
    Workload index 5."""
    rng = np.random.Generator(np.random.PCG64(workload_seed(5) if seed is None else seed))
    t = 2 * np.pi * (np.arange(n) + 0.5) / n
    rho = np.zeros((n, n, n), dtype=np.float64)
    for _ in range(nmodes):
        k, l, m = (int(v) for v in rng.integers(-kmax, kmax + 1, 3))
        if k == 0 and l == 0 and m == 0:
            k = 1
        a, ph = float(rng.normal()), float(rng.uniform(0, 2 * np.pi))
        ex, ey, ez = np.exp(1j * k * t), np.exp(1j * l * t), np.exp(1j * (m * t + ph))
        rho += a * np.real(ez[:, None, None] * (ey[:, None] * ex[None, :])[None, :, :])
    if noise_sigma > 0:
        rho += noise_sigma * rng.standard_normal((n, n, n))
    return rho - rho.mean()


def random_field3(rng: np.random.Generator, nx: int, ny: int, nz: int,
                  zero_mean: bool = True) -> np.ndarray:
    """Uniform(-1, 1) white 3D field of shape (nz, ny, nx) (tests only)."""
    a = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    return a - a.mean() if zero_mean else a


def euler_kh_primitives(nx: int, ny: int, seed: int | None = None, delta: float = 0.01,
                        nmodes: int = 8, kmax: int = 8) -> np.ndarray:
    """Primitive planes (rho, u, v, p), shape (4, ny, nx), of a periodic double
    shear layer on the unit square (cell centres): rho = 1 + b(y) and
    u = b(y) - 1/2 with b(y) = (tanh((y - 1/4)/delta) - tanh((y - 3/4)/delta))/2,
    p = 2.5, and v a seeded sum of `nmodes` sine modes in x (k in 1..kmax,
    N(0, 1) amplitudes scaled to 0.01) localised at the two layers by
    Gaussians of width 0.05."""
    seed = workload_seed(6) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(nx, dtype=np.float64) + 0.5) / nx
    y = (np.arange(ny, dtype=np.float64) + 0.5) / ny
    b = 0.5 * (np.tanh((y - 0.25) / delta) - np.tanh((y - 0.75) / delta))
    amps = 0.01 * rng.standard_normal(nmodes)
    ks = rng.integers(1, kmax + 1, size=nmodes)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)
    vx = np.zeros(nx)
    for a, k, ph in zip(amps, ks, phases):
        vx += a * np.sin(2.0 * np.pi * k * x + ph)
    loc = np.exp(-((y - 0.25) / 0.05) ** 2) + np.exp(-((y - 0.75) / 0.05) ** 2)
    W = np.empty((4, ny, nx))
    W[0] = (1.0 + b)[:, None]
    W[1] = (b - 0.5)[:, None]
    W[2] = loc[:, None] * vx[None, :]
    W[3] = 2.5
    return W

"""Oracle of the geometric multigrid V-cycle for the periodic 2D Poisson
problem, with red-black SOR as the smoother.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check, the benchmark's CPU legs).

The paper names multigrid with red-black SOR smoothing as what Proto builds on
its operators (Sec. VI) and describes no cycle, so this follows the textbook
cell-centred V-cycle. On a grid of nx x ny cells of width h (Delta phi = rho,
5-point L_h, periodic), one cycle V(phi, rho, level) is:
  1. nu1 red-black SOR sweeps on L_h phi = rho (oracle.rbsor_n);
  2. r = rho - L_h phi (oracle.apply_stencil);
  3. r_c = R r: the mean of each 2 x 2 block of cells (the coarse cell is
     their union, width 2h);
  4. e_c = V(0, r_c, level + 1) on the coarse grid, L_2h e_c = r_c;
  5. phi <- phi + P e_c: bilinear interpolation between coarse cell centres
     (weights 9/16, 3/16, 3/16, 1/16 from the nearest four, periodic);
  6. nu2 red-black SOR sweeps.
On the coarsest level the cycle is coarse_sweeps red-black SOR sweeps.
Levels halve both extents while both halves stay even (down to 2 x 2).
Every arithmetic step is FP64: the C oracle for the sweeps and the stencil,
numpy for the transfers in the fixed orders stated below.
"""
from __future__ import annotations

import numpy as np

from . import apply_stencil, rbsor_n, residual_norm


def level_shapes(nx: int, ny: int, max_levels: int = 0) -> list[tuple[int, int]]:
    """(nx, ny) of every level, finest first. Every level keeps both extents
    even (the red-black colouring), so coarsening stops when an extent is not
    a multiple of 4, or at max_levels levels (0: no cap)."""
    shapes = [(nx, ny)]
    while nx % 4 == 0 and ny % 4 == 0:
        if max_levels and len(shapes) >= max_levels:
            break
        nx, ny = nx // 2, ny // 2
        shapes.append((nx, ny))
    return shapes


def auto_coarse_sweeps(nx: int, ny: int) -> int:
    """Sweeps on the coarsest grid when the caller gives 0: one red-black
    Gauss-Seidel sweep solves a 2 x 2 grid exactly; otherwise 2 n^2 sweeps,
    n = max(nx, ny), bring its slowest mode (gain about 1 - 2 pi^2 / n^2 per
    sweep) down by about 1e-12."""
    n = max(nx, ny)
    return 1 if n <= 2 else 2 * n * n


def restrict(r: np.ndarray) -> np.ndarray:
    """Mean of each 2 x 2 block: ((r[2J,2I] + r[2J,2I+1]) + (r[2J+1,2I] +
    r[2J+1,2I+1])) * 0.25."""
    a, b = r[0::2, 0::2], r[0::2, 1::2]
    c, d = r[1::2, 0::2], r[1::2, 1::2]
    return ((a + b) + (c + d)) * 0.25


def prolong(e: np.ndarray) -> np.ndarray:
    """Bilinear interpolation from coarse cell centres to fine cell centres.
    Fine cell (2J + b, 2I + a) lies a quarter of a coarse cell from centre
    (J, I), towards I - 1 (a = 0) or I + 1 (a = 1) in x and likewise in y, so
    its value is 9/16 e(J, I) + 3/16 (e(J, I') + e(J', I)) + 1/16 e(J', I'),
    evaluated as ((0.5625 c + 0.1875 (x + y)) + 0.0625 d)."""
    ny, nx = e.shape
    out = np.empty((2 * ny, 2 * nx), dtype=np.float64)
    for b in (0, 1):
        sy = 1 if b == 0 else -1           # np.roll by +1 brings row J - 1 to J
        for a in (0, 1):
            sx = 1 if a == 0 else -1
            c = e
            x = np.roll(e, sx, axis=1)     # e(J, I')
            y = np.roll(e, sy, axis=0)     # e(J', I)
            d = np.roll(x, sy, axis=0)     # e(J', I')
            out[b::2, a::2] = (0.5625 * c + 0.1875 * (x + y)) + 0.0625 * d
    return out


def vcycle(phi, rho, h: float, shapes, level: int, nu1: int, nu2: int, omega: float,
           coarse_sweeps: int) -> np.ndarray:
    """One V-cycle on level `level` (shapes[level] is phi's shape); returns
    the new phi."""
    phi = np.array(phi, dtype=np.float64)
    if level == len(shapes) - 1:
        out, _ = rbsor_n(phi, rho, h, omega, coarse_sweeps)
        return out
    phi, _ = rbsor_n(phi, rho, h, omega, nu1)
    r = rho - apply_stencil(phi, h)
    rc = restrict(r)
    ec = vcycle(np.zeros_like(rc), rc, 2.0 * h, shapes, level + 1, nu1, nu2, omega,
                coarse_sweeps)
    phi = phi + prolong(ec)
    phi, _ = rbsor_n(phi, rho, h, omega, nu2)
    return phi


def mg_solve(phi0, rho, h: float, ncycles: int, nu1: int = 2, nu2: int = 2,
             omega: float = 1.0, coarse_sweeps: int = 0, max_levels: int = 0
             ) -> tuple[np.ndarray, np.ndarray]:
    """ncycles V-cycles from phi0. Returns (phi, reports) with reports[k] =
    ||rho - L phi_k||_inf for k = 0 .. ncycles (phi_k after k cycles).
    nx and ny must be even (the red-black colouring)."""
    phi = np.array(phi0, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = phi.shape
    shapes = level_shapes(nx, ny, max_levels)
    if coarse_sweeps <= 0:
        coarse_sweeps = auto_coarse_sweeps(*shapes[-1])
    reps = [residual_norm(phi, rho, h)[0]]
    for _ in range(ncycles):
        phi = vcycle(phi, rho, h, shapes, 0, nu1, nu2, omega, coarse_sweeps)
        reps.append(residual_norm(phi, rho, h)[0])
    return phi, np.array(reps)

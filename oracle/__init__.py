"""FP64 CPU oracle for the fused periodic 2D Poisson relaxation (ProtoX, Sec. IV).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg. The product library never imports it, and it
imports nothing from the product package. The arithmetic lives in oracle.c
(plain C, FP64, -ffp-contract=off); this module marshals numpy arrays.

Functions and the passages they follow:
  sweep            one fused sweep: Laplace, Jacobi (Eq. "jacobi" with weight
                   omega) and the input-state max-norm (OL rules, Sec. IV)
  relax_n          repeated fused sweeps with residual reports
  relax_unfused    the three-pass program of Fig. "Proto"
  relax_ghosted    fused sweeps on ghosted (m = n + 2) storage
  relax_omp        OpenMP fused sweeps, used only to time the CPU baseline
  apply_stencil    L phi = s / h^2
  residual_norm    ||rho - L phi||_inf and ||rho||_inf
  sweep3, relax3_n the fused sweep in 3D (7-point Laplacian, Eq. "jacobi"
                   with D = 3: weight omega h^2 / 6)
Refinement, CNN and multigrid pieces live in oracle/refine.py, oracle/cnn.py
and oracle/mg.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    if True:
        lib.oracle_fill_ghosts.argtypes = [i, i, i64, _dp]
        lib.oracle_apply_stencil.argtypes = [i, i, i64, d, _dp, _dp]
        lib.oracle_residual_norm.argtypes = [i, i, i64, d, _dp, _dp, _dp, _dp]
        lib.oracle_sweep.argtypes = [i, i, i64, d, d, _dp, _dp, _dp]
        lib.oracle_sweep.restype = d
        lib.oracle_relax_n.argtypes = [i, i, d, d, _dp, _dp, i, i, _dp, _dp]
        lib.oracle_rbsor_n.argtypes = [i, i, d, d, _dp, _dp, i, i, _dp, _dp]
        lib.oracle_rbsor_n.restype = i
        lib.oracle_relax_n.restype = i
        lib.oracle_relax_unfused.argtypes = [i, i, d, d, _dp, _dp, i, _dp]
        lib.oracle_relax_unfused.restype = i
        lib.oracle_relax_ghosted.argtypes = [i, i, d, d, _dp, _dp, _dp, i, _dp]
        lib.oracle_relax_ghosted.restype = i
        lib.oracle_relax_n_omp.argtypes = [i, i, d, d, _dp, _dp, _dp, i, i, _dp]
        lib.oracle_relax_n_omp.restype = i
        lib.oracle_sweep3.argtypes = [i, i, i, d, d, _dp, _dp, _dp]
        lib.oracle_sweep3.restype = d
        lib.oracle_relax3_n.argtypes = [i, i, i, d, d, _dp, _dp, i, i, _dp, _dp]
        lib.oracle_relax3_n.restype = i
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _shape(a: np.ndarray) -> tuple[int, int]:
    if a.ndim != 2:
        raise ValueError("expected a 2D (ny, nx) array")
    return int(a.shape[1]), int(a.shape[0])


def apply_stencil(phi, h: float) -> np.ndarray:
    """L phi with periodic wrap, scaled by 1/h^2."""
    phi = _f64(phi)
    nx, ny = _shape(phi)
    out = np.empty_like(phi)
    _load().oracle_apply_stencil(nx, ny, nx, h, _ptr(phi), _ptr(out))
    return out


def residual_norm(phi, rho, h: float) -> tuple[float, float]:
    """(||rho - L phi||_inf, ||rho||_inf)."""
    phi, rho = _f64(phi), _f64(rho)
    nx, ny = _shape(phi)
    r, p = ctypes.c_double(), ctypes.c_double()
    _load().oracle_residual_norm(nx, ny, nx, h, _ptr(phi), _ptr(rho),
                                 ctypes.byref(r), ctypes.byref(p))
    return r.value, p.value


def sweep(phi, rho, h: float, omega: float) -> tuple[np.ndarray, float]:
    """One fused sweep: (phi', R) with R the residual max-norm of the input phi."""
    phi, rho = _f64(phi), _f64(rho)
    nx, ny = _shape(phi)
    out = np.empty_like(phi)
    R = _load().oracle_sweep(nx, ny, nx, h, omega, _ptr(phi), _ptr(rho), _ptr(out))
    return out, R


def report_count(nsweeps: int, every: int) -> int:
    """Number of residual reports of a relax_n call: states 0, every, 2*every, ... < nsweeps."""
    if every <= 0 or nsweeps <= 0:
        return 0
    return (nsweeps + every - 1) // every


def relax_n(phi0, rho, h: float, omega: float, nsweeps: int, every: int = 0
            ) -> tuple[np.ndarray, np.ndarray]:
    """nsweeps fused sweeps from phi0; returns (phi^n, reports) where
    reports[k] = ||rho - L phi^(k*every)||_inf."""
    phi0, rho = _f64(phi0), _f64(rho)
    nx, ny = _shape(phi0)
    out = np.empty_like(phi0)
    rep = np.zeros(max(1, report_count(nsweeps, every)), dtype=np.float64)
    rc = _load().oracle_relax_n(nx, ny, h, omega, _ptr(phi0), _ptr(rho), nsweeps,
                                every, _ptr(out), _ptr(rep))
    if rc != 0:
        raise MemoryError("oracle_relax_n: allocation failed")
    return out, rep[:report_count(nsweeps, every)]


def rbsor_n(phi0, rho, h: float, omega: float, nsweeps: int, every: int = 0
            ) -> tuple[np.ndarray, np.ndarray]:
    """nsweeps red-black SOR sweeps from phi0 (red = (i + j) even first, then
    black, each in place with the Jacobi per-point update); returns (phi^n,
    reports) with reports[k] = ||rho - L phi^(k*every)||_inf of the input
    state of that sweep. nx and ny must be even."""
    phi0, rho = _f64(phi0), _f64(rho)
    nx, ny = _shape(phi0)
    if nx % 2 or ny % 2:
        raise ValueError("red-black SOR needs even nx and ny")
    out = np.empty_like(phi0)
    rep = np.zeros(max(1, report_count(nsweeps, every)), dtype=np.float64)
    rc = _load().oracle_rbsor_n(nx, ny, h, omega, _ptr(phi0), _ptr(rho), nsweeps, every,
                                _ptr(out), _ptr(rep))
    if rc != 0:
        raise MemoryError("oracle_rbsor_n: allocation failed")
    return out, rep[:report_count(nsweeps, every)]


def _shape3(a: np.ndarray) -> tuple[int, int, int]:
    if a.ndim != 3:
        raise ValueError("3D fields are (nz, ny, nx) arrays")
    nz, ny, nx = a.shape
    return nx, ny, nz


def sweep3(phi, rho, h: float, omega: float) -> tuple[np.ndarray, float]:
    """One fused 3D sweep (7-point Laplacian, Jacobi weight omega h^2 / 6):
    (phi', R) with R the residual max-norm of the input phi."""
    phi, rho = _f64(phi), _f64(rho)
    nx, ny, nz = _shape3(phi)
    out = np.empty_like(phi)
    R = _load().oracle_sweep3(nx, ny, nz, h, omega, _ptr(phi), _ptr(rho), _ptr(out))
    return out, R


def relax3_n(phi0, rho, h: float, omega: float, nsweeps: int, every: int = 0
             ) -> tuple[np.ndarray, np.ndarray]:
    """nsweeps fused 3D sweeps from phi0 (nz, ny, nx); returns (phi^n, reports)
    with reports[k] = ||rho - L phi^(k*every)||_inf."""
    phi0, rho = _f64(phi0), _f64(rho)
    nx, ny, nz = _shape3(phi0)
    out = np.empty_like(phi0)
    rep = np.zeros(max(1, report_count(nsweeps, every)), dtype=np.float64)
    rc = _load().oracle_relax3_n(nx, ny, nz, h, omega, _ptr(phi0), _ptr(rho), nsweeps, every,
                                 _ptr(out), _ptr(rep))
    if rc != 0:
        raise MemoryError("oracle_relax3_n: allocation failed")
    return out, rep[:report_count(nsweeps, every)]


def relax_unfused(phi0, rho, h: float, omega: float, iters: int
                  ) -> tuple[np.ndarray, np.ndarray]:
    """Three-pass program (temp = Laplacian, in-place Jacobi, residual pass) on
    ghosted storage. Returns (phi after iters, residual after each iteration)."""
    phi0, rho = _f64(phi0), _f64(rho)
    nx, ny = _shape(phi0)
    g = np.zeros((ny + 2, nx + 2), dtype=np.float64)
    g[1:-1, 1:-1] = phi0
    res = np.zeros(max(1, iters), dtype=np.float64)
    rc = _load().oracle_relax_unfused(nx, ny, h, omega, _ptr(g), _ptr(rho), iters, _ptr(res))
    if rc != 0:
        raise MemoryError("oracle_relax_unfused: allocation failed")
    return np.ascontiguousarray(g[1:-1, 1:-1]), res[:iters]


def relax_ghosted(X, rho, h: float, omega: float, nsweeps: int
                  ) -> tuple[np.ndarray, np.ndarray]:
    """Fused sweeps on a ghosted (ny+2, nx+2) array X (ghost values ignored on
    input). Returns (final ghosted array, per-sweep input residuals)."""
    X = _f64(X).copy()
    rho = _f64(rho)
    ny, nx = X.shape[0] - 2, X.shape[1] - 2
    Y = np.zeros_like(X)
    res = np.zeros(max(1, nsweeps), dtype=np.float64)
    which = _load().oracle_relax_ghosted(nx, ny, h, omega, _ptr(X), _ptr(Y), _ptr(rho),
                                         nsweeps, _ptr(res))
    return (X if which == 0 else Y), res[:nsweeps]


def fill_ghosts(g) -> np.ndarray:
    g = _f64(g).copy()
    ny, nx = g.shape[0] - 2, g.shape[1] - 2
    _load().oracle_fill_ghosts(nx, ny, nx + 2, _ptr(g))
    return g


def relax_omp(phi0, rho, h: float, omega: float, nsweeps: int, nthreads: int
              ) -> tuple[np.ndarray, float, int]:
    """OpenMP fused sweeps (timing baseline). Returns (phi, last R, threads used)."""
    a = _f64(phi0).copy()
    rho = _f64(rho)
    nx, ny = _shape(a)
    b = np.empty_like(a)
    R = ctypes.c_double()
    used = _load().oracle_relax_n_omp(nx, ny, h, omega, _ptr(a), _ptr(b), _ptr(rho),
                                      nsweeps, nthreads, ctypes.byref(R))
    return (a if nsweeps % 2 == 0 else b), R.value, used

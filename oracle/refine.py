"""Oracle of the mixed-precision solve: weighted-Jacobi sweeps (Sec. IV,
Eq. "jacobi") run inside an iterative-refinement loop.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check, the benchmark's CPU legs).

The paper itself only sweeps in one precision. The outer loop here is the
standard iterative-refinement scheme applied to those sweeps:
  1. r = rho - L phi in FP64, R = ||r||_inf; stop when R <= rtol ||rho||_inf;
  2. scale r by s = 2^-ilogb(R) (exact) and round it to the inner precision;
  3. solve L e = s r approximately by `inner` Jacobi sweeps from e = 0, each
     sweep's result rounded to the inner precision (FP32 storage);
  4. phi <- phi + e / s in FP64.
Every arithmetic step is the FP64 oracle (oracle.sweep, oracle.apply_stencil,
oracle.residual_norm) plus explicit float32 rounding of stored values.
With FP64 inner storage the loop is algebraically plain Jacobi (phi + e_n
obeys the same recurrence as n sweeps from phi), which the tests use as a pin.
"""
from __future__ import annotations

import math

import numpy as np

from . import apply_stencil, residual_norm, sweep


def power_scale(R: float) -> float:
    """2^-ilogb(R): the power of two that brings R into [1, 2)."""
    m, e = math.frexp(R)  # R = m 2^e, m in [0.5, 1)
    return math.ldexp(1.0, -(e - 1))


def refine_solve(rho, h: float, omega: float, rtol: float, inner: int, max_cycles: int,
                 fp32: bool = True, phi0=None):
    """Returns (phi, history) where history[c] = ||rho - L phi_c||_inf at the
    start of cycle c (the last entry is the final state's residual)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.zeros_like(rho) if phi0 is None else np.array(phi0, dtype=np.float64)
    _, P = residual_norm(phi, rho, h)
    hist = []
    for cyc in range(max_cycles + 1):
        r = rho - apply_stencil(phi, h)
        R = float(np.max(np.abs(r)))
        hist.append(R)
        if R <= rtol * P or cyc == max_cycles or R == 0.0:
            break
        s = power_scale(R)
        rs = r * s
        if fp32:
            rs = rs.astype(np.float32).astype(np.float64)
        e = np.zeros_like(rho)
        for _ in range(inner):
            e, _ = sweep(e, rs, h, omega)
            if fp32:
                e = e.astype(np.float32).astype(np.float64)
        phi = phi + e / s
    return phi, hist

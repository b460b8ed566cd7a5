"""Pins of the refinement oracle (oracle/refine.py)."""
import math

import numpy as np

import oracle
import synth
from oracle import refine

OMEGA = 2.0 / 3.0


def test_power_scale_is_exact_power_of_two():
    for R in (1.0, 1.5, 3.0, 1e-9, 7.3e5, 2.0**-40):
        s = refine.power_scale(R)
        assert math.frexp(s)[0] == 0.5  # a power of two
        assert 1.0 <= R * s < 2.0


def test_fp64_inner_refinement_is_plain_jacobi():
    """phi + e_n, with e_n from n sweeps on L e = r from 0, obeys the same
    recurrence as n plain sweeps from phi: cycles of n inner sweeps equal
    plain Jacobi in blocks of n (up to rounding)."""
    n, h = 32, 1.0 / 32
    rho = synth.random_field(np.random.default_rng(4), n, n)
    phi_r, hist = refine.refine_solve(rho, h, OMEGA, 0.0, 20, 5, fp32=False)
    phi_p, _ = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 100, 0)
    assert np.max(np.abs(phi_r - phi_p)) <= 1e-12 * np.max(np.abs(phi_p))
    for c, R in enumerate(hist):
        phi_c, _ = oracle.relax_n(np.zeros_like(rho), rho, h, OMEGA, 20 * c, 0)
        Rc, _ = oracle.residual_norm(phi_c, rho, h)
        assert abs(R - Rc) <= 1e-10 * hist[0]


def test_fp32_inner_refinement_reaches_fp64_accuracy():
    """FP32-storage sweeps alone stall near eps32 / (h^2 mu_min); the refined
    solution reaches 1e-10, which the plain FP32 iteration cannot."""
    n, h = 32, 1.0 / 32
    rho, _ = synth.modes_rho(n, n, 6, 6, 11)
    phi, hist = refine.refine_solve(rho, h, OMEGA, 1e-10, 200, 60, fp32=True)
    R, P = oracle.residual_norm(phi, rho, h)
    assert R <= 1e-10 * P
    assert hist[-1] == R
    # plain FP32 storage over the same number of sweeps stalls far above 1e-10
    e = np.zeros_like(rho)
    r32 = rho.astype(np.float32).astype(np.float64)
    for _ in range(200 * (len(hist) - 1)):
        e, _ = oracle.sweep(e, r32, h, OMEGA)
        e = e.astype(np.float32).astype(np.float64)
    R32, _ = oracle.residual_norm(e, rho, h)
    assert R32 > 1e-8 * P
    # and the FP32 refinement needs about as many cycles as FP64-inner refinement
    _, hist64 = refine.refine_solve(rho, h, OMEGA, 1e-10, 200, 60, fp32=False)
    assert abs(len(hist64) - len(hist)) <= 1

"""The oracle pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of oracle.c (on the CPU),
builds it, swaps it in for the real oracle and checks that at least one
pin of test_oracle_pins fails. The real oracle is restored afterwards.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import tests.test_oracle_pins as pins

MUTANTS = {
    "centre_tap": ("return ((pW + pE) + (pS + pN)) - 4.0 * pC;",
                   "return ((pW + pE) + (pS + pN)) - 3.0 * pC;"),
    "repeated_tap": ("return ((pW + pE) + (pS + pN)) - 4.0 * pC;",
                     "return ((pW + pE) + (pS + pS)) - 4.0 * pC;"),
    "transposed_wrap": ("wrapi(j + 1, ny)", "wrapi(j + 1, nx)"),
    "weight_half": ("double w = omega / 4.0, lam = omega * h * h / 4.0;\n  double R = 0.0;\n  for (int j = 0; j < ny; ++j)\n    for (int i = 0; i < nx; ++i) {\n      int64_t c",
                    "double w = omega / 2.0, lam = omega * h * h / 4.0;\n  double R = 0.0;\n  for (int j = 0; j < ny; ++j)\n    for (int i = 0; i < nx; ++i) {\n      int64_t c"),
    "lambda_without_omega": ("lam = omega * h * h / 4.0;\n  double R = 0.0;\n  for (int j = 0; j < ny; ++j)\n    for (int i = 0; i < nx; ++i) {\n      int64_t c",
                             "lam = h * h / 4.0;\n  double R = 0.0;\n  for (int j = 0; j < ny; ++j)\n    for (int i = 0; i < nx; ++i) {\n      int64_t c"),
    "rho_sign": ("phinew[c] = (phi[c] + w * s) - lam * rv;", "phinew[c] = (phi[c] + w * s) + lam * rv;"),
    "residual_sign": ("double r = fabs(ih2 * s - rv);\n      R = maxnan(R, r);\n    }\n  return R;",
                      "double r = fabs(ih2 * s + rv);\n      R = maxnan(R, r);\n    }\n  return R;"),
    "residual_of_output": ("double R = oracle_sweep(nx, ny, nx, h, omega, a, rho, b);\n    if (resid && every > 0 && s % every == 0) resid[s / every] = R;",
                           "oracle_sweep(nx, ny, nx, h, omega, a, rho, b);\n    double R; oracle_residual_norm(nx, ny, nx, h, b, rho, &R, 0);\n    if (resid && every > 0 && s % every == 0) resid[s / every] = R;"),
    "unscaled_stencil": ("out[(int64_t)j * ld + i] = ih2 * taps(", "out[(int64_t)j * ld + i] = taps("),
}

PIN_FUNCS = [
    pins.test_stencil_eigenmodes_closed_form,
    pins.test_small_field_trajectory_matches_closed_form,
    lambda: pins.test_dense_matrix_jacobi(3, 5),
    lambda: pins.test_special_gain_values(16, 16, 1.0 / 3.0),
    pins.test_residual_reports_are_input_state_norms,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    mut = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(so), str(c), "-lm"])
    saved = oracle._load()
    oracle._lib = oracle.bind(ctypes.CDLL(str(so)))
    caught = []
    try:
        for f in PIN_FUNCS:
            try:
                f()
            except AssertionError:
                caught.append(f)
    finally:
        oracle._lib = saved
    assert caught, f"mutant {name} passed every pin"

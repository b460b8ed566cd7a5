"""Writes the golden fixtures of tests/golden/ from the FP64 oracle only.

small_field_residuals.txt: the 64 x 64 workload (8 seeded modes, k, l in 1..16,
omega = 2/3, phi0 = 0), 1000 fused sweeps, the max-norm residual of states
0, 10, ..., 990 (the input state of sweeps 1, 11, ..., 991), one value per line,
17 significant digits. Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    _, rep = oracle.relax_n(np.zeros_like(rho), rho, 1.0 / 64, 2.0 / 3.0, 1000, 10)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_field_residuals.txt")
    with open(out, "w") as f:
        f.write("# 64x64 small-field workload, omega 2/3, phi0 = 0: ||rho - L phi^(10k)||_inf, "
                "k = 0..99 (FP64 oracle)\n")
        for v in rep:
            f.write(f"{v:.17g}\n")
    print(out)


if __name__ == "__main__":
    main()

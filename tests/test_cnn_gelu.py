"""The network kernels' GELU, restated on the CPU: erf from Abramowitz and
Stegun, Handbook of Mathematical Functions, formula 7.1.26 (for x >= 0,
erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1 / (1 +
p x), |error| <= 1.5e-7), evaluated in FP32 with the kernels' order of
operations (exact reciprocal and exponential here; the hardware ones add
relative errors near 2^-22). Checked against scipy's erf: the bound of the
formula, and the slack the GPU activation test leaves beyond one BF16
rounding, 1e-6 |z| + 0.01 u |GELU(z)| with u = 2^-8."""
import numpy as np
from scipy.special import erf

P, A = 0.3275911, (0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)


def gelu_kernel_form(z):
    f = np.float32
    t = f(1) / (f(P * 0.70710678118654752) * np.abs(z) + f(1))
    q = f(0.5 * A[4]) * t + f(0.5 * A[3])
    for a in (A[2], A[1], A[0]):
        q = q * t + f(0.5 * a)
    E = np.exp(f(-0.5) * z * z).astype(np.float32)
    h = (q * t) * E
    phi = np.where(z >= 0, f(1) - h, h)
    return (z * phi).astype(np.float64), phi.astype(np.float64), E.astype(np.float64)


def test_erf_within_the_formula_bound():
    z = np.linspace(-12, 12, 400001).astype(np.float32)
    _, phi, _ = gelu_kernel_form(z)
    ref = 0.5 * (1 + erf(z.astype(np.float64) / np.sqrt(2)))
    # Phi = (1 + erf) / 2: half the formula's bound plus FP32 rounding
    assert np.max(np.abs(phi - ref)) <= 0.5 * 1.5e-7 + 3e-7


def test_gelu_within_the_activation_slack():
    z = np.linspace(-12, 12, 4000001).astype(np.float32)
    g, _, _ = gelu_kernel_form(z)
    zd = z.astype(np.float64)
    ref = zd * 0.5 * (1 + erf(zd / np.sqrt(2)))
    assert np.max(np.abs(g - ref)) <= 4.3e-7
    assert np.all(np.abs(g - ref) <= 1e-6 * np.abs(zd) + 0.01 * 2.0 ** -8 * np.abs(ref))


def test_gelu_derivative_terms():
    z = np.linspace(-12, 12, 400001).astype(np.float32)
    _, phi, E = gelu_kernel_form(z)
    zd = z.astype(np.float64)
    d = phi + zd * 0.39894228040143268 * E
    ref = 0.5 * (1 + erf(zd / np.sqrt(2))) + zd * np.exp(-zd * zd / 2) / np.sqrt(2 * np.pi)
    assert np.max(np.abs(d - ref)) <= 5e-7

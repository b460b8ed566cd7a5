"""Golden fixture of the 64 x 64 workload (tests/golden/small_field_residuals.txt,
written by tests/golden/make_golden.py from the oracle). The stored history is
pinned to the closed-form trajectory r_n = sum_m A_m g_m^n v_m (every mode is a
discrete eigenfunction), and the CUDA path reproduces it."""
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    return np.loadtxt(os.path.join(HERE, "golden", "small_field_residuals.txt"))


def test_golden_history_is_the_closed_form():
    n, omega = 64, 2.0 / 3.0
    rho, modes = synth.small_field_rho(synth.workload_seed(0))
    gold = load()
    assert gold.shape == (100,)
    for k in (0, 1, 10, 50, 99):
        st = 10 * k
        r = np.zeros_like(rho)
        for m in modes:
            g = 1 - omega * (np.sin(np.pi * m.k / n) ** 2 + np.sin(np.pi * m.l / n) ** 2)
            vx, vy = synth.mode_vectors(m, n, n)
            r += m.amp * g**st * np.outer(vy, vx)
        assert abs(gold[k] - np.max(np.abs(r))) <= 1e-11 * np.max(np.abs(rho))


@pytest.mark.gpu
def test_gpu_reproduces_golden_history():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    rho, _ = synth.small_field_rho(synth.workload_seed(0))
    r = torch.from_numpy(rho).cuda()
    phi = torch.zeros_like(r)
    out = torch.empty_like(r)
    res = torch.zeros(100, dtype=torch.float64, device="cuda")
    px.relax_n(phi, out, r, 1.0 / 64, 2.0 / 3.0, 1000, 1, res, 10)
    gold = load()
    scale = 8 * float(out.abs().max()) * 64 * 64 + float(np.max(np.abs(rho)))
    assert np.max(np.abs(res.cpu().numpy() - gold)) <= 1e-10 * scale

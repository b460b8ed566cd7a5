"""What the trained network gains over the method without it.

The network shipped in paper_2307_07931_b300/data (trained by
paper_2307_07931_b300.learned) is applied to fresh 256 x 256 fields of the
learned-guess recipe, drawn from a seed stream used neither for training nor
for the recorded evaluation. The gain is measured in the method's own terms:
plain FP64 Jacobi sweeps to a relative residual of 1e-8 from phi0 = 0 against
from the network's guess (both judged by the same FP64 residual reports), and
wall time to 1e-8 of plain FP64 from zero against guess + mixed precision.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "paper_2307_07931_b300", "data")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    from paper_2307_07931_b300 import learned
    meta = json.load(open(os.path.join(DATA, "learned_guess.json")))
    net = px.Cnn(seed=0, dilations=tuple(meta["dilations"]))
    net.set_params(np.load(os.path.join(DATA, "learned_guess_params.npy")))
    rho = torch.from_numpy(learned.make_fields(learned.EVAL_SEED + 777, 16)).cuda()
    yield px, learned, net, rho
    net.close()


def test_guess_reduces_sweeps_to_1e8(setup):
    px, learned, net, rho = setup
    n = rho.shape[0]
    h = 1.0 / learned.N
    every, smax = 2000, 160000
    pn = np.array([px.residual_norm(torch.zeros_like(rho[i]), rho[i], h)[1] for i in range(n)])
    phi_z = torch.zeros_like(rho)
    rz = learned.batched_relax(px, torch, rho, phi_z, smax, every).cpu().numpy()
    phi_g = torch.empty_like(rho)
    net.guess(rho, phi_g, h)
    rg = learned.batched_relax(px, torch, rho, phi_g, smax, every).cpu().numpy()
    sz = learned.first_below(rz, pn, every, 1e-8)
    sg = learned.first_below(rg, pn, every, 1e-8)
    assert (sg >= 0).all()
    sz = np.where(sz >= 0, sz, smax)  # not reached within smax counts as smax (a lower bound)
    assert sg.mean() <= 0.9 * sz.mean(), (sz, sg)


def test_guess_plus_mixed_beats_plain_fp64_wall_time(setup):
    import time
    px, learned, net, rho = setup
    h = 1.0 / learned.N
    for i in range(2):
        r = rho[i]
        phi = torch.zeros_like(r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        px.solve(phi, r, h, "plain", rtol=1e-8, check_every=1000, tblock=1, max_sweeps=10**7)
        t_plain = time.perf_counter() - t0
        phi = torch.zeros_like(r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.guess(r[None], phi[None], h)
        info = px.solve(phi, r, h, "refine", rtol=1e-8, inner_sweeps=1000, tblock=8, max_sweeps=10**7)
        t_mix = time.perf_counter() - t0
        assert info["rel_resid"] <= 1e-8
        assert t_mix < t_plain, (t_mix, t_plain)

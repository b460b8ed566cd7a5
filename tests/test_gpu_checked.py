"""The checked build (libprotox_checked.so, -DPX_CHECKED): every global index
the relaxation, fused FP64 red-black and Euler kernels compute is checked against the field's
extent before the access (the stand-in for a memory sanitizer). On the
workloads below no check fails, and the checked build's results are bitwise
those of the normal build (the checks change no arithmetic). The checked
library runs in a child process (one library per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORK = r"""
import numpy as np, torch
def run(px):
    g = torch.Generator(device="cuda"); g.manual_seed(19)
    out = {}
    for (nx, ny, dt, tb, fam) in [(4096, 2048, torch.float32, 8, 0), (4096, 2052, torch.float32, 4, 0),
                                  (1000, 300, torch.float32, 8, 0), (1024, 512, torch.float32, 1, 0),
                                  (260, 150, torch.float64, 1, 0), (4100, 2049, torch.float32, 8, 3)]:
        ctx = px.Context(0)
        ctx.set_option(px.PX_OPT_FP32_FAMILY, fam)
        rho = torch.randn(ny, nx, device="cuda", dtype=dt, generator=g)
        phi = torch.randn(ny, nx, device="cuda", dtype=dt, generator=g)
        o = torch.empty_like(phi)
        r = torch.zeros(9, dtype=torch.float64, device="cuda")
        px.relax_n(phi, o, rho, 1.0 / nx, 2 / 3, 9, tb, r, 1, ctx=ctx)
        # pitched (scalar) layout
        pp = torch.zeros(ny, nx + 3, device="cuda", dtype=dt)[:, :nx]; pp.copy_(phi)
        pr = torch.zeros(ny, nx + 3, device="cuda", dtype=dt)[:, :nx]; pr.copy_(rho)
        po = torch.zeros(ny, nx + 3, device="cuda", dtype=dt)[:, :nx]
        px.relax_n(pp, po, pr, 1.0 / nx, 2 / 3, 3, 0, None, 0, ctx=ctx)
        torch.cuda.synchronize()
        out[f"relax_{nx}_{ny}_{tb}_{fam}"] = o.double().cpu().numpy()
        out[f"res_{nx}_{ny}_{tb}_{fam}"] = r.cpu().numpy()
        out[f"pitched_{nx}_{ny}_{tb}_{fam}"] = po.double().cpu().numpy()
        ctx.close()
    for (nx, ny) in [(1030, 514), (62, 6), (4096, 1024)]:
        rho = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
        phi = torch.randn(ny, nx, device="cuda", dtype=torch.float64, generator=g)
        o = torch.empty_like(phi)
        r = torch.zeros(5, dtype=torch.float64, device="cuda")
        px.rbsor_n(phi, o, rho, 1.0 / nx, 1.3, 5, r, 1)  # one fused launch per sweep
        torch.cuda.synchronize()
        out[f"rb_{nx}_{ny}"] = o.cpu().numpy()
        out[f"rbres_{nx}_{ny}"] = r.cpu().numpy()
    from oracle import euler as E
    rng = np.random.default_rng(4)
    for (nx, ny, dt) in [(130, 70, torch.float64), (512, 256, torch.float32), (33, 17, torch.float32)]:
        W = np.stack([1 + 0.3 * rng.uniform(-1, 1, (ny, nx)), 0.3 * rng.uniform(-1, 1, (ny, nx)),
                      0.3 * rng.uniform(-1, 1, (ny, nx)), 1 + 0.3 * rng.uniform(-1, 1, (ny, nx))])
        u = torch.from_numpy(E.conserved(W)).to(dt).cuda()
        o = torch.empty_like(u)
        d = torch.zeros(4, dtype=torch.float64, device="cuda")
        px.euler_step(u, o, 1.0 / nx, 1.0 / ny, 4, dt=d)
        torch.cuda.synchronize()
        out[f"euler_{nx}_{ny}"] = o.double().cpu().numpy()
        out[f"eulerdt_{nx}_{ny}"] = d.cpu().numpy()
    return out
"""

CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2307_07931_b300 as px
lib = px.load_library(px.LIB_CHECKED_PATH)
assert lib.px_is_checked_build() == 1
ns = {}
exec(sys.argv[3], ns)
out = ns["run"](px)
ctx = px.Context(0)
count, first = ctx.checked_faults()
np.savez(sys.argv[2], faults=np.array([count, first], dtype=np.uint64), **out)
"""


def test_checked_build_finds_nothing_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    from paper_2307_07931_b300 import build as pxbuild
    pxbuild.build(checked=True)  # no-op when up to date
    import paper_2307_07931_b300 as px
    assert px.load_library().px_is_checked_build() == 0
    with pytest.raises(px.PxError) as ei:
        px.context().checked_faults()
    assert ei.value.status == px.PX_EUNSUPPORTED
    res = str(tmp_path / "checked.npz")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, res, WORK], capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    got = np.load(res)
    assert int(got["faults"][0]) == 0, hex(int(got["faults"][1]))
    ns = {}
    exec(WORK, ns)
    ref = ns["run"](px)
    for k, v in ref.items():
        assert np.array_equal(got[k], v), k

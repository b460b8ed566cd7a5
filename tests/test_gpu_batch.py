"""GPU parity of the batched persistent relaxation (px_batch_plan / px_batch_run)
against the FP64 oracle, instance by instance, through the C ABI.

Each instance of a batch is an independent problem, so the oracle of a batch
is oracle.relax_n per instance. Tolerances are those of the single-grid tests:
FP64 n * 1e-12 relative, FP32 n * 2e-6 (inputs rounded to FP32 on both sides).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGA = 2.0 / 3.0


@pytest.fixture(scope="module")
def px():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as m
    return m


def make_instances(specs, seed):
    rng = np.random.default_rng(seed)
    phis, rhos, host = [], [], []
    for (nx, ny, dt) in specs:
        tdt = torch.float64 if dt == "f64" else torch.float32
        rho = synth.random_field(rng, nx, ny)
        phi = synth.random_field(rng, nx, ny, zero_mean=False)
        if dt == "f32":
            rho = rho.astype(np.float32).astype(np.float64)
            phi = phi.astype(np.float32).astype(np.float64)
        rhos.append(torch.from_numpy(rho).to(tdt).cuda())
        phis.append(torch.from_numpy(phi).to(tdt).cuda())
        host.append((phi, rho))
    return phis, rhos, host


def check(specs, phis, host, resid, nsweeps, every):
    nrep = (nsweeps + every - 1) // every
    res = resid.cpu().numpy().reshape(len(specs), nrep)
    for i, ((nx, ny, dt), (phi0, rho)) in enumerate(zip(specs, host)):
        h = 1.0 / nx
        ref, R = oracle.relax_n(phi0, rho, h, OMEGA, nsweeps, every)
        got = phis[i].double().cpu().numpy()
        tol = nsweeps * (1e-12 if dt == "f64" else 2e-6)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= tol, (i, nx, ny, dt, err)
        sc = 8 * max(np.max(np.abs(ref)), np.max(np.abs(phi0))) / h**2 + np.max(np.abs(rho))
        assert np.max(np.abs(res[i] - R)) <= tol * sc, (i, nx, ny, dt)


SPECS = [(32, 32, "f32"), (48, 48, "f64"), (64, 64, "f32"), (96, 96, "f64"), (128, 128, "f32"),
         (160, 160, "f32"), (112, 112, "f64"), (128, 128, "f64"), (256, 256, "f32"),
         (80, 48, "f32"), (512, 512, "f64"), (48, 96, "f64"), (1024, 64, "f32")]


@pytest.mark.parametrize("nsweeps", [7, 12])
def test_mixed_batch_matches_oracle(px, nsweeps):
    every = 2
    b = px.Batch([px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
                  for nx, ny, dt in SPECS], nsweeps, OMEGA, every)
    d = b.describe()
    modes = {k.split("@")[0]: v["mode"] for k, v in d["classes"].items()}
    assert d["cluster_size"] in (2, 4, 8)
    assert all(k.endswith(f"@c{d['cluster_size']}") for k in d["classes"])
    assert modes["f32:32x32"] == "whole" and modes["f64:512x512"] == "banded"
    nrep = (nsweeps + every - 1) // every
    for rep in range(2):  # the graph is replayed with new data
        phis, rhos, host = make_instances(SPECS, 100 * nsweeps + rep)
        resid = torch.full((len(SPECS) * nrep,), -1.0, dtype=torch.float64, device="cuda")
        b.run(phis, rhos, resid)
        torch.cuda.synchronize()
        check(SPECS, phis, host, resid, nsweeps, every)
    b.close()


def test_autotune_cache_roundtrip(px, tmp_path):
    specs = [(64, 64, "f32"), (96, 96, "f64"), (256, 256, "f32"), (256, 256, "f64")]
    grids = [px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
             for nx, ny, dt in specs]
    cache = str(tmp_path / "tune.json")
    b = px.Batch(grids, 10, OMEGA, 0, tune_cache=cache, tune=True)
    d = b.describe()
    assert all(v["tuned"] for v in d["classes"].values())
    assert all(v["rate_per_sm"] > 0 for v in d["classes"].values())
    data = json.load(open(cache))
    assert data["gpu"] == torch.cuda.get_device_name(0)
    assert set(d["classes"]) <= set(data["classes"])  # every candidate cluster size is cached
    # second plan reads the cache (no measurement) and runs correctly
    b2 = px.Batch(grids, 10, OMEGA, 1, tune_cache=cache, tune=False)
    d2 = b2.describe()
    for k, v in d2["classes"].items():
        assert v["tuned"] and v["mode"] == d["classes"][k]["mode"]
    phis, rhos, host = make_instances(specs, 5)
    resid = torch.zeros(len(specs) * 10, dtype=torch.float64, device="cuda")
    b2.run(phis, rhos, resid)
    torch.cuda.synchronize()
    check(specs, phis, host, resid, 10, 1)
    b.close()
    b2.close()


def test_batch_rejects_unsupported_layouts(px):
    with pytest.raises(px.PxError) as ei:
        px.Batch([px.Grid(30, 30, 30, 0, px.PX_F32, 1 / 30)], 4)
    assert ei.value.status == px.PX_EUNSUPPORTED
    with pytest.raises(px.PxError) as ei:
        px.Batch([px.Grid(32, 32, 34, 1, px.PX_F32, 1 / 32)], 4)
    assert ei.value.status == px.PX_EUNSUPPORTED


@pytest.mark.parametrize("tuned", [False, True])
def test_batched_workload_full_size(px, tmp_path, tuned):
    """1024 instances, N = 16 j (32..1024) log-uniform, FP64/FP32 by coin,
    8 modes each, 300 sweeps. Untuned (default rates, no configuration under
    the shared-memory cap): one persistent launch; tuned (as the benchmark
    plans it): the FP64 and FP32 launches side by side. Every instance's
    state-0 report is max|rho| exactly; a sample of instances (the largest of
    each dtype and small ones) is checked against the oracle."""
    ns, dts = synth.batch_sizes(1024)
    specs, phis, rhos, hostr = [], [], [], []
    for i, (n, dt) in enumerate(zip(ns, dts)):
        n = int(n)
        tdt = torch.float64 if dt == 0 else torch.float32
        rho = synth.batch_rho(n, i)
        r_t = torch.from_numpy(rho).to(tdt).cuda()
        specs.append((n, n, "f64" if dt == 0 else "f32"))
        rhos.append(r_t)
        phis.append(torch.zeros_like(r_t))
        hostr.append(rho if dt == 0 else rho.astype(np.float32).astype(np.float64))
    grids = [px.Grid(n, n, n, 0, px.PX_F64 if d == "f64" else px.PX_F32, 1.0 / n)
             for n, _, d in specs]
    b = px.Batch(grids, 300, OMEGA, 100, tune_cache=str(tmp_path / "t.json") if tuned else None,
                 tune=tuned)
    assert b.describe()["launches"] == (2 if tuned else 1)
    resid = torch.zeros(1024 * 3, dtype=torch.float64, device="cuda")
    b.run(phis, rhos, resid)
    torch.cuda.synchronize()
    res = resid.cpu().numpy().reshape(1024, 3)
    for i in range(1024):
        assert res[i, 0] == np.max(np.abs(hostr[i]))
    pick = set()
    for d in ("f64", "f32"):
        idx = [i for i, s in enumerate(specs) if s[2] == d]
        idx.sort(key=lambda i: specs[i][0])
        pick.update([idx[-1], idx[0], idx[len(idx) // 2]])
    for i in sorted(pick):
        n, _, d = specs[i]
        h = 1.0 / n
        ref, R = oracle.relax_n(np.zeros_like(hostr[i]), hostr[i], h, OMEGA, 300, 100)
        got = phis[i].double().cpu().numpy()
        tol = 300 * (1e-12 if d == "f64" else 2e-6)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), (i, n, d)
        sc = 8 * np.max(np.abs(ref)) / h**2 + np.max(np.abs(hostr[i]))
        assert np.max(np.abs(res[i] - R)) <= tol * sc, (i, n, d)
    b.close()


def test_plan_reports_allocation_failure(px):
    """A plan whose BANDED scratch cannot be allocated returns PX_ENOMEM at plan
    time, before anything is launched (the allocation failure is made on the
    host side by the size of the request)."""
    n = 1 << 29
    with pytest.raises(px.PxError) as ei:
        px.Batch([px.Grid(n, n, n, 0, px.PX_F32, 1.0 / n)], 2)
    assert ei.value.status == px.PX_ENOMEM
    # the context stays usable
    b = px.Batch([px.Grid(64, 64, 64, 0, px.PX_F32, 1 / 64)], 2)
    b.close()


def test_plan_picks_cluster_size_by_makespan(px):
    """One large FP64 instance among small ones: on 2-CTA clusters it alone would
    set the makespan, so the plan takes the candidate cluster size with the
    smallest predicted makespan (a larger one), and still matches the oracle."""
    specs = [(512, 512, "f64")] + [(32, 32, "f32")] * 40 + [(64, 64, "f64")] * 8
    b = px.Batch([px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
                  for nx, ny, dt in specs], 6, OMEGA, 3)
    d = b.describe()
    cands = d["candidates"]
    assert len(cands) >= 1
    best = min(c["predicted_ms"] for c in cands)
    assert abs(d["predicted_ms"] - best) <= 1e-9 * max(1.0, best)
    chosen = [c for c in cands if c["cluster_size"] == d["cluster_size"]
              and c["launches"] == d["launches"]][0]
    assert chosen["predicted_ms"] == best
    if any(c["cluster_size"] > 2 for c in cands):
        assert d["cluster_size"] > 2, cands
    phis, rhos, host = make_instances(specs, 77)
    resid = torch.full((len(specs) * 2,), -1.0, dtype=torch.float64, device="cuda")
    b.run(phis, rhos, resid)
    torch.cuda.synchronize()
    check(specs, phis, host, resid, 6, 3)
    b.close()


def _forced_cache(path, specs, mode, tb, ry=8):
    """A tune cache that pins every class (all cluster sizes) to one mode."""
    classes = {}
    for (nx, ny, dt) in specs:
        for cs in (2, 4, 8):
            m = mode if (mode != 2 or dt == "f32") else 1
            classes[f"{dt}:{nx}x{ny}@c{cs}"] = {"mode": m, "ry": ry, "tb": tb if m == 2 else 1,
                                                 "rate_per_sm": 1e9}
    with open(path, "w") as f:
        json.dump({"gpu": torch.cuda.get_device_name(0), "classes": classes}, f)


@pytest.mark.parametrize("tb,nsweeps,every", [(4, 7, 2), (4, 12, 3), (8, 13, 1), (8, 9, 0)])
def test_temporally_blocked_banded_mode(px, tmp_path, tb, nsweeps, every):
    """FP32 instances in the temporally blocked mode (tb sweeps per cluster
    barrier, tiles with a tb-cell periodic halo in shared memory) give bitwise
    the states and reports of the per-sweep banded mode, and match the oracle;
    shapes cover several tiles, ragged tiles, bands thinner than the halo and
    odd block counts (the copy back)."""
    specs = [(256, 256, "f32"), (160, 96, "f32"), (128, 20, "f32"), (36, 300, "f32"),
             (512, 128, "f32"), (96, 96, "f64"), (132, 70, "f32")]
    grids = [px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
             for nx, ny, dt in specs]
    results = {}
    for mode in (1, 2):
        cache = str(tmp_path / f"t{mode}.json")
        _forced_cache(cache, specs, mode, tb)
        b = px.Batch(grids, nsweeps, OMEGA, every, tune_cache=cache, tune=False)
        d = b.describe()
        want = "banded_t" if mode == 2 else "banded"
        assert all(v["mode"] == want for k, v in d["classes"].items() if k.startswith("f32")), d
        phis, rhos, host = make_instances(specs, 17)
        nrep = (nsweeps + every - 1) // every if every else 0
        resid = torch.zeros(max(1, len(specs) * nrep), dtype=torch.float64, device="cuda")
        b.run(phis, rhos, resid if every else None)
        torch.cuda.synchronize()
        if every:
            check(specs, phis, host, resid, nsweeps, every)
        results[mode] = ([p.cpu() for p in phis], resid.cpu())
        b.close()
    for a, c in zip(results[1][0], results[2][0]):
        assert torch.equal(a, c)
    assert torch.equal(results[1][1], results[2][1])


def test_mixed_plan_side_by_side_launches(px, tmp_path):
    """A batch of FP64 and FP32 instances runs as two launches side by side
    (one CTA of each on every SM: the FP64 sweeps are bound by the FP64 pipe,
    the FP32 ones by memory): classes whose mode needs more shared memory
    than the cap take their configuration under the cap (cache keys with the
    suffix "s"), and every instance still matches the oracle, states and
    reports, over two replays of the graph."""
    # enough small instances of both precisions that each launch holds
    # several per CTA (side by side then beats one launch in the planner's
    # model), plus classes over the cap, banded ones and ragged shapes
    specs = ([(64, 64, "f64")] * 296 + [(64, 64, "f32")] * 296 +
             [(32, 32, "f32"), (160, 160, "f32"), (128, 128, "f32"), (96, 96, "f64"),
              (48, 48, "f64"), (256, 256, "f32"), (256, 128, "f64"), (80, 48, "f32"),
              (1024, 64, "f32"), (112, 112, "f64")])
    whole_bytes = lambda nx, ny, dt: 2 * nx * ny * (8 if dt == "f64" else 4)
    classes = {}
    for (nx, ny, dt) in set(specs):
        for cs in (2, 4, 8):
            k = f"{dt}:{nx}x{ny}@c{cs}"
            fits = whole_bytes(nx, ny, dt) <= 200 * 1024
            classes[k] = {"mode": 0 if fits else 1, "ry": 8, "tb": 1, "rate_per_sm": 1e9}
            classes[k + "s"] = {"mode": 0 if whole_bytes(nx, ny, dt) <= 100 * 1024 else 1,
                                "ry": 8, "tb": 1, "rate_per_sm": 1e9}
    cache = str(tmp_path / "co.json")
    with open(cache, "w") as f:
        json.dump({"gpu": torch.cuda.get_device_name(0), "classes": classes}, f)
    nsweeps, every = 9, 2
    b = px.Batch([px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
                  for nx, ny, dt in specs], nsweeps, OMEGA, every, tune_cache=cache, tune=False)
    d = b.describe()
    assert d["launches"] == 2, d
    sbs = d["side_by_side"]
    assert d["smem"] <= sbs["smem_cap"] and sbs["fp32_smem"] <= sbs["smem_cap"]
    modes = {k.split("@")[0]: v["mode"] for k, v in d["classes"].items()}
    assert modes["f32:160x160"] == "banded" and modes["f64:96x96"] == "banded"
    assert modes["f32:32x32"] == "whole" and modes["f64:48x48"] == "whole"
    nrep = (nsweeps + every - 1) // every
    for rep in range(2):
        phis, rhos, host = make_instances(specs, 31 + rep)
        resid = torch.full((len(specs) * nrep,), -1.0, dtype=torch.float64, device="cuda")
        b.run(phis, rhos, resid)
        torch.cuda.synchronize()
        check(specs, phis, host, resid, nsweeps, every)
    b.close()
    # PX_OPT_BATCH_LAUNCHES = 1 keeps the same batch in one persistent launch,
    # with the same states and reports bit for bit (the per-instance sweeps
    # do not depend on the launch that runs them; configurations under the
    # cap are pinned for both plans by the cache)
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_BATCH_LAUNCHES, 1)
        assert ctx.get_option(px.PX_OPT_BATCH_LAUNCHES) == 1
        b1 = px.Batch([px.Grid(nx, ny, nx, 0, px.PX_F64 if dt == "f64" else px.PX_F32, 1.0 / nx)
                       for nx, ny, dt in specs], nsweeps, OMEGA, every, tune_cache=cache,
                      tune=False, ctx=ctx)
        assert b1.describe()["launches"] == 1
        phis2, rhos2, _ = make_instances(specs, 32)
        resid2 = torch.zeros_like(resid)
        b1.run(phis2, rhos2, resid2)
        torch.cuda.synchronize()
        b1.close()
        # the last two-launch run above used seed 32 as well
        for i, (nx, ny, dt) in enumerate(specs):
            if whole_bytes(nx, ny, dt) <= 100 * 1024:  # same mode in both plans
                assert torch.equal(phis[i], phis2[i]), (i, nx, ny, dt)
        assert torch.isfinite(resid2).all()
    finally:
        ctx.close()

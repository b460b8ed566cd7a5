"""Learned initial guess: data, labels, training and evaluation on one GPU.

Pipeline (every numerical step runs in the library's kernels through the C
ABI; PyTorch holds device memory and gathers training batches):
  1. fields: seeded 256 x 256 right-hand sides, 1-32 sine/cosine modes
     (k, l in 1..32) plus 0-4 periodic Gaussian blobs (sigma 2..20 cells),
     mean-zeroed (synth.learned_guess_rho); separate seed streams for the
     training and the held-out fields;
  2. labels: the FP64 solution of each training field, by FP64 multigrid
     V(2,2) cycles from 0 (px_mg_solve) to a relative residual of 1e-10 (or,
     with --label-solver jacobi, the plain FP64 solver for a fixed number of
     sweeps as batched persistent launches); the FP64 residual of every label
     is measured and reported;
  3. training: Adam on the MSE between the network output and phi / s for
     inputs rho h^2 / s (s = max|rho h^2|), cosine learning-rate decay, batches
     drawn with random symmetries of the square and periodic shifts (the
     periodic Poisson problem is equivariant to both);
  4. evaluation on held-out fields: sweeps of plain FP64 Jacobi to a relative
     residual of 1e-8 from phi0 = 0 and from the network's guess (batched, from
     residual reports), and wall time to 1e-8 on a sample of fields for plain
     FP64 from zero, FP32-in-FP64-refinement from zero, and the network guess
     followed by either solver.

Run: python -m paper_2307_07931_b300.learned --out DIR [--train N --eval N ...]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

N = 256
OMEGA = 2.0 / 3.0
TRAIN_SEED = 20230721          # learned-guess workload seed (training stream)
EVAL_SEED = 20230721 + 1000    # held-out stream


def make_fields(seed: int, count: int, n: int = N) -> np.ndarray:
    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((count, n, n))
    for i in range(count):
        out[i] = synth.learned_guess_rho(rng, n)
    return out


def make_fields_gpu(torch, seed: int, count: int, n: int = N, chunk: int = 1024):
    """make_fields on the device, generated and uploaded chunk by chunk (the
    same seed stream, so the same fields) to bound host memory."""
    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    out = torch.empty(count, n, n, dtype=torch.float64, device="cuda")
    buf = np.empty((chunk, n, n))
    for s0 in range(0, count, chunk):
        m = min(chunk, count - s0)
        for i in range(m):
            buf[i] = synth.learned_guess_rho(rng, n)
        out[s0:s0 + m].copy_(torch.from_numpy(buf[:m]))
    return out


def batched_relax(px, torch, rho, phi, sweeps: int, every: int, chunk: int = 1024):
    """phi (in place) <- `sweeps` plain FP64 sweeps of every field; returns the
    residual reports (count, ceil(sweeps / every)) of states 0, every, ..."""
    count = rho.shape[0]
    nrep = (sweeps + every - 1) // every
    reps = torch.zeros(count, nrep, dtype=torch.float64, device="cuda")
    plans = {}
    for s0 in range(0, count, chunk):
        m = min(chunk, count - s0)
        if m not in plans:
            g = px.Grid(N, N, N, 0, px.PX_F64, 1.0 / N)
            plans[m] = px.Batch([g] * m, sweeps, OMEGA, every)
        sub = reps[s0:s0 + m].reshape(-1)
        plans[m].run([phi[i] for i in range(s0, s0 + m)], [rho[i] for i in range(s0, s0 + m)], sub)
    torch.cuda.synchronize()
    for b in plans.values():
        b.close()
    return reps


def mg_labels(px, torch, rho, phi, cycles: int, rtol: float):
    """phi[i] <- FP64 multigrid V(2,2) cycles from 0 for every field, `cycles`
    per call, repeated until the final report meets rtol ||rho||; returns the
    relative residuals (the FP64 residual max-norm of each final state over
    ||rho||, both from the call's reports) and the cycles spent."""
    count = rho.shape[0]
    h = 1.0 / N
    res = torch.zeros(count, cycles + 1, dtype=torch.float64, device="cuda")
    for i in range(count):
        px.mg_solve(phi[i], rho[i], h, cycles, resid=res[i])
    R = res.cpu().numpy()
    rel = R[:, -1] / R[:, 0]
    spent = np.full(count, cycles)
    for i in np.nonzero(~(rel <= rtol))[0]:  # the rare field that needs more cycles
        r2 = torch.zeros(cycles + 1, dtype=torch.float64, device="cuda")
        for _ in range(8):
            px.mg_solve(phi[i], rho[i], h, cycles, resid=r2)
            spent[i] += cycles
            rel[i] = float(r2[-1]) / R[i, 0]
            if rel[i] <= rtol:
                break
    torch.cuda.synchronize()
    return rel, spent


def rel_residuals(px, torch, phi, rho):
    out = np.empty(rho.shape[0])
    for i in range(rho.shape[0]):
        R, P = px.residual_norm(phi[i], rho[i], 1.0 / N)
        out[i] = R / P
    return out


def first_below(reps, rho_norms, every: int, tol: float):
    """Sweeps to reach tol from the reports (state index of the first report
    below tol); -1 where it was not reached."""
    rel = reps / rho_norms[:, None]
    hit = rel <= tol
    idx = np.where(hit.any(axis=1), hit.argmax(axis=1), -1)
    return np.where(idx >= 0, idx * every, -1)


def augment(torch, x, t, rng):
    k = int(rng.integers(0, 4))
    if k:
        x = torch.rot90(x, k, dims=(1, 2))
        t = torch.rot90(t, k, dims=(1, 2))
    if rng.integers(0, 2):
        x = torch.flip(x, dims=(2,))
        t = torch.flip(t, dims=(2,))
    sy, sx = (int(v) for v in rng.integers(0, N, 2))
    x = torch.roll(x, shifts=(sy, sx), dims=(1, 2)).contiguous()
    t = torch.roll(t, shifts=(sy, sx), dims=(1, 2)).contiguous()
    return x, t


def save_checkpoint(path: str, net, step: int, rng, hist):
    """Parameters, Adam moments and step of the network, the data-order RNG
    state and the loss history, written atomically."""
    state, adam_step = net.state()
    tmp = path + ".tmp.npz"
    np.savez(tmp, state=state, adam_step=adam_step, step=step,
             rng=json.dumps(rng.bit_generator.state), hist=np.array(hist, dtype=np.float64))
    os.replace(tmp, path)


def load_checkpoint(path: str, net, rng):
    z = np.load(path)
    net.set_state(z["state"], int(z["adam_step"]))
    rng.bit_generator.state = json.loads(str(z["rng"]))
    hist = [tuple(v) for v in z["hist"].tolist()]
    return int(z["step"]), hist


def train(px, torch, net, X, T, steps: int, batch: int, lr0: float, seed: int, log,
          ckpt: str | None = None, ckpt_every: int = 0, stop_at: int | None = None):
    """Adam with cosine decay. With `ckpt`, the full training state is written
    every `ckpt_every` steps and an existing checkpoint is resumed; a resumed run
    continues bit for bit as the uninterrupted one (fixed-order reductions, the
    same batch indices and augmentations from the restored RNG). `stop_at` ends
    the run early at that step (an interrupted run)."""
    rng = np.random.default_rng(seed)
    ntrain = X.shape[0]
    hist = []
    start = 0
    if ckpt and os.path.exists(ckpt):
        start, hist = load_checkpoint(ckpt, net, rng)
        log(f"resumed from {ckpt} at step {start}")
    t0 = time.perf_counter()
    for s in range(start, steps):
        idx = torch.from_numpy(rng.integers(0, ntrain, batch)).cuda()
        xb, tb = augment(torch, X.index_select(0, idx), T.index_select(0, idx), rng)
        lr = 1e-5 + 0.5 * (lr0 - 1e-5) * (1 + math.cos(math.pi * s / max(1, steps)))
        want = (s % 200 == 0) or s == steps - 1
        loss = net.train_step(xb, tb, lr, want_loss=want)
        if want:
            hist.append((s, loss))
            log(f"step {s} loss {loss:.4e} lr {lr:.2e} {time.perf_counter() - t0:.1f}s")
        if ckpt and ckpt_every > 0 and (s + 1) % ckpt_every == 0:
            save_checkpoint(ckpt, net, s + 1, rng, hist)
        if stop_at is not None and s + 1 >= stop_at:
            break
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def timed_solves(px, torch, net, rho, sample: int, rtol: float):
    """Per-field wall time to rtol (host clock around the calls, which
    synchronise): plain FP64 from 0, mixed from 0, guess + plain FP64,
    guess + mixed."""
    h = 1.0 / N
    res = {k: [] for k in ("plain_f64_zero", "mixed_zero", "cnn_plain_f64", "cnn_mixed")}
    sweeps = {k: [] for k in res}
    for i in range(sample):
        r = rho[i]
        for key in res:
            phi = torch.zeros_like(r)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if key.startswith("cnn"):
                net.guess(r[None], phi[None], h)
            if key.endswith("mixed") or key == "mixed_zero":
                info = px.solve(phi, r, h, "refine", rtol=rtol, inner_sweeps=1000, tblock=8,
                                max_sweeps=10**7)
            else:
                info = px.solve(phi, r, h, "plain", rtol=rtol, check_every=1000, tblock=1,
                                max_sweeps=10**7)
            res[key].append(time.perf_counter() - t0)
            sweeps[key].append(info["sweeps"])
    return {k: {"mean_ms": 1000 * float(np.mean(v)), "median_ms": 1000 * float(np.median(v)),
                "mean_sweeps": float(np.mean(sweeps[k]))} for k, v in res.items()}


def main():
    import torch
    import paper_2307_07931_b300 as px
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--train", type=int, default=50000)
    ap.add_argument("--eval", type=int, default=4096)
    ap.add_argument("--label-solver", default="mg", choices=["mg", "jacobi"])
    ap.add_argument("--label-rtol", type=float, default=1e-10)
    ap.add_argument("--label-cycles", type=int, default=10, help="multigrid cycles per call")
    ap.add_argument("--label-sweeps", type=int, default=40000, help="plain sweeps (jacobi labels)")
    ap.add_argument("--eval-sweeps", type=int, default=160000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--timed", type=int, default=32)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--ckpt", default=None, help="checkpoint file (.npz); resumed if present")
    ap.add_argument("--ckpt-every", type=int, default=1000)
    ap.add_argument("--dilations", default="1,3,9,27,81,1",
                    help="per-layer dilations of the 3x3 layers ('1,1,1,1,1,1' = plain)")
    a = ap.parse_args()
    os.makedirs(a.out, exist_ok=True)
    logf = open(os.path.join(a.out, "learned_log.txt"), "w")

    def log(msg):
        print(msg, flush=True)
        logf.write(msg + "\n")
        logf.flush()

    px.load_library()
    res = {"config": {k: v for k, v in vars(a).items() if k not in ("out", "ckpt")}, "grid": N,
           "omega": OMEGA}
    t0 = time.perf_counter()
    rho_tr = make_fields_gpu(torch, TRAIN_SEED, a.train)
    rho_ev = make_fields_gpu(torch, EVAL_SEED, a.eval)
    res["fields_s"] = time.perf_counter() - t0
    log(f"fields {a.train} + {a.eval} in {res['fields_s']:.1f}s")

    # labels: the FP64 solution of every training field
    t0 = time.perf_counter()
    phi_tr = torch.zeros_like(rho_tr)
    if a.label_solver == "mg":
        rel, spent = mg_labels(px, torch, rho_tr, phi_tr, a.label_cycles, a.label_rtol)
        how = f"FP64 multigrid V(2,2), {a.label_cycles} cycles per call, {int(spent.max())} at most"
    else:
        batched_relax(px, torch, rho_tr, phi_tr, a.label_sweeps, a.label_sweeps)
        rel = rel_residuals(px, torch, phi_tr, rho_tr)
        how = f"{a.label_sweeps} plain FP64 sweeps"
    res["label_s"] = time.perf_counter() - t0
    res["label_solver"] = how
    res["label_rel_resid"] = {"max": float(rel.max()), "median": float(np.median(rel)),
                              "p90": float(np.quantile(rel, 0.9))}
    log(f"labels: {how} in {res['label_s']:.1f}s, rel resid "
        f"median {np.median(rel):.2e} max {rel.max():.2e}")

    dil = tuple(int(v) for v in a.dilations.split(","))
    net = px.Cnn(seed=a.seed, dilations=dil)
    X = torch.empty(a.train, N, N, dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    for s0 in range(0, a.train, 256):
        s1 = min(a.train, s0 + 256)
        net.prepare(rho_tr[s0:s1], phi_tr[s0:s1], X[s0:s1], T[s0:s1], 1.0 / N)
    # Jacobi from 0 keeps the mean of phi at 0 (the zero mode has gain 1 and
    # rho is mean-zero), so the targets are already the mean-zero solution.
    del phi_tr
    hist, tsec = train(px, torch, net, X, T, a.steps, a.batch, a.lr, a.seed, log,
                       ckpt=a.ckpt, ckpt_every=a.ckpt_every)
    res["train"] = {"steps": a.steps, "batch": a.batch, "seconds": tsec,
                    "ms_per_step": 1000 * tsec / max(1, a.steps), "loss_history": hist}
    np.save(os.path.join(a.out, "learned_guess_params.npy"), net.params())
    del X, T

    # evaluation: sweeps to 1e-8 from 0 and from the guess (batched FP64)
    t0 = time.perf_counter()
    phi_z = torch.zeros_like(rho_ev)
    reps_z = batched_relax(px, torch, rho_ev, phi_z, a.eval_sweeps, a.every).cpu().numpy()
    tz = time.perf_counter() - t0
    del phi_z
    phi_g = torch.empty_like(rho_ev)
    t0 = time.perf_counter()
    for s0 in range(0, a.eval, 64):
        s1 = min(a.eval, s0 + 64)
        net.guess(rho_ev[s0:s1], phi_g[s0:s1], 1.0 / N)
    torch.cuda.synchronize()
    tguess = time.perf_counter() - t0
    rp = np.array([px.residual_norm(phi_g[i], rho_ev[i], 1.0 / N) for i in range(a.eval)])
    pn = rp[:, 1]
    g_rel0 = rp[:, 0] / pn
    t0 = time.perf_counter()
    reps_g = batched_relax(px, torch, rho_ev, phi_g, a.eval_sweeps, a.every).cpu().numpy()
    tg = time.perf_counter() - t0
    sz = first_below(reps_z, pn, a.every, 1e-8)
    sg = first_below(reps_g, pn, a.every, 1e-8)
    both = (sz >= 0) & (sg >= 0)
    res["eval"] = {
        "fields": a.eval, "max_sweeps": a.eval_sweeps, "report_every": a.every,
        "converged_from_zero": int((sz >= 0).sum()), "converged_from_guess": int((sg >= 0).sum()),
        "mean_sweeps_from_zero": float(sz[both].mean()) if both.any() else None,
        "mean_sweeps_from_guess": float(sg[both].mean()) if both.any() else None,
        "median_sweeps_from_zero": float(np.median(sz[both])) if both.any() else None,
        "median_sweeps_from_guess": float(np.median(sg[both])) if both.any() else None,
        "sweep_ratio_mean": float(sz[both].mean() / max(1.0, sg[both].mean())) if both.any() else None,
        "guess_rel_resid_median": float(np.median(g_rel0)),
        "guess_time_ms_per_field": 1000 * tguess / a.eval,
        "batched_eval_s": {"from_zero": tz, "from_guess": tg},
    }
    log(json.dumps(res["eval"]))
    res["timed"] = timed_solves(px, torch, net, rho_ev, min(a.timed, a.eval), 1e-8)
    log(json.dumps(res["timed"]))
    net.close()
    with open(os.path.join(a.out, "learned_results.json"), "w") as f:
        json.dump(res, f, indent=1)
    logf.close()


if __name__ == "__main__":
    main()

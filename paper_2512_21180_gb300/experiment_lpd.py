"""Learned primal-dual vs PDHG-TV on simulated data (the learned workload).

Trains the unrolled learned primal-dual network on seeded ellipsoid phantoms with
Poisson noise (128^3 at 4 mm, 200 angles, 256x192 panel at 1.6 mm with +80 mm
offset, I0 = 1e5 photons/pixel), starting every reconstruction from FDK_w, and
compares it with 100 iterations of FP32 PDHG-TV (lambda tuned on held-out
phantoms) on test phantoms: PSNR over the full field of view (voxels seen by at
least half of the projections, Sec. 2.4) and GPU seconds per volume.

    python -m paper_2512_21180_gb300.experiment_lpd [--train 512] [--test 32] [--epochs 2]
           [--minutes 20] [--out results.json]

Everything runs in libcbct (projectors, convs, simulation, FDK, PDHG, Adam);
PyTorch holds the buffers.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import inputs as I
from . import ops
from .lpd import LPD, masked_mse
from .projector import Geometry

WORKLOAD = "lpd128"
I0 = 1e5


def psnr(x: torch.Tensor, ref: torch.Tensor, mask: torch.Tensor) -> float:
    """10 log10(max(ref)^2 / MSE) over the mask (the data range is the reference's
    maximum, a reading: the paper does not state it)."""
    m = mask.bool()
    mse = torch.mean((x[m] - ref[m]).double() ** 2).item()
    peak = ref[m].max().item()
    return 10.0 * math.log10(peak * peak / max(mse, 1e-30))


def make_set(geom: Geometry, g: dict, seeds, noise_seed0: int):
    out = []
    for j, s in enumerate(seeds):
        x = ops.phantom(geom, I.phantom_params(WORKLOAD, s))
        _, y = ops.simulate(geom, x, I0, seed=noise_seed0 + j)
        x0 = ops.fdk(geom, y)[0]
        out.append((x, y[0], x0))
    return out


def timed(fn, reps: int = 3):
    for _ in range(1):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        r = fn()
    e1.record()
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1) / reps / 1e3


def profile_pass(args) -> int:
    torch.cuda.set_device(0)
    geom = Geometry(I.geometry(WORKLOAD))
    V = ops.fov(geom)
    x = ops.phantom(geom, I.phantom_params(WORKLOAD, 30_000))
    _, y = ops.simulate(geom, x, I0, seed=1)
    x0 = ops.fdk(geom, y)[0]
    model = LPD(geom, n_iter=args.n_iter, seed=1)
    for _ in range(2):
        model.forward(y[0], x0)
    torch.cuda.synchronize()
    model.forward(y[0], x0)
    out = model.forward(y[0], x0, save_for_backward=True)
    model.zero_grad()
    _, gr = masked_mse(out, x, V, 0.5)
    model.backward(gr)
    model.adam_step(1e-4)
    torch.cuda.synchronize()
    print("profile pass done", flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--tune", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--minutes", type=float, default=20.0, help="training time budget")
    ap.add_argument("--batch", type=int, default=8, help="effective batch (gradient accumulation)")
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--clip", type=float, default=1.0, help="global gradient-norm clip (loss in mu_ref^2 units)")
    ap.add_argument("--warmup", type=int, default=40, help="linear learning-rate warm-up steps")
    ap.add_argument("--n-iter", type=int, default=8)
    ap.add_argument("--pdhg-iters", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    ap.add_argument("--profile", action="store_true",
                    help="only run 2 warm-up passes, then one inference and one training step on one phantom "
                         "(a short command for profilers)")
    args = ap.parse_args(argv)
    if args.profile:
        return profile_pass(args)

    torch.cuda.set_device(0)
    g = I.geometry(WORKLOAD)
    geom = Geometry(g)
    V = ops.fov(geom)
    full = (V >= 0.5).float()
    log = {"workload": "128^3 at 4 mm, 200 angles, 256x192 at 1.6 mm, +80 mm offset, Poisson I0=1e5",
           "train": args.train, "test": args.test}

    t0 = time.time()
    train = make_set(geom, g, range(10_000, 10_000 + args.train), 1)
    tune = make_set(geom, g, range(20_000, 20_000 + args.tune), 50_000)
    test = make_set(geom, g, range(30_000, 30_000 + args.test), 90_000)
    log["data_s"] = time.time() - t0
    print(f"data ready in {log['data_s']:.1f} s", file=sys.stderr, flush=True)

    # ---- PDHG-TV: step sizes from the operator norm, lambda tuned on held-out phantoms
    nP = ops.opnorm(geom, 0.0, 30)
    gam = nP / math.sqrt(12.0)
    nK = ops.opnorm(geom, gam, 30)
    sig = tau = 0.99 / nK
    lams = [1e-3, 3e-3, 1e-2, 3e-2, 1e-1, 3e-1, 1.0, 3.0, 10.0]
    best = None
    for lam in lams:
        ps = [psnr(ops.pdhg(geom, y, x0, args.pdhg_iters, lam, gam, sig, tau)[0], x, full) for x, y, x0 in tune]
        m = float(np.mean(ps))
        print(f"pdhg lambda {lam:g}: tune PSNR {m:.2f}", file=sys.stderr, flush=True)
        if best is None or m > best[1]:
            best = (lam, m)
    lam = best[0]
    log["pdhg"] = {"lambda": lam, "iters": args.pdhg_iters, "sigma": sig, "tau": tau, "gamma": gam}

    # ---- train the learned primal-dual network
    model = LPD(geom, n_iter=args.n_iter, seed=1)
    t_train = time.time()
    step = 0
    est_steps = 10 ** 9
    losses = []
    norms = []
    order = np.random.default_rng(0)
    done = False
    for ep in range(args.epochs):
        perm = order.permutation(len(train))
        for b0 in range(0, len(perm) - args.batch + 1, args.batch):
            model.zero_grad()
            tot = 0.0
            for j in perm[b0:b0 + args.batch]:
                x, y, x0 = train[j]
                out = model.forward(y, x0, save_for_backward=True)
                loss, gr = masked_mse(out, x, V, 0.5)
                model.backward(gr)
                tot += loss.item()
            # loss in units of mu_ref^2 (O(1)); linear warm-up, then cosine decay over the
            # number of steps the time budget allows (estimated after the warm-up)
            if step == args.warmup and step > 0:
                est_steps = max(step + 1, int(args.minutes * 60 / ((time.time() - t_train) / step)))
            if step < args.warmup:
                lr = args.lr * (step + 1) / max(1, args.warmup)
            else:
                lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * min(1.0, (step - args.warmup) /
                                                                   max(1, est_steps - args.warmup))))
            gscale = 1.0 / (args.batch * model.mu_ref ** 2)
            norms.append(model.clip_grads(args.clip, grad_scale=gscale))
            model.adam_step(lr, grad_scale=gscale)
            step += 1
            losses.append(tot / args.batch)
            if step % 8 == 0:
                print(f"epoch {ep} step {step} loss {np.mean(losses[-8:]):.3e} grad norm "
                      f"{np.median(norms[-8:]):.3e} lr {lr:.2e} ({time.time() - t_train:.0f} s)",
                      file=sys.stderr, flush=True)
            if time.time() - t_train > args.minutes * 60:
                done = True
                break
        if done:
            break
    if args.save:
        np.save(args.save, model.get_params())
    log["training"] = {"steps": step, "effective_batch": args.batch, "lr": args.lr, "warmup": args.warmup,
                       "clip": args.clip, "grad_norm_median": float(np.median(norms)) if norms else None,
                       "seconds": time.time() - t_train, "loss_first": losses[0] if losses else None,
                       "loss_last8": float(np.mean(losses[-8:])) if losses else None}

    # ---- evaluate: PSNR and GPU seconds per volume
    res = {"fdk": [], "pdhg": [], "lpd": []}
    t_lpd = t_pdhg = t_fdk = 0.0
    for x, y, x0 in test:
        _, tf = timed(lambda: ops.fdk(geom, y), reps=1)
        r_p, tp = timed(lambda: ops.pdhg(geom, y, x0, args.pdhg_iters, lam, gam, sig, tau)[0], reps=1)
        r_l, tl = timed(lambda: model.forward(y, x0), reps=1)
        t_fdk += tf
        t_pdhg += tp
        t_lpd += tl
        res["fdk"].append(psnr(x0, x, full))
        res["pdhg"].append(psnr(r_p, x, full))
        res["lpd"].append(psnr(r_l, x, full))
    n = len(test)
    log["psnr_fullfov"] = {k: {"mean": float(np.mean(v)), "sd": float(np.std(v))} for k, v in res.items()}
    log["seconds_per_volume"] = {"fdk": t_fdk / n, "pdhg": t_pdhg / n, "lpd": t_lpd / n + t_fdk / n}
    log["lpd_speedup_vs_pdhg"] = (t_pdhg / n) / (t_lpd / n + t_fdk / n)
    log["lpd_minus_pdhg_psnr_db"] = log["psnr_fullfov"]["lpd"]["mean"] - log["psnr_fullfov"]["pdhg"]["mean"]
    print(json.dumps(log), flush=True)
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "w") as f:
            json.dump(log, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Learned primal-dual vs PDHG-TV on simulated data (the learned workload).

Trains the unrolled learned primal-dual network on seeded ellipsoid phantoms with
Poisson noise (128^3 at 4 mm, 200 angles, 256x192 panel at 1.6 mm with +80 mm
offset, I0 = 1e5 photons/pixel), starting every reconstruction from FDK_w, and
compares it with 100 iterations of FP32 PDHG-TV (lambda tuned on held-out
phantoms) on test phantoms: PSNR over the full field of view (voxels seen by at
least half of the projections, Sec. 2.6) and GPU seconds per volume.

    python -m paper_2512_21180_gb300.experiment_lpd [--train 512] [--test 32] [--epochs 2]
           [--minutes 20] [--residual-input] [--vol-batch 4] [--out results.json] [--save w.npy]

The comparison is made at equal PSNR (equal_psnr): the smallest number of PDHG
iterations whose mean test PSNR reaches the learned reconstruction's, and the GPU
time of each to get there.

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


def widen_params(flat: np.ndarray, n_iter: int, n_mem: int, width: int, residual_input: bool) -> np.ndarray:
    """Parameters for the network with the data-residual channel from those of the same
    network without it (or unchanged when they already fit): each dual block's first
    layer gains zero weights for the extra input, so both networks compute the same
    function and training continues from there."""
    from .lpd import layer_shapes
    new_shapes = layer_shapes(n_iter, n_mem, width, residual_input)
    if flat.size == sum(co * t * ci + co for co, t, ci in new_shapes):
        return flat.astype(np.float32)
    old_shapes = layer_shapes(n_iter, n_mem, width, False)
    if flat.size != sum(co * t * ci + co for co, t, ci in old_shapes):
        raise ValueError("parameter count fits neither layout")
    out, o = [], 0
    for (co, t, ci), (_, _, ci2) in zip(old_shapes, new_shapes):
        w = flat[o:o + co * t * ci].reshape(co, t, ci)
        o += co * t * ci
        w2 = np.zeros((co, t, ci2), dtype=np.float32)
        w2[:, :, :ci] = w
        out += [w2.reshape(-1), flat[o:o + co]]
        o += co
    return np.concatenate(out).astype(np.float32)


def event_seconds(fn, reps: int = 3, warmup: int = 1) -> float:
    """GPU seconds per call of fn (CUDA events on the current stream, after warm-up)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def equal_psnr(geom: Geometry, model: LPD, test, full: torch.Tensor, lam: float, gam: float, sig: float, tau: float,
               kmax: int = 1600, batch: int = 4) -> dict:
    """The learned reconstruction against PDHG-TV at equal PSNR on a test set of
    (x_true, y, x0 = FDK_w) triples: the mean PSNR over FullFoV of the LPD (FDK_w start +
    unrolled iterations), the smallest PDHG iteration count k* whose mean PSNR reaches it
    (bisection over k, PDHG's mean PSNR taken as non-decreasing in k; doubling past 100
    when needed, up to kmax), and GPU seconds per volume of FDK_w + LPD and of FDK_w + k*
    PDHG iterations, one volume per call and (batch > 1) `batch` volumes per call."""
    cache = {}

    def pdhg_psnr(k):
        if k not in cache:
            cache[k] = float(np.mean([psnr(ops.pdhg(geom, y, x0, k, lam, gam, sig, tau)[0], x, full)
                                      for x, y, x0 in test]))
        return cache[k]

    p_lpd = float(np.mean([psnr(model.forward(y, x0), x, full) for x, y, x0 in test]))
    p_fdk = float(np.mean([psnr(x0, x, full) for x, y, x0 in test]))
    _, y1, _ = test[0]
    t_lpd = event_seconds(lambda: model.forward(y1, ops.fdk(geom, y1)[0]))
    p100 = pdhg_psnr(100)
    lo, hi = 0, 100
    if p100 < p_lpd:
        lo, hi = 100, 200
        while hi <= kmax and pdhg_psnr(hi) < p_lpd:
            lo, hi = hi, 2 * hi
    if hi <= kmax:
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if pdhg_psnr(mid) >= p_lpd:
                hi = mid
            else:
                lo = mid
        k_eq = hi
    else:
        k_eq = None
    t_pdhg = lambda k: event_seconds(lambda: ops.pdhg(geom, y1, ops.fdk(geom, y1)[0], k, lam, gam, sig, tau),
                                     reps=1)
    t100 = t_pdhg(100)
    out = {"n_test": len(test), "lambda": lam, "psnr_fdk": p_fdk, "psnr_lpd": p_lpd, "psnr_pdhg100": p100,
           "lpd_s_per_volume": t_lpd, "pdhg100_s_per_volume": t100, "pdhg100_over_lpd": t100 / t_lpd,
           "pdhg_iters_to_lpd_psnr": k_eq,
           "pdhg_psnr_by_iters": {str(k): v for k, v in sorted(cache.items())}}
    if k_eq is not None:
        t_eq = t_pdhg(k_eq)
        out.update({"pdhg_s_at_lpd_psnr": t_eq, "pdhg_over_lpd_at_equal_psnr": t_eq / t_lpd})
    else:
        out.update({"pdhg_s_at_lpd_psnr": None, "pdhg_over_lpd_at_equal_psnr": None,
                    "note": f"PDHG does not reach the LPD's PSNR within {kmax} iterations"})
    if batch > 1 and len(test) >= batch:
        # both methods on `batch` volumes per call (one launch of each kernel covers the batch)
        mb = LPD(geom, n_iter=model.n_iter, n_mem=model.n_mem, width=model.width, mu_ref=model.mu_ref,
                 residual_input=model.residual_input, reversible=model.reversible and not model.lire, lire=model.lire,
                 p4=model.p4, unet=model.unet, weight_norm=model.weight_norm, max_batch=batch)
        mb.set_params(model.get_params())
        if model.reversible:
            mb.set_perms(model.perms())
        yb = torch.stack([t[1] for t in test[:batch]])
        tb_lpd = event_seconds(lambda: mb.forward(yb, ops.fdk(geom, yb))) / batch
        tb_eq = None
        if k_eq is not None:
            tb_eq = event_seconds(lambda: ops.pdhg(geom, yb, ops.fdk(geom, yb), k_eq, lam, gam, sig, tau),
                                  reps=1) / batch
        tb100 = event_seconds(lambda: ops.pdhg(geom, yb, ops.fdk(geom, yb), 100, lam, gam, sig, tau), reps=1) / batch
        out[f"batch{batch}"] = {"lpd_s_per_volume": tb_lpd, "pdhg100_s_per_volume": tb100,
                                "pdhg100_over_lpd": tb100 / tb_lpd,
                                "pdhg_s_at_lpd_psnr": tb_eq,
                                "pdhg_over_lpd_at_equal_psnr": None if tb_eq is None else tb_eq / tb_lpd}
        mb.close()
    return out


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


def time_training(args) -> int:
    """GPU seconds per volume of one training step (forward with stored states, masked
    loss, backward, clipping, Adam) on `vol_batch` volumes per call, and of one inference
    pass, for the configured network on the learned workload. Prints one JSON line."""
    torch.cuda.set_device(0)
    geom = Geometry(I.geometry(WORKLOAD))
    V = ops.fov(geom)
    vb = args.vol_batch
    model = LPD(geom, n_iter=args.n_iter, n_mem=args.n_mem, width=args.width, seed=1,
                residual_input=args.residual_input, max_batch=vb, reversible=args.reversible, lire=args.lire,
                p4=args.p4, unet=args.unet, weight_norm=args.weight_norm)
    xs, ys = [], []
    for j in range(vb):
        x = ops.phantom(geom, I.phantom_params(WORKLOAD, 10_000 + j))
        _, y = ops.simulate(geom, x, I0, seed=j)
        xs.append(x)
        ys.append(y[0])
    x = torch.stack(xs)
    y = torch.stack(ys)
    x0 = ops.fdk(geom, y)
    Vb = V.expand((vb,) + tuple(V.shape)).contiguous()

    def step():
        model.zero_grad()
        out = model.forward(y, x0, save_for_backward=True)
        _, gr = masked_mse(out, x, Vb, 0.5)
        model.backward(gr)
        model.clip_grads(1.0, grad_scale=1.0 / model.mu_ref ** 2)
        model.adam_step(1e-5, grad_scale=1.0 / model.mu_ref ** 2)

    t_train = event_seconds(step, reps=args.reps, warmup=2) / vb
    t_inf = event_seconds(lambda: model.forward(y, x0), reps=args.reps, warmup=1) / vb
    print(json.dumps({"workload": "128^3 at 4 mm, 200 angles, 256x192 at 1.6 mm, +80 mm offset",
                      "n_iter": args.n_iter, "n_mem": args.n_mem, "width": args.width,
                      "residual_input": args.residual_input,
                      "reversible": model.reversible, "lire": model.lire, "p4": model.p4, "unet": model.unet,
                      "weight_norm": model.weight_norm,
                      "volumes_per_call": vb, "train_s_per_volume": t_train, "inference_s_per_volume": t_inf}),
          flush=True)
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
    ap.add_argument("--residual-input", action="store_true",
                    help="dual blocks also receive the FP32-formed data residual mu_ref P f_1 - y")
    ap.add_argument("--vol-batch", type=int, default=4, help="volumes per forward/backward call")
    ap.add_argument("--n-mem", type=int, default=5, help="memory channels (even for --reversible / --lire)")
    ap.add_argument("--width", type=int, default=32, help="hidden channels of the blocks: 32 or 64")
    ap.add_argument("--reversible", action="store_true", help="additive coupling + permutations (no stored iterates)")
    ap.add_argument("--lire", action="store_true", help="the iteration of Algorithm 1 (implies --reversible)")
    ap.add_argument("--p4", action="store_true", help="P4-equivariant primal blocks")
    ap.add_argument("--unet", action="store_true", help="P4 U-Net primal blocks (depth 1)")
    ap.add_argument("--weight-norm", action="store_true", help="forced weight normalisation of every layer")
    ap.add_argument("--lams", default="0.3,1,2,3,5,10,20", help="PDHG lambda grid (tuned on held-out phantoms)")
    ap.add_argument("--init", default=None, help="start from these parameters (.npy)")
    ap.add_argument("--pdhg-iters", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained parameters (.npy)")
    ap.add_argument("--time-train", action="store_true",
                    help="only time one training step and one inference pass per volume (no data sets)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--profile", action="store_true",
                    help="only run 2 warm-up passes, then one inference and one training step on one phantom "
                         "(a short command for profilers)")
    args = ap.parse_args(argv)
    if args.profile:
        return profile_pass(args)
    if args.time_train:
        return time_training(args)

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
    lams = [float(v) for v in args.lams.split(",")]
    best = None
    for lam in lams:
        ps = [psnr(ops.pdhg(geom, y, x0, args.pdhg_iters, lam, gam, sig, tau)[0], x, full) for x, y, x0 in tune]
        m = float(np.mean(ps))
        print(f"pdhg lambda {lam:g}: tune PSNR {m:.2f}", file=sys.stderr, flush=True)
        if best is None or m > best[1]:
            best = (lam, m)
    lam = best[0]
    log["pdhg"] = {"lambda": lam, "iters": args.pdhg_iters, "sigma": sig, "tau": tau, "gamma": gam,
                   "grid": lams, "best_is_grid_edge": lam in (lams[0], lams[-1])}

    # ---- train the learned primal-dual network
    vb = max(1, min(args.vol_batch, args.batch))
    if args.batch % vb:
        raise SystemExit("--batch must be a multiple of --vol-batch")
    model = LPD(geom, n_iter=args.n_iter, n_mem=args.n_mem, width=args.width, seed=1,
                residual_input=args.residual_input, max_batch=vb, reversible=args.reversible, lire=args.lire,
                p4=args.p4, unet=args.unet, weight_norm=args.weight_norm)
    if args.init:
        model.set_params(widen_params(np.load(args.init), args.n_iter, model.n_mem, model.width,
                                      args.residual_input))
    Vb = V.expand((vb,) + tuple(V.shape)).contiguous()
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
            idx = perm[b0:b0 + args.batch]
            for c0 in range(0, len(idx), vb):
                items = [train[j] for j in idx[c0:c0 + vb]]
                x = torch.stack([t[0] for t in items])
                y = torch.stack([t[1] for t in items])
                x0 = torch.stack([t[2] for t in items])
                out = model.forward(y, x0, save_for_backward=True)
                loss, gr = masked_mse(out, x, Vb, 0.5)     # mean over the vb volumes' FoV voxels
                model.backward(gr)
                tot += loss.item() * vb
            # loss in units of mu_ref^2 (O(1)); linear warm-up, then cosine decay over the
            # number of steps the time budget allows (estimated after the warm-up)
            if step == args.warmup and step > 0:
                est_steps = max(step + 1, int(args.minutes * 60 / ((time.time() - t_train) / step)))
            if step < args.warmup:
                lr = args.lr * (step + 1) / max(1, args.warmup)
            else:
                lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * min(1.0, (step - args.warmup) /
                                                                   max(1, est_steps - args.warmup))))
            gscale = vb / (args.batch * model.mu_ref ** 2)
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
        meta = {"n_iter": args.n_iter, "n_mem": model.n_mem, "width": model.width, "mu_ref": model.mu_ref,
                "residual_input": bool(args.residual_input), "reversible": model.reversible, "lire": model.lire,
                "p4": model.p4, "pdhg_lambda": lam, "workload": WORKLOAD, "file": os.path.basename(args.save),
                "train_phantoms": args.train, "train_seconds": time.time() - t_train, "adam_steps": step}
        if model.reversible:
            meta["perms"] = model.perms().tolist()
        with open(os.path.splitext(args.save)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1)
    log["training"] = {"steps": step, "effective_batch": args.batch, "lr": args.lr, "warmup": args.warmup,
                       "clip": args.clip, "grad_norm_median": float(np.median(norms)) if norms else None,
                       "seconds": time.time() - t_train, "loss_first": losses[0] if losses else None,
                       "loss_last8": float(np.mean(losses[-8:])) if losses else None}

    # ---- evaluate at equal PSNR on the test phantoms (inference one volume at a time)
    model1 = LPD(geom, n_iter=args.n_iter, n_mem=args.n_mem, width=args.width, seed=1,
                 residual_input=args.residual_input, reversible=args.reversible, lire=args.lire, p4=args.p4,
                 unet=args.unet, weight_norm=args.weight_norm)
    model1.set_params(model.get_params())
    if model.reversible:
        model1.set_perms(model.perms())
    log["eval"] = equal_psnr(geom, model1, test, full, lam, gam, sig, tau)
    print(json.dumps(log), flush=True)
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "w") as f:
            json.dump(log, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())

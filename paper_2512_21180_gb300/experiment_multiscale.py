"""Multiscale learned primal-dual at clinical size: timing of inference and of one
training step (the multiscale workload).

Coarse level 128x128x96 at 4 mm (every second of 400 angles, 256x192 binned panel)
feeding the fine level 256x256x192 at 2 mm (400 angles, 512x384 at 0.8 mm, +160 mm
offset); a batch of 4 seeded phantoms simulated with Poisson noise at I0 = 5e4;
8 unrolled iterations per level, BF16 tensor-core blocks, activations recomputed in
the backward pass. Prints one JSON line.

    python -m paper_2512_21180_gb300.experiment_multiscale [--batch 4] [--n-iter 8] [--reps 2]

Everything runs in libcbct; PyTorch holds the buffers.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import torch

from . import inputs as I
from . import ops
from .lpd import masked_mse
from .multiscale import MultiscaleLPD, vol_down

WORKLOAD = "clinical"
I0 = 5e4


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--n-iter", type=int, default=8)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    g = I.geometry(WORKLOAD)
    model = MultiscaleLPD(g, n_iter=(args.n_iter, args.n_iter), seed=1)
    gf = model.geom_fine
    V = ops.fov(gf)
    Vc = ops.fov(model.geom_coarse)
    t0 = time.time()
    data = []
    for b in range(args.batch):
        x = ops.phantom(gf, I.phantom_params(WORKLOAD, 40_000 + b))
        _, y = ops.simulate(gf, x, I0, seed=b)
        x0 = ops.fdk(gf, y)[0]
        data.append((x, y[0], x0))
    torch.cuda.synchronize()
    prep_s = time.time() - t0
    st = torch.cuda.current_stream()

    def infer():
        return [model.forward(y, x0)[0] for _, y, x0 in data]

    def train_step():
        model.zero_grad()
        tot = 0.0
        for x, y, x0 in data:
            out, outc = model.forward(y, x0, save_for_backward=True)
            loss, gr = masked_mse(out, x, V, 0.5)
            lossc, grc = masked_mse(outc, vol_down(x), Vc, 0.5)
            model.backward(gr, grc)
            tot += loss.item()
        model.adam_step(1e-4, grad_scale=1.0 / (len(data) * 0.02 ** 2))
        return tot / len(data)

    res = {"workload": "multiscale: coarse 128x128x96 at 4 mm (200 angles, 256x192) -> fine 256x256x192 at 2 mm "
                       "(400 angles, 512x384 at 0.8 mm, +160 mm offset); Poisson I0=5e4; "
                       f"{args.n_iter}+{args.n_iter} iterations, width 32",
           "batch": args.batch, "data_prep_s": prep_s}
    for name, fn in (("inference", infer), ("training_step", train_step)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        res[name + "_s_per_batch"] = e0.elapsed_time(e1) / args.reps / 1e3
    res["inference_s_per_volume"] = res["inference_s_per_batch"] / args.batch
    free, total = torch.cuda.mem_get_info()
    res["device_gb_in_use"] = (total - free) / 1e9   # library workspaces included
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

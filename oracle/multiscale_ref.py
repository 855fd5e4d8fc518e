"""FP64 reference of the multiscale scheme (test infrastructure only).

The paper's multiscale reconstruction (Sec. 2.6) runs a coarse level on
half-resolution data first and carries its result to the fine level. Written out
from the definitions, in NumPy / PyTorch float64:
  * coarse volume grid: voxels twice as large, half as many per axis (same centre);
  * coarse data: every second angle, each coarse pixel the mean of a 2 x 2 block;
  * volume pooling: mean over 2 x 2 x 2 blocks;
  * upsampling: nearest neighbour (each coarse value copied to its 2 x 2 x 2 children);
  * two-level learned primal-dual: coarse LPD from the pooled start, its final primal
    and dual memory states upsampled as the fine level's initial states.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lpd_ref


def coarse_geometry(g: dict) -> dict:
    h = dict(g)
    h["n"] = tuple(n // 2 for n in g["n"])
    h["vox"] = tuple(2.0 * v for v in g["vox"])
    h["nu"], h["nv"] = g["nu"] // 2, g["nv"] // 2
    h["du"], h["dv"] = 2.0 * g["du"], 2.0 * g["dv"]
    h["n_angles"] = g["n_angles"] // 2
    return h


def vol_down(x):
    """Mean over 2 x 2 x 2 blocks of the last three axes."""
    a, b, c = x.shape[-3:]
    return x.reshape(x.shape[:-3] + (a // 2, 2, b // 2, 2, c // 2, 2)).mean(axis=(-5, -3, -1))


def proj_down(y):
    """Every second angle (axis -3), mean over 2 x 2 pixel blocks."""
    y = y[..., ::2, :, :]
    a, b, c = y.shape[-3:]
    return y.reshape(y.shape[:-3] + (a, b // 2, 2, c // 2, 2)).mean(axis=(-3, -1))


def up(x):
    """Nearest-neighbour 2x upsampling of the last three axes."""
    for ax in (-3, -2, -1):
        x = np.repeat(x, 2, axis=ax) if isinstance(x, np.ndarray) else torch.repeat_interleave(x, 2, dim=ax)
    return x


def lpd_multiscale(Gc, Gf, y: torch.Tensor, x0: torch.Tensor, wc: torch.Tensor, wf: torch.Tensor,
                   params_c, params_f, n_mem: int = 5, mu_ref: float = 1.0, bp_c: float = 1.0, bp_f: float = 1.0,
                   round_grads: bool = False):
    """(fine output, coarse output). params_* = (dual_params, primal_params) of each level;
    round_grads as in lpd_ref.lpd."""
    yc = proj_down(y)
    xc, fc, hc = lpd_ref.lpd(Gc, yc, vol_down(x0), wc, params_c[0], params_c[1], n_mem=n_mem, mu_ref=mu_ref,
                             bp_scale=bp_c, return_state=True, round_grads=round_grads)
    x = lpd_ref.lpd(Gf, y, None, wf, params_f[0], params_f[1], n_mem=n_mem, mu_ref=mu_ref, bp_scale=bp_f,
                    f0=up(fc), h0=up(hc), round_grads=round_grads)
    return x, xc

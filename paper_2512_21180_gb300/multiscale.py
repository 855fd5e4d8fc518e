"""Multiscale learned primal-dual (the multiscale scheme of Sec. 2.6): a coarse level at
half resolution — voxels twice as large, every second angle, 2 x 2 binned detector
pixels — runs first, and its primal and dual memory states, upsampled by nearest
neighbour, initialise the fine level. Gradients flow back through the adjoint of the
upsampling (box sums). Every step runs in libcbct; this module only wires the calls.
"""
from __future__ import annotations

import torch

from . import ops
from .lpd import LPD
from .projector import Geometry


def coarse_geometry(g: dict) -> dict:
    """The half-resolution level of a geometry dict (all of n, nu, nv, n_angles even)."""
    for k in ("nu", "nv", "n_angles"):
        if g[k] % 2:
            raise ValueError(f"{k} must be even for a coarse level")
    if any(n % 2 for n in g["n"]):
        raise ValueError("volume sizes must be even for a coarse level")
    h = dict(g)
    h["n"] = tuple(n // 2 for n in g["n"])
    h["vox"] = tuple(2.0 * v for v in g["vox"])
    h["nu"], h["nv"] = g["nu"] // 2, g["nv"] // 2
    h["du"], h["dv"] = 2.0 * g["du"], 2.0 * g["dv"]
    h["n_angles"] = g["n_angles"] // 2
    return h


def proj_down(y: torch.Tensor) -> torch.Tensor:
    """Coarse-level data: every second angle, 2 x 2 pixel means ([.., A, V, U])."""
    return ops.resample_down(y, (2, 2, 2), pick0=True, scale=0.25)


def vol_down(x: torch.Tensor) -> torch.Tensor:
    """2 x 2 x 2 average pooling ([.., Z, Y, X])."""
    return ops.resample_down(x, (2, 2, 2))


def up(x: torch.Tensor) -> torch.Tensor:
    """Nearest-neighbour 2x upsampling of the last three axes (volumes and projections)."""
    return ops.resample_up(x, (2, 2, 2))


def up_adjoint(g: torch.Tensor) -> torch.Tensor:
    """Adjoint of `up`: sums over each 2 x 2 x 2 box."""
    return ops.resample_down(g, (2, 2, 2), scale=1.0)


class MultiscaleLPD:
    """Two-level learned primal-dual: coarse (half resolution) -> fine."""

    def __init__(self, g_fine: dict, n_iter=(8, 8), seed: int = 0, **kw):
        self.g_fine, self.g_coarse = dict(g_fine), coarse_geometry(g_fine)
        self.geom_fine, self.geom_coarse = Geometry(self.g_fine), Geometry(self.g_coarse)
        self.coarse = LPD(self.geom_coarse, n_iter=n_iter[0], seed=seed, **kw)
        self.fine = LPD(self.geom_fine, n_iter=n_iter[1], seed=seed + 1, **kw)

    def forward(self, y: torch.Tensor, x0: torch.Tensor, save_for_backward: bool = False):
        """(fine reconstruction, coarse reconstruction) from data y and the fine FDK start x0."""
        yc = proj_down(y.reshape(self.geom_fine.proj_shape))
        xc = self.coarse.forward_latent(yc, x0=vol_down(x0.reshape(self.geom_fine.vol_shape)),
                                        save_for_backward=save_for_backward)
        fc, hc = self.coarse.state()
        x = self.fine.forward_latent(y, f0=up(fc), h0=up(hc), save_for_backward=save_for_backward)
        return x, xc

    def backward(self, grad_x: torch.Tensor, grad_xc: torch.Tensor | None = None):
        """Accumulates both levels' parameter gradients (loss on the fine output and,
        optionally, on the coarse one)."""
        gf0, gh0 = self.fine.backward_latent(grad_x=grad_x)
        self.coarse.backward_latent(grad_x=grad_xc, grad_fN=up_adjoint(gf0), grad_hN=up_adjoint(gh0),
                                    want_states=False)

    def zero_grad(self):
        self.coarse.zero_grad()
        self.fine.zero_grad()

    def adam_step(self, lr: float, grad_scale: float = 1.0):
        self.coarse.adam_step(lr, grad_scale=grad_scale)
        self.fine.adam_step(lr, grad_scale=grad_scale)

"""Python binding of the learned primal-dual module (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import LpdDesc, check
from .projector import Geometry


def _st() -> int:
    return torch.cuda.current_stream().cuda_stream


class LPD:
    """Unrolled learned primal-dual network on the GPU (weights live in libcbct)."""

    def __init__(self, geom: Geometry, n_iter: int = 8, n_mem: int = 5, width: int = 32, slope: float = 0.2,
                 mu_ref: float = 0.02, bp_scale: float = 0.0, seed: int = 0, residual_input: bool = False,
                 max_batch: int = 1, reversible: bool = False, lire: bool = False, p4: bool = False,
                 unet: bool = False, weight_norm: bool = False):
        self.geom = geom
        d = LpdDesc(n_iter, n_mem, width, slope, mu_ref, bp_scale, seed, int(residual_input), int(max_batch),
                    int(reversible or lire), int(lire), int(p4 or unet), int(unet), int(weight_norm))
        h = ctypes.c_void_p()
        with torch.cuda.device(geom.device):
            check(_lib.load().lpd_create(geom.handle, ctypes.byref(d), ctypes.byref(h)), "lpd_create")
        self.handle = h
        self.n_iter, self.n_mem, self.width, self.mu_ref = n_iter, n_mem, width, mu_ref
        self.residual_input, self.max_batch = bool(residual_input), int(max_batch)
        self.reversible, self.lire, self.p4, self.unet = bool(reversible or lire), bool(lire), bool(p4 or unet), bool(unet)
        self.weight_norm = bool(weight_norm)
        self.batch = 1
        n = ctypes.c_longlong()
        pp, gp = ctypes.c_void_p(), ctypes.c_void_p()
        bs = ctypes.c_float()
        check(_lib.load().lpd_info(h, ctypes.byref(n), ctypes.byref(pp), ctypes.byref(gp), ctypes.byref(bs)),
              "lpd_info")
        self.nparams = int(n.value)
        self.bp_scale = float(bs.value)
        self.step = 0

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.load().lpd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters -----------------------------------------------------------------
    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        check(_lib.load().lpd_get_params(self.handle, out.ctypes.data, self.nparams), "lpd_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(_lib.load().lpd_set_params(self.handle, p.ctypes.data, self.nparams), "lpd_set_params")

    def perms(self) -> np.ndarray:
        """[n_iter, 2, n_mem] channel permutations of a reversible model (perm_f, perm_h)."""
        out = np.zeros((self.n_iter, 2, self.n_mem), dtype=np.int32)
        check(_lib.load().lpd_get_perms(self.handle, out.ctypes.data), "lpd_get_perms")
        return out

    def set_perms(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.int32).reshape(self.n_iter, 2, self.n_mem)
        check(_lib.load().lpd_set_perms(self.handle, p.ctypes.data), "lpd_set_perms")

    def device_status(self, clear: bool = False) -> int:
        """The model's device status word (0 = no convolution kernel gave up a bounded wait)."""
        out = ctypes.c_int(0)
        check(_lib.load().lpd_device_status(self.handle, ctypes.byref(out), int(clear)), "lpd_device_status")
        return int(out.value)

    def grads(self) -> np.ndarray:
        """Host copy of the accumulated parameter gradients."""
        out = np.zeros(self.nparams, dtype=np.float32)
        check(_lib.load().lpd_get_grads(self.handle, out.ctypes.data, self.nparams), "lpd_get_grads")
        return out

    # compute ----------------------------------------------------------------------
    def forward(self, y: torch.Tensor, x0: torch.Tensor, save_for_backward: bool = False) -> torch.Tensor:
        """y [na, nv, nu] and x0 [nz, ny, nx] (one volume), or [B, ...] each (a batch of
        B <= max_batch volumes, reconstructed together); the output has x0's shape."""
        g = self.geom
        batched = y.dim() == 4
        B = y.shape[0] if batched else 1
        yy = y.reshape((B,) + g.proj_shape).contiguous()
        xx = x0.reshape((B,) + g.vol_shape).contiguous()
        out = torch.empty((B,) + g.vol_shape, device=yy.device, dtype=torch.float32)
        check(_lib.load().lpd_forward(self.handle, yy.data_ptr(), xx.data_ptr(), out.data_ptr(), B,
                                      int(save_for_backward), _st()), "lpd_forward")
        self.batch = B
        return out if batched else out[0]

    def backward(self, grad_x: torch.Tensor, want_y: bool = False, want_x0: bool = False):
        """Gradients for the last forward pass (its batch); returns (dL/dy, dL/dx0) shaped
        like that pass's y and x0 (or None)."""
        g = self.geom
        B = self.batch
        gx = grad_x.reshape((B,) + g.vol_shape).contiguous()
        shp_p = ((B,) if grad_x.dim() == 4 else ()) + g.proj_shape
        shp_v = ((B,) if grad_x.dim() == 4 else ()) + g.vol_shape
        gy = torch.empty(shp_p, device=gx.device) if want_y else None
        g0 = torch.empty(shp_v, device=gx.device) if want_x0 else None
        check(_lib.load().lpd_backward(self.handle, gx.data_ptr(), None if gy is None else gy.data_ptr(),
                                       None if g0 is None else g0.data_ptr(), _st()), "lpd_backward")
        return gy, g0

    # latent states (multiscale levels) -------------------------------------------
    def forward_latent(self, y: torch.Tensor, x0: torch.Tensor | None = None, f0: torch.Tensor | None = None,
                       h0: torch.Tensor | None = None, save_for_backward: bool = False,
                       want_x: bool = True) -> torch.Tensor | None:
        """Forward from initial states f0 [n_mem, *vol] (units of mu_ref) and h0
        [n_mem, *proj]; either may be None (x0 / mu_ref repeated, zero)."""
        g = self.geom
        yy = y.reshape(g.proj_shape).contiguous()
        xx = None if x0 is None else x0.reshape(g.vol_shape).contiguous()
        ff = None if f0 is None else f0.reshape((self.n_mem,) + g.vol_shape).contiguous()
        hh = None if h0 is None else h0.reshape((self.n_mem,) + g.proj_shape).contiguous()
        out = torch.empty(g.vol_shape, device=yy.device) if want_x else None
        ptr = lambda t: None if t is None else t.data_ptr()
        check(_lib.load().lpd_forward_latent(self.handle, yy.data_ptr(), ptr(xx), ptr(ff), ptr(hh), ptr(out),
                                             int(save_for_backward), _st()), "lpd_forward_latent")
        self.batch = 1
        return out

    def state(self):
        """(f_N [n_mem, *vol], h_N [n_mem, *proj]) of the last forward pass."""
        g = self.geom
        f = torch.empty((self.n_mem,) + g.vol_shape, device="cuda")
        h = torch.empty((self.n_mem,) + g.proj_shape, device="cuda")
        check(_lib.load().lpd_get_state(self.handle, f.data_ptr(), h.data_ptr(), _st()), "lpd_get_state")
        return f, h

    def backward_latent(self, grad_x: torch.Tensor | None = None, grad_fN: torch.Tensor | None = None,
                        grad_hN: torch.Tensor | None = None, want_states: bool = True):
        """Accumulates parameter gradients; returns (dL/df_0, dL/dh_0) (or Nones)."""
        g = self.geom
        ptr = lambda t: None if t is None else t.contiguous().data_ptr()
        gf0 = torch.empty((self.n_mem,) + g.vol_shape, device="cuda") if want_states else None
        gh0 = torch.empty((self.n_mem,) + g.proj_shape, device="cuda") if want_states else None
        check(_lib.load().lpd_backward_latent(self.handle, ptr(grad_x), ptr(grad_fN), ptr(grad_hN), None, None,
                                              ptr(gf0), ptr(gh0), _st()), "lpd_backward_latent")
        return gf0, gh0

    def zero_grad(self):
        check(_lib.load().lpd_zero_grad(self.handle, _st()), "lpd_zero_grad")

    def clip_grads(self, max_norm: float, grad_scale: float = 1.0) -> float:
        """Scales the accumulated gradient so that ||grad_scale g|| <= max_norm (zero if
        the norm is not finite); returns the norm before clipping."""
        out = ctypes.c_double(0.0)
        check(_lib.load().lpd_clip_grads(self.handle, float(max_norm), float(grad_scale), ctypes.byref(out), _st()),
              "lpd_clip_grads")
        return float(out.value)

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  grad_scale: float = 1.0):
        self.step += 1
        check(_lib.load().lpd_adam_step(self.handle, lr, beta1, beta2, eps, self.step, grad_scale, _st()),
              "lpd_adam_step")


def masked_mse(x: torch.Tensor, ref: torch.Tensor, V: torch.Tensor | None = None, thr: float = 0.5,
               want_grad: bool = True):
    """(loss [device scalar], grad) of the mean squared error over V >= thr."""
    x = x.contiguous()
    ref = ref.contiguous()
    loss = torch.zeros(1, device=x.device)
    grad = torch.empty_like(x) if want_grad else None
    check(_lib.load().cbct_masked_mse(x.data_ptr(), ref.data_ptr(), None if V is None else V.contiguous().data_ptr(),
                                      float(thr), x.numel(), loss.data_ptr(),
                                      None if grad is None else grad.data_ptr(), _st()), "cbct_masked_mse")
    return loss, grad


def p4_primal_layout(cin: int, cout: int):
    """Base-parameter layout of one P4 primal block: ("lift", 8, cin), ("group", 8, 8),
    ("avg", cout, 8) — weights [8][27][cin], [8][4][27][8], [cout][4][27][8], each followed
    by its bias."""
    return [("lift", 8, cin), ("group", 8, 8), ("avg", cout, 8)]


UNET_F = 4  # base filters of the U-Net's full-resolution layers (4F group channels; 8F at half resolution)


def p4_unet_layout(cin: int, cout: int, f: int = UNET_F):
    """Base-parameter layout of one P4 U-Net primal block (six 3x3x3 layers): the lift
    ("lift", f, cin) with weights [f][27][cin], then group layers (co, ci) with weights
    [co][4][27][ci]: g2 (f, f), g3 (2f, f), g4 (2f, 2f), g5 (f, 3f) reading [up(r), s],
    and the averaged output layer (cout, f); each followed by its bias."""
    return [("lift", f, cin), ("group", f, f), ("group", 2 * f, f), ("group", 2 * f, 2 * f), ("group", f, 3 * f),
            ("avg", cout, f)]


def lire_layout(n_iter: int, n_mem: int = 8, width: int = 32):
    """Parameter layout of a LIRE-mode model, per iteration: ("conv", cout, 27, cin) for
    the three dual and three primal layers (weights [cout][27][cin] then bias), then
    ("out", n_mem) for the output convolution (omega [n_mem] then beta)."""
    k = n_mem // 2
    out = []
    for _ in range(n_iter):
        for _blk in range(2):
            out += [("conv", width, 27, k + 4), ("conv", width, 27, width), ("conv", k, 27, width)]
        out.append(("out", n_mem))
    return out


def layer_shapes(n_iter: int, n_mem: int = 5, width: int = 32, residual_input: bool = False,
                 reversible: bool = False):
    """[(cout, taps, cin)] in the library's parameter order (a reversible model's blocks
    read and write half of the n_mem channels)."""
    k = n_mem // 2 if reversible else n_mem
    out = []
    for _ in range(n_iter):
        out += [(width, 9, k + 2 + int(residual_input)), (width, 9, width), (k, 9, width),
                (width, 27, k + 1), (width, 27, width), (k, 27, width)]
    return out

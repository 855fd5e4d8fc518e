"""Python binding of the simulation and per-geometry calls (argument marshalling
only; the arithmetic runs in libcbct.so)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check
from .projector import Geometry


def _st(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def phantom(geom: Geometry, ell: np.ndarray, supersample: int = 1, out: torch.Tensor | None = None) -> torch.Tensor:
    """Voxelised ellipsoid phantom [nz, ny, nx] (float32, on the geometry's device)."""
    e = np.ascontiguousarray(ell, dtype=np.float64).reshape(-1, 17)
    if out is None:
        out = torch.empty(geom.vol_shape, device=geom.device, dtype=torch.float32)
    assert out.is_contiguous() and out.dtype == torch.float32 and out.numel() == int(np.prod(geom.vol_shape))
    with torch.cuda.device(geom.device):
        check(_lib.load().cbct_phantom(geom.handle, e.ctypes.data, e.shape[0], supersample, out.data_ptr(), _st(out)),
              "cbct_phantom")
    return out


def poisson(line_integrals: torch.Tensor, I0: float, seed: int) -> torch.Tensor:
    p = line_integrals.contiguous()
    assert p.dtype == torch.float32 and p.is_cuda
    out = torch.empty(p.shape, dtype=torch.int32, device=p.device)
    with torch.cuda.device(p.device):
        check(_lib.load().cbct_poisson(p.data_ptr(), p.numel(), float(I0), int(seed), out.data_ptr(), _st(p)),
              "cbct_poisson")
    return out


def neglog(counts: torch.Tensor, I0: float) -> torch.Tensor:
    c = counts.contiguous()
    assert c.dtype == torch.int32 and c.is_cuda
    out = torch.empty(c.shape, dtype=torch.float32, device=c.device)
    with torch.cuda.device(c.device):
        check(_lib.load().cbct_neglog(c.data_ptr(), c.numel(), float(I0), out.data_ptr(), _st(c)), "cbct_neglog")
    return out


def simulate(geom: Geometry, vol: torch.Tensor, I0: float, seed: int):
    """(line integrals P vol, noisy log data y) for a batch of volumes."""
    v = vol.contiguous()
    if v.dim() == 3:
        v = v.unsqueeze(0)
    B = v.shape[0]
    p = torch.empty((B,) + geom.proj_shape, device=v.device, dtype=torch.float32)
    y = torch.empty_like(p)
    with torch.cuda.device(v.device):
        check(_lib.load().cbct_simulate(geom.handle, v.data_ptr(), B, float(I0), int(seed), p.data_ptr(),
                                        y.data_ptr(), _st(v)), "cbct_simulate")
    return p, y


def _f64(a):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def detector_response(energies_kev) -> np.ndarray:
    """resp(e) of the polychromatic model (host only)."""
    E, pE = _f64(energies_kev)
    out = np.zeros(len(E))
    check(_lib.load().cbct_detector_response(pE, len(E), out.ctypes.data_as(ctypes.c_void_p)),
          "cbct_detector_response")
    return out


def water_bone(mu: torch.Tensor, mu_water60: float) -> torch.Tensor:
    """rho[batch][2][...] (water, bone) of mu_60 volumes mu[batch][...] (a 3-D
    volume is one item)."""
    v = mu.contiguous()
    assert v.dtype == torch.float32 and v.is_cuda
    if v.dim() == 3:
        v = v.unsqueeze(0)
    B = v.shape[0]
    out = torch.empty((B, 2) + tuple(v.shape[1:]), dtype=torch.float32, device=v.device)
    with torch.cuda.device(v.device):
        check(_lib.load().cbct_water_bone(v.data_ptr(), v[0].numel(), B, float(mu_water60), out.data_ptr(), _st(v)),
              "cbct_water_bone")
    return out


def poly_reading(line_integrals: torch.Tensor, I0: torch.Tensor, energies_kev, mu_water, mu_bone, seed: int,
                 noise: bool = True, want_counts: bool = False):
    """(reading, y, counts or None) from water / bone line integrals
    [batch][2][n_angles][nv][nu] and intensity maps I0[n_e][nv][nu]."""
    L = line_integrals.contiguous()
    i0 = I0.contiguous()
    assert L.dtype == torch.float32 and i0.dtype == torch.float32 and L.is_cuda and i0.is_cuda
    assert L.dim() == 5 and L.shape[1] == 2
    B = L.shape[0]
    E, pE = _f64(energies_kev)
    mw, pW = _f64(mu_water)
    mb, pB = _f64(mu_bone)
    ne = len(E)
    assert len(mw) == ne and len(mb) == ne and i0.shape[0] == ne
    per_item = L[0, 0].numel()
    npix = L.shape[-1] * L.shape[-2]
    assert i0.numel() == ne * npix, "I0 must be [n_e][nv][nu]"
    reading = torch.empty((B,) + tuple(L.shape[2:]), dtype=torch.float32, device=L.device)
    y = torch.empty_like(reading)
    counts = (torch.empty((B,) + tuple(L.shape[2:]) + (ne,), dtype=torch.int32, device=L.device)
              if want_counts else None)
    with torch.cuda.device(L.device):
        check(_lib.load().cbct_poly_reading(L.data_ptr(), B, per_item, npix, ne, pE, pW, pB, i0.data_ptr(),
                                            int(seed), 1 if noise else 0, reading.data_ptr(), y.data_ptr(),
                                            counts.data_ptr() if counts is not None else None, _st(L)),
              "cbct_poly_reading")
    return reading, y, counts


def poly_simulate(geom: Geometry, mu: torch.Tensor, I0: torch.Tensor, energies_kev, mu_water, mu_bone,
                  mu_water60: float, seed: int, noise: bool = True):
    """(water / bone line integrals [batch][2][...], normalised polychromatic data
    y [batch][n_angles][nv][nu]) for a batch of mu_60 volumes."""
    v = mu.contiguous()
    i0 = I0.contiguous()
    if v.dim() == 3:
        v = v.unsqueeze(0)
    assert v.dtype == torch.float32 and i0.dtype == torch.float32 and v.is_cuda and i0.is_cuda
    B = v.shape[0]
    E, pE = _f64(energies_kev)
    mw, pW = _f64(mu_water)
    mb, pB = _f64(mu_bone)
    assert len(mw) == len(E) and len(mb) == len(E) and i0.numel() == len(E) * geom.nv * geom.nu, \
        "tables of n_e entries and I0 [n_e][nv][nu]"
    L = torch.empty((B, 2) + geom.proj_shape, device=v.device, dtype=torch.float32)
    y = torch.empty((B,) + geom.proj_shape, device=v.device, dtype=torch.float32)
    with torch.cuda.device(v.device):
        check(_lib.load().cbct_poly_simulate(geom.handle, v.data_ptr(), B, float(mu_water60), len(E), pE, pW, pB,
                                             i0.data_ptr(), int(seed), 1 if noise else 0, L.data_ptr(),
                                             y.data_ptr(), _st(v)), "cbct_poly_simulate")
    return L, y


def redundancy_weight(geom: Geometry) -> torch.Tensor:
    w = torch.empty(geom.nu, device=geom.device, dtype=torch.float32)
    with torch.cuda.device(geom.device):
        check(_lib.load().cbct_redundancy_weight(geom.handle, w.data_ptr(), _st(w)), "cbct_redundancy_weight")
    return w


def fov(geom: Geometry) -> torch.Tensor:
    V = torch.empty(geom.vol_shape, device=geom.device, dtype=torch.float32)
    with torch.cuda.device(geom.device):
        check(_lib.load().cbct_fov(geom.handle, V.data_ptr(), _st(V)), "cbct_fov")
    return V


def _b(t: torch.Tensor, shape):
    t = t.contiguous()
    if t.dim() == len(shape):
        t = t.unsqueeze(0)
    assert tuple(t.shape[1:]) == tuple(shape) and t.dtype == torch.float32 and t.is_cuda
    return t


def fdk(geom: Geometry, proj: torch.Tensor) -> torch.Tensor:
    """FDK_w reconstruction of [B, na, nv, nu] projections -> [B, nz, ny, nx]."""
    p = _b(proj, geom.proj_shape)
    out = torch.empty((p.shape[0],) + geom.vol_shape, device=p.device, dtype=torch.float32)
    with torch.cuda.device(p.device):
        check(_lib.load().cbct_fdk(geom.handle, p.data_ptr(), out.data_ptr(), p.shape[0], 0, _st(p)), "cbct_fdk")
    return out


def opnorm(geom: Geometry, gamma: float = 0.0, iters: int = 30) -> float:
    import ctypes
    out = ctypes.c_double(0.0)
    with torch.cuda.device(geom.device):
        check(_lib.load().cbct_opnorm(geom.handle, float(gamma), int(iters), ctypes.byref(out),
                                      torch.cuda.current_stream().cuda_stream), "cbct_opnorm")
    return out.value


def pdhg(geom: Geometry, y: torch.Tensor, x0: torch.Tensor, niter: int, lam: float, gamma: float, sigma: float,
         tau: float, nonneg: bool = True) -> torch.Tensor:
    yy = _b(y, geom.proj_shape)
    xx = _b(x0, geom.vol_shape)
    out = torch.empty_like(xx)
    with torch.cuda.device(yy.device):
        check(_lib.load().cbct_pdhg(geom.handle, yy.data_ptr(), xx.data_ptr(), out.data_ptr(), yy.shape[0], int(niter),
                                    float(lam), float(gamma), float(sigma), float(tau), int(nonneg), _st(yy)),
              "cbct_pdhg")
    return out


def landweber(geom: Geometry, y: torch.Tensor, x: torch.Tensor, niter: int, tau: float,
              nonneg: bool = False) -> torch.Tensor:
    yy = _b(y, geom.proj_shape)
    xx = _b(x, geom.vol_shape).clone()
    with torch.cuda.device(yy.device):
        check(_lib.load().cbct_landweber(geom.handle, yy.data_ptr(), xx.data_ptr(), yy.shape[0], int(niter),
                                         float(tau), int(nonneg), _st(yy)), "cbct_landweber")
    return xx


# ---- resampling between multiscale levels (a11) ----------------------------------------

def resample_down(x: torch.Tensor, f=(2, 2, 2), pick0: bool = False, scale: float | None = None) -> torch.Tensor:
    """Box sum over f (or, with pick0, every f0-th slice along the first axis) of the last
    three axes, times scale (default: the mean over the box)."""
    x = x.contiguous()
    n0, n1, n2 = x.shape[-3:]
    nch = x.numel() // (n0 * n1 * n2)
    if scale is None:
        scale = 1.0 / ((1 if pick0 else f[0]) * f[1] * f[2])
    out = torch.empty(x.shape[:-3] + (n0 // f[0], n1 // f[1], n2 // f[2]), device=x.device)
    _lib.check(_lib.load().cbct_resample_down(x.data_ptr(), nch, n0, n1, n2, f[0], f[1], f[2], int(pick0),
                                              float(scale), out.data_ptr(), _st(x)), "cbct_resample_down")
    return out


def resample_up(x: torch.Tensor, f=(2, 2, 2)) -> torch.Tensor:
    """Nearest-neighbour upsampling of the last three axes by f."""
    x = x.contiguous()
    n0, n1, n2 = x.shape[-3:]
    nch = x.numel() // (n0 * n1 * n2)
    out = torch.empty(x.shape[:-3] + (n0 * f[0], n1 * f[1], n2 * f[2]), device=x.device)
    _lib.check(_lib.load().cbct_resample_up(x.data_ptr(), nch, n0, n1, n2, f[0], f[1], f[2], out.data_ptr(),
                                            _st(x)), "cbct_resample_up")
    return out

"""Python binding of the projector pair: geometry handle, the two operators and
their autograd wrappers (a torch.autograd.Function whose backward is the other
operator). Argument marshalling only: all arithmetic runs in libcbct.so.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import GeomDesc, check


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class Geometry:
    """Owns a `cbct_geom` handle (per-angle ray tables on one CUDA device).

    `g` is a geometry dict as produced by `inputs.geometry` (keys n, vox, center,
    nu, nv, du, dv, u_offset, v_offset, sid, sdd, n_angles)."""

    def __init__(self, g: dict, angles=None, normalize: bool = False, device=None):
        self.g = dict(g)
        self.n = tuple(int(v) for v in g["n"])
        self.nu, self.nv, self.na = int(g["nu"]), int(g["nv"]), int(g["n_angles"])
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        lib = _lib.load()
        self._angles = None
        if angles is not None:
            import numpy as np
            self._angles = np.ascontiguousarray(angles, dtype=np.float64)
            assert self._angles.shape == (self.na,)
        d = GeomDesc()
        d.nx, d.ny, d.nz = self.n
        d.vox = (ctypes.c_double * 3)(*[float(v) for v in g["vox"]])
        d.center = (ctypes.c_double * 3)(*[float(v) for v in g.get("center", (0, 0, 0))])
        d.nu, d.nv = self.nu, self.nv
        d.du, d.dv = float(g["du"]), float(g["dv"])
        d.u_offset, d.v_offset = float(g["u_offset"]), float(g.get("v_offset", 0.0))
        d.sid, d.sdd = float(g["sid"]), float(g["sdd"])
        d.n_angles = self.na
        d.angles = None if self._angles is None else self._angles.ctypes.data
        d.normalize = 1 if normalize else 0
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.geometry_create(ctypes.byref(d), ctypes.byref(h)), "geometry_create")
        self.handle = h
        self.scale = lib.geometry_scale(h)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            with torch.cuda.device(self.device):
                _lib.load().geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def vol_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def proj_shape(self):
        return (self.na, self.nv, self.nu)

    def device_status(self, clear: bool = False) -> int:
        """The geometry's device status word (0 = no kernel gave up a bounded wait)."""
        out = ctypes.c_int(0)
        with torch.cuda.device(self.device):
            check(_lib.load().cbct_device_status(self.handle, ctypes.byref(out), int(clear)), "device_status")
        return int(out.value)

    def count_samples(self) -> int:
        out = ctypes.c_longlong(0)
        with torch.cuda.device(self.device):
            check(_lib.load().cbct_count_samples(self.handle, ctypes.byref(out),
                                                 torch.cuda.current_stream().cuda_stream), "count_samples")
        return int(out.value)


def _batched(t: torch.Tensor, shape, what: str):
    if t.dim() == len(shape):
        t = t.unsqueeze(0)
    if tuple(t.shape[1:]) != tuple(shape):
        raise ValueError(f"{what}: expected [B, {', '.join(map(str, shape))}], got {tuple(t.shape)}")
    if not t.is_cuda:
        raise ValueError(f"{what}: tensor must live on a CUDA device")
    if t.dtype not in (torch.float32, torch.float64):
        raise ValueError(f"{what}: dtype must be float32 or float64")
    return t.contiguous()


def forward_project(geom: Geometry, vol: torch.Tensor, out: torch.Tensor | None = None,
                    accumulate: bool = False) -> torch.Tensor:
    """proj = P vol (or proj += P vol); vol [B, nz, ny, nx] -> proj [B, na, nv, nu]."""
    squeeze = vol.dim() == 3
    v = _batched(vol, geom.vol_shape, "forward_project")
    B = v.shape[0]
    if out is None:
        out = torch.empty((B,) + geom.proj_shape, device=v.device, dtype=v.dtype)
        accumulate = False
    o = out if out.dim() == 4 else out.unsqueeze(0)
    assert o.is_contiguous() and o.dtype == v.dtype and tuple(o.shape) == (B,) + geom.proj_shape
    lib = _lib.load()
    fn = lib.forward_project if v.dtype == torch.float32 else lib.forward_project_f64
    with torch.cuda.device(v.device):
        check(fn(geom.handle, _ptr(v), _ptr(o), B, int(accumulate), _stream(v)), "forward_project")
    return out[0] if (squeeze and out.dim() == 4) else out


def back_project(geom: Geometry, proj: torch.Tensor, out: torch.Tensor | None = None,
                 accumulate: bool = False) -> torch.Tensor:
    """vol = P* proj (or vol += P* proj); proj [B, na, nv, nu] -> vol [B, nz, ny, nx]."""
    squeeze = proj.dim() == 3
    p = _batched(proj, geom.proj_shape, "back_project")
    B = p.shape[0]
    if out is None:
        out = torch.empty((B,) + geom.vol_shape, device=p.device, dtype=p.dtype)
        accumulate = False
    o = out if out.dim() == 4 else out.unsqueeze(0)
    assert o.is_contiguous() and o.dtype == p.dtype and tuple(o.shape) == (B,) + geom.vol_shape
    lib = _lib.load()
    fn = lib.back_project if p.dtype == torch.float32 else lib.back_project_f64
    with torch.cuda.device(p.device):
        check(fn(geom.handle, _ptr(p), _ptr(o), B, int(accumulate), _stream(p)), "back_project")
    return out[0] if (squeeze and out.dim() == 4) else out


class Project(torch.autograd.Function):
    """y = P x; the gradient of a loss L(y) w.r.t. x is P* dL/dy (a4)."""

    @staticmethod
    def forward(ctx, geom: Geometry, vol: torch.Tensor):
        ctx.geom = geom
        return forward_project(geom, vol)

    @staticmethod
    def backward(ctx, g):
        return None, back_project(ctx.geom, g.contiguous())


class BackProject(torch.autograd.Function):
    """x = P* y; the gradient w.r.t. y is P dL/dx (a4)."""

    @staticmethod
    def forward(ctx, geom: Geometry, proj: torch.Tensor):
        ctx.geom = geom
        return back_project(geom, proj)

    @staticmethod
    def backward(ctx, g):
        return None, forward_project(ctx.geom, g.contiguous())


def project(geom: Geometry, vol: torch.Tensor) -> torch.Tensor:
    return Project.apply(geom, vol)


def backproject(geom: Geometry, proj: torch.Tensor) -> torch.Tensor:
    return BackProject.apply(geom, proj)

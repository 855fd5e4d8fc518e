"""FP64 CPU oracle (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package. It is an independent, plain restatement of what the
GPU library computes; it never imports or links the GPU library.

The C part (`oracle.c`) holds the projector pair, geometry, field-of-view
tensor, redundancy weight, FDK, PDHG-TV, Philox/Poisson simulation, phantom
voxeliser and the polychromatic primary (water-bone split, detector response,
resp-weighted per-energy draws); `lpd_ref.py` holds the learned primal-dual reference in plain
PyTorch CPU FP64 and `multiscale_ref.py` the two-level scheme built on it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no FP contraction) into liboracle.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_long, ctypes.c_double
            sig = {
                "o_frame": (None, [P, P, P, i32, P]),
                "o_principal_axis": (i32, [P, P, P, i32, i32, i32]),
                "o_forward": (None, [P, P, P, P, P, P]),
                "o_forward_rays": (None, [P, P, P, P, P, i64, P]),
                "o_adjoint": (None, [P, P, P, P, P]),
                "o_adjoint_voxels": (None, [P, P, P, P, P, i64, P]),
                "o_fov": (None, [P, P, P, P]),
                "o_redundancy": (None, [P, P, P]),
                "o_fdk": (None, [P, P, P, P, P]),
                "o_grad": (None, [P, P, P]),
                "o_div": (None, [P, P, P]),
                "o_pdhg": (None, [P, P, P, P, P, i32, f64, f64, f64, f64, P]),
                "o_fdk_pad": (i32, [P, P]),
                "o_philox": (None, [P, P, P]),
                "o_poisson": (None, [P, i64, f64, ctypes.c_uint64, P]),
                "o_poisson_lam": (None, [P, i64, ctypes.c_uint64, P]),
                "o_neglog": (None, [P, i64, f64, P]),
                "o_phantom": (None, [P, P, P, i32, i32, P]),
                "o_num_threads": (i32, []),
                "o_water_bone": (None, [P, i64, f64, P, P]),
                "o_resp": (f64, [f64]),
                "o_poly_lam": (None, [P, P, i64, i64, i32, P, P, P, P]),
                "o_poly_reading": (None, [P, i64, i32, P, ctypes.c_uint64, i32, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Geom:
    """Geometry description for the oracle (mm, radians)."""

    def __init__(self, g: dict, angles=None):
        self.g = dict(g)
        self.n = tuple(int(v) for v in g["n"])
        self.nu, self.nv, self.na = int(g["nu"]), int(g["nv"]), int(g["n_angles"])
        self.dims = np.array([*self.n, self.nu, self.nv, self.na], dtype=np.int32)
        self.par = np.array([*g["vox"], *g["center"], g["du"], g["dv"], g["u_offset"],
                             g.get("v_offset", 0.0), g["sid"], g["sdd"]], dtype=np.float64)
        self.angles = None if angles is None else np.ascontiguousarray(angles, dtype=np.float64)

    @property
    def vol_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def proj_shape(self):
        return (self.na, self.nv, self.nu)

    def _a(self):
        return None if self.angles is None else _ptr(self.angles)


def frame(G: Geom, k: int) -> np.ndarray:
    out = np.zeros(12)
    lib().o_frame(_ptr(G.dims), _ptr(G.par), G._a(), k, _ptr(out))
    return out


def principal_axis(G: Geom, k: int, iu: int, iv: int) -> int:
    return lib().o_principal_axis(_ptr(G.dims), _ptr(G.par), G._a(), k, iu, iv)


def forward(G: Geom, vol: np.ndarray, return_count: bool = False):
    vol = np.ascontiguousarray(vol, dtype=np.float64).reshape(G.vol_shape)
    proj = np.zeros(G.proj_shape)
    cnt = ctypes.c_long(0)
    lib().o_forward(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(vol), _ptr(proj), ctypes.byref(cnt))
    return (proj, cnt.value) if return_count else proj


def forward_rays(G: Geom, vol: np.ndarray, ray_ids) -> np.ndarray:
    vol = np.ascontiguousarray(vol, dtype=np.float64).reshape(G.vol_shape)
    ids = np.ascontiguousarray(ray_ids, dtype=np.int64)
    out = np.zeros(len(ids))
    lib().o_forward_rays(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(vol), _ptr(ids), len(ids), _ptr(out))
    return out


def adjoint(G: Geom, proj: np.ndarray) -> np.ndarray:
    proj = np.ascontiguousarray(proj, dtype=np.float64).reshape(G.proj_shape)
    vol = np.zeros(G.vol_shape)
    lib().o_adjoint(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(proj), _ptr(vol))
    return vol


def adjoint_voxels(G: Geom, proj: np.ndarray, vox_ids) -> np.ndarray:
    proj = np.ascontiguousarray(proj, dtype=np.float64).reshape(G.proj_shape)
    ids = np.ascontiguousarray(vox_ids, dtype=np.int64)
    out = np.zeros(len(ids))
    lib().o_adjoint_voxels(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(proj), _ptr(ids), len(ids), _ptr(out))
    return out


def fov(G: Geom) -> np.ndarray:
    V = np.zeros(G.vol_shape)
    lib().o_fov(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(V))
    return V


def redundancy(G: Geom) -> np.ndarray:
    w = np.zeros(G.nu)
    lib().o_redundancy(_ptr(G.dims), _ptr(G.par), _ptr(w))
    return w


def fdk_pad(G: Geom) -> int:
    return lib().o_fdk_pad(_ptr(G.dims), _ptr(G.par))


def fdk(G: Geom, proj: np.ndarray) -> np.ndarray:
    proj = np.ascontiguousarray(proj, dtype=np.float64).reshape(G.proj_shape)
    vol = np.zeros(G.vol_shape)
    lib().o_fdk(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(proj), _ptr(vol))
    return vol


def grad(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.array([x.shape[2], x.shape[1], x.shape[0]], dtype=np.int32)
    g3 = np.zeros((3,) + x.shape)
    lib().o_grad(_ptr(n), _ptr(x), _ptr(g3))
    return g3


def div(g3: np.ndarray) -> np.ndarray:
    g3 = np.ascontiguousarray(g3, dtype=np.float64)
    n = np.array([g3.shape[3], g3.shape[2], g3.shape[1]], dtype=np.int32)
    d = np.zeros(g3.shape[1:])
    lib().o_div(_ptr(n), _ptr(g3), _ptr(d))
    return d


def pdhg(G: Geom, y: np.ndarray, x0: np.ndarray, niter: int, lam: float, sigma: float,
         tau: float, gamma: float = 1.0) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(G.proj_shape)
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(G.vol_shape)
    x = np.zeros(G.vol_shape)
    lib().o_pdhg(_ptr(G.dims), _ptr(G.par), G._a(), _ptr(y), _ptr(x0), niter, lam, gamma, sigma, tau, _ptr(x))
    return x


def opnorm_P(G: Geom, iters: int = 50, seed: int = 0) -> float:
    """||P|| by power iteration on P^T P (FP64)."""
    x = np.random.default_rng(seed).random(G.vol_shape)
    s = 0.0
    for _ in range(iters):
        x /= np.linalg.norm(x)
        y = adjoint(G, forward(G, x))
        s = np.sqrt(np.linalg.norm(y))
        x = y
    return float(s)


def opnorm_K(G: Geom, iters: int = 50, seed: int = 0, gamma: float = 1.0) -> float:
    """||K|| for K = [P; gamma grad] by power iteration on K^T K (FP64)."""
    x = np.random.default_rng(seed).random(G.vol_shape)
    s = 0.0
    for _ in range(iters):
        x /= np.linalg.norm(x)
        y = adjoint(G, forward(G, x)) - gamma * gamma * div(grad(x))
        s = np.sqrt(np.linalg.norm(y))
        x = y
    return float(s)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson(p: np.ndarray, I0: float, seed: int) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float32)
    out = np.zeros(p.shape, dtype=np.int32)
    lib().o_poisson(_ptr(p), p.size, float(I0), int(seed), _ptr(out))
    return out


def poisson_lam(lam: np.ndarray, seed: int) -> np.ndarray:
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.zeros(lam.shape, dtype=np.int32)
    lib().o_poisson_lam(_ptr(lam), lam.size, int(seed), _ptr(out))
    return out


def neglog(counts: np.ndarray, I0: float) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    y = np.zeros(counts.shape)
    lib().o_neglog(_ptr(counts), counts.size, float(I0), _ptr(y))
    return y


def phantom(G: Geom, ell: np.ndarray, ss: int = 1) -> np.ndarray:
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    vol = np.zeros(G.vol_shape)
    lib().o_phantom(_ptr(G.dims), _ptr(G.par), _ptr(ell), ell.shape[0], ss, _ptr(vol))
    return vol


def num_threads() -> int:
    return lib().o_num_threads()


# ---- polychromatic primary (Sec. 2.1, "Primary simulation") ----

def water_bone(mu: np.ndarray, mu_w60: float):
    """Water and bone relative densities of a mu_60 volume (Sec. 2.1, the
    water-bone decomposition equations, tau0 = 0)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    rw = np.zeros(mu.shape)
    rb = np.zeros(mu.shape)
    lib().o_water_bone(_ptr(mu), mu.size, float(mu_w60), _ptr(rw), _ptr(rb))
    return rw, rb


def resp(e_kev: float) -> float:
    """Detector response at e keV: piecewise linear through (20, 5), (60, 20), (120, 10)."""
    return float(lib().o_resp(float(e_kev)))


def poly_lam(Lw: np.ndarray, Lb: np.ndarray, mu_w, mu_b, I0: np.ndarray) -> np.ndarray:
    """Mean counts [n][ne] of each energy bin from FP32 water / bone line integrals
    (any leading shape whose last two axes are the panel's nv x nu) and FP32
    intensity maps I0[ne][nv][nu]."""
    Lw = np.ascontiguousarray(Lw, dtype=np.float32)
    Lb = np.ascontiguousarray(Lb, dtype=np.float32)
    I0 = np.ascontiguousarray(I0, dtype=np.float32)
    mw = np.ascontiguousarray(mu_w, dtype=np.float64)
    mb = np.ascontiguousarray(mu_b, dtype=np.float64)
    ne = len(mw)
    npix = I0.shape[-1] * I0.shape[-2]
    lam = np.zeros((Lw.size, ne))
    lib().o_poly_lam(_ptr(Lw), _ptr(Lb), Lw.size, npix, ne, _ptr(mw), _ptr(mb), _ptr(I0), _ptr(lam))
    return lam


def poly_reading(lam: np.ndarray, energies, seed: int, noise: bool = True, return_counts: bool = False):
    """resp-weighted sum over the bins of Poisson(lam) (or of lam, noise=False);
    lam is [n][ne] with the bins in the order of `energies`."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    E = np.ascontiguousarray(energies, dtype=np.float64)
    n, ne = lam.shape
    out = np.zeros(n)
    counts = np.zeros((n, ne), dtype=np.int32)
    lib().o_poly_reading(_ptr(lam), n, ne, _ptr(E), int(seed), 1 if noise else 0, _ptr(out),
                         _ptr(counts) if noise else None)
    return (out, counts) if return_counts else out


def poly_air(energies, I0: np.ndarray) -> np.ndarray:
    """Expected air reading sum_e resp(e) I0[e] per pixel (the normalisation's gain)."""
    I0 = np.asarray(I0, dtype=np.float64)
    acc = np.zeros(I0.shape[1:])
    for j, e in enumerate(energies):
        acc = acc + resp(e) * I0[j]
    return acc


def poly_neglog(reading: np.ndarray, air: np.ndarray, energies) -> np.ndarray:
    """y_primary = -log(min(reading / air, 1)) (Sec. 2.4, normalised primary data);
    air broadcasts over the leading (angle, batch) axes. A reading below that of one
    photon in the least responsive bin (zero photons) is raised to it, so that y
    stays finite (the monochromatic transform clamps counts to one the same way)."""
    floor = min(resp(e) for e in energies)
    r = np.maximum(np.asarray(reading, dtype=np.float64), floor) / air
    return -np.log(np.minimum(r, 1.0))


def poly_primary(G: Geom, mu: np.ndarray, mu_w60: float, energies, mu_w, mu_b, I0: np.ndarray,
                 seed: int, noise: bool = True):
    """The primary model in the paper's order (Sec. 2.1): split mu into water and
    bone, form mu_tilde_e = rho_w mu_w[e] + rho_b mu_b[e] for each bin, project it,
    take the mean counts I0[e] exp(-P mu_tilde_e), draw (or not) and sum with resp.
    Returns (reading [na][nv][nu], y_primary)."""
    rw, rb = water_bone(mu, mu_w60)
    ne = len(energies)
    lam = np.zeros(G.proj_shape + (ne,))
    for j in range(ne):
        p = forward(G, rw * mu_w[j] + rb * mu_b[j])
        lam[..., j] = np.asarray(I0[j], dtype=np.float64) * np.exp(-p)
    reading = poly_reading(lam.reshape(-1, ne), energies, seed, noise).reshape(G.proj_shape)
    return reading, poly_neglog(reading, poly_air(energies, I0), energies)

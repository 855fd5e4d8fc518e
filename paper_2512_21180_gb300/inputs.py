"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds only workload descriptions and random draws: geometry sizes,
ellipsoid phantom parameters and random test arrays. It contains none of the
reconstruction method's arithmetic (no projection, interpolation, weighting or
voxelisation), so both the CUDA path and the independent CPU checker can use it
without sharing any computation.

The workloads stand in for the paper's clinical CT data (Sec. 2.4: 256^3 volumes
at 2 mm, SID 1000 mm, isocentre-detector 536 mm, offset flat panel, full 2*pi
orbit; Sec. 2.2), which is not available: seeded random-ellipsoid phantoms with
soft-tissue, bone-like and air-like values replace the CT scans.
"""
from __future__ import annotations

import math

import numpy as np

# Acquisition constants of the simulated scanner (Sec. 2.2): source-isocentre
# distance 1000 mm, isocentre-detector 536 mm, so source-detector 1536 mm.
SID_MM = 1000.0
SDD_MM = 1536.0


def geometry(name: str) -> dict:
    """Named workload geometries.

    Keys: n (nx, ny, nz), vox (mm, 3), center (mm, 3), nu, nv, du, dv,
    u_offset, v_offset (mm), sid, sdd (mm), n_angles, batch.
    """
    g = dict(center=(0.0, 0.0, 0.0), v_offset=0.0, sid=SID_MM, sdd=SDD_MM, batch=1)
    if name == "small64":      # 64^3 at 4 mm, 64 angles, 96x64 at 1.6 mm, centred panel
        g.update(n=(64, 64, 64), vox=(4.0, 4.0, 4.0), nu=96, nv=64, du=1.6, dv=1.6,
                 u_offset=0.0, n_angles=64)
    elif name == "clinical":   # 256x256x192 at 2 mm, 400 angles, 512x384 at 0.8 mm, +160 mm offset
        g.update(n=(256, 256, 192), vox=(2.0, 2.0, 2.0), nu=512, nv=384, du=0.8, dv=0.8,
                 u_offset=160.0, n_angles=400)
    elif name == "diff128":    # batch 2 of 128^3 at 4 mm, 200 angles, 256x192 at 1.6 mm, +80 mm offset
        g.update(n=(128, 128, 128), vox=(4.0, 4.0, 4.0), nu=256, nv=192, du=1.6, dv=1.6,
                 u_offset=80.0, n_angles=200, batch=2)
    elif name == "lpd128":     # learned primal-dual workload, same geometry as diff128, batch 1
        g.update(n=(128, 128, 128), vox=(4.0, 4.0, 4.0), nu=256, nv=192, du=1.6, dv=1.6,
                 u_offset=80.0, n_angles=200)
    elif name == "coarse128":  # multiscale coarse level: 128x128x96 at 4 mm, clinical panel binned 2x2
        g.update(n=(128, 128, 96), vox=(4.0, 4.0, 4.0), nu=256, nv=192, du=1.6, dv=1.6,
                 u_offset=160.0, n_angles=200)
    elif name == "tiny16":     # 16^3, 8 angles, 24x16 detector (gradcheck / dense-matrix case)
        g.update(n=(16, 16, 16), vox=(4.0, 4.0, 4.0), nu=24, nv=16, du=4.0, dv=4.0,
                 u_offset=0.0, n_angles=8)
    else:
        raise KeyError(name)
    return g


def scaled(g: dict, **kw) -> dict:
    """Copy of a geometry dict with some keys replaced."""
    h = dict(g)
    h.update(kw)
    return h


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a uniform random unit quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


ELL_COLS = 17  # cx cy cz | ax ay az | R (row-major 3x3, rows = ellipsoid axes) | value | mode


def ellipsoids(g: dict, seed: int, n_soft: int = 10, n_bone: int = 0, n_air: int = 0,
               body: bool = False, axes_mm=(10.0, 100.0), mu=(0.01, 0.03),
               body_frac=(0.42, 0.36, 0.47), center_frac: float = 0.8) -> np.ndarray:
    """Seeded random-ellipsoid phantom parameters, one row per ellipsoid.

    Rows are applied in order: mode 0 adds `value` inside the ellipsoid, mode 1
    overwrites with `value` (bone-like 0.04/mm and air-like 0 inserts). Centres are
    uniform in a cylinder of radius center_frac x the half-width of the volume and
    axial extent 0.8 x its height; orientations are uniform random rotations. The
    optional body ellipsoid has semi-axes body_frac x the volume's extent.
    """
    rng = np.random.default_rng(seed)
    n = np.asarray(g["n"], dtype=np.int64)
    vox = np.asarray(g["vox"], dtype=np.float64)
    ext = n * vox
    ctr = np.asarray(g["center"], dtype=np.float64)
    r_cyl = center_frac * 0.5 * min(ext[0], ext[1])
    h_cyl = 0.8 * 0.5 * ext[2]
    rows = []

    def center():
        r = r_cyl * math.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * math.pi)
        return ctr + np.array([r * math.cos(phi), r * math.sin(phi), rng.uniform(-h_cyl, h_cyl)])

    def row(c, a, rot, val, mode):
        return np.concatenate([c, a, rot.reshape(-1), [val, mode]])

    if body:
        a = np.asarray(body_frac) * ext
        rows.append(row(ctr.copy(), a, np.eye(3), 0.02, 0))
    for _ in range(n_soft):
        a = rng.uniform(axes_mm[0], axes_mm[1], size=3)
        rows.append(row(center(), a, _random_rotation(rng), rng.uniform(mu[0], mu[1]), 0))
    for _ in range(n_bone):
        a = rng.uniform(5.0, 25.0, size=3)
        rows.append(row(center(), a, _random_rotation(rng), 0.04, 1))
    for _ in range(n_air):
        a = rng.uniform(5.0, 25.0, size=3)
        rows.append(row(center(), a, _random_rotation(rng), 0.0, 1))
    return np.asarray(rows, dtype=np.float64).reshape(-1, ELL_COLS)


def phantom_params(name: str, seed: int) -> np.ndarray:
    """The phantom recipe of each named workload."""
    g = geometry(name)
    if name == "clinical":
        # body + 31 soft-tissue + 4 bone-like + 4 air-like = 40 ellipsoids
        return ellipsoids(g, seed, n_soft=31, n_bone=4, n_air=4, body=True)
    if name in ("diff128", "lpd128", "coarse128"):
        # the body stays inside the field of view of the +80 mm panel (radius ~182 mm)
        return ellipsoids(g, seed, n_soft=15, n_bone=3, n_air=2, body=True, axes_mm=(8.0, 60.0),
                          body_frac=(0.30, 0.26, 0.47), center_frac=0.5)
    return ellipsoids(g, seed, n_soft=10)


def random_volume(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Uniform [0, 1) random array (operator tests)."""
    return np.random.default_rng(seed).random(shape).astype(dtype)


def random_normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def smooth_volume(n, seed: int, n_blobs: int = 12) -> np.ndarray:
    """Sum of isotropic Gaussian blobs sampled at voxel centres, [nz, ny, nx], float64."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.zeros((nz, ny, nx))
    for _ in range(n_blobs):
        c = rng.uniform(0.25, 0.75, size=3) * np.array([nx, ny, nz])
        s = rng.uniform(0.12, 0.25) * min(n)
        amp = rng.uniform(0.5, 1.5)
        v += amp * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    return v


def line_integrals(shape, seed: int, lo: float = 0.0, hi: float = 12.0) -> np.ndarray:
    """Random line-integral values for photon-count sampling tests (float32)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def lpd_weights(layer_shapes, seed: int, last_scale: float = 0.1) -> np.ndarray:
    """Seeded network weights in the library's flat order: per layer (cout, taps,
    cin) a He-normal weight [cout][taps][cin] (x last_scale for the last layer of each
    3-layer block) followed by a small normal bias [cout]."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (cout, taps, cin) in enumerate(layer_shapes):
        sd = math.sqrt(2.0 / (cin * taps)) * (last_scale if i % 3 == 2 else 1.0)
        out.append(rng.standard_normal(cout * taps * cin) * sd)
        out.append(rng.standard_normal(cout) * 0.01)
    return np.concatenate(out).astype(np.float32)


# ---- polychromatic primary: stand-in tables (Sec. 2.1) ----
# The paper bins the spectrum into ten 10 keV bins centred at 25 ... 115 keV and
# takes per-energy attenuation of water and bone from xraylib and per-pixel
# intensity maps I0_e from a simulated phase file (collimator and bow-tie filter).
# Neither the tables nor the phase file are available, so these smooth synthetic
# stand-ins are used instead; every library call takes the tables as inputs.

POLY_ENERGIES_KEV = tuple(25.0 + 10.0 * i for i in range(10))
MU_WATER_60 = 0.0206  # 1/mm, approximately water at 60 keV


def poly_tables():
    """(energies keV, water 1/mm, bone 1/mm, spectrum weights summing to 1) for the
    ten bins: attenuation as a photoelectric-like (60/E)^3 term plus a slowly
    falling scattering-like (60/E)^0.25 term, 0.0206 /mm for water and 0.0604 /mm
    for cortical bone at 60 keV (bone with a larger photoelectric share); spectrum
    a Kramers-like (120 - E)/E shape hardened by exp(-2 (30/E)^3)."""
    E = np.array(POLY_ENERGIES_KEV)
    x = 60.0 / E
    mu_w = 0.0012 * x ** 3 + 0.0194 * x ** 0.25
    mu_b = 0.0180 * x ** 3 + 0.0424 * x ** 0.25
    s = (120.0 - E) / E * np.exp(-2.0 * (30.0 / E) ** 3)
    return E, mu_w, mu_b, s / s.sum()


def poly_intensity(g: dict, photons_per_mm2: float = 16000.0) -> np.ndarray:
    """Unattenuated counts I0[e][nv][nu] (float32) per energy bin and detector pixel:
    photons per mm^2 (the paper draws 16000-66000) x pixel area x spectrum weight x
    a bow-tie profile 0.3 + 0.7 exp(-(u'/150 mm)^2) over the lateral panel
    coordinate u' (including the panel offset)."""
    _, _, _, s = poly_tables()
    nu, nv = int(g["nu"]), int(g["nv"])
    u = (np.arange(nu) - 0.5 * (nu - 1)) * g["du"] + g["u_offset"]
    bowtie = 0.3 + 0.7 * np.exp(-(u / 150.0) ** 2)
    per_pixel = photons_per_mm2 * g["du"] * g["dv"]
    I0 = per_pixel * s[:, None, None] * np.broadcast_to(bowtie, (nv, nu))[None]
    return np.ascontiguousarray(I0, dtype=np.float32)


"""Pins of the FP64 oracle's projector pair against mathematics, not against itself.

Each check would fail on a plausible slip in the oracle: a wrong step weight or
plane loop (axis-aligned sums, constant volume), a sign or offset error in the
geometry (closed-form chords of off-centre ellipsoids, rotation symmetry), a
wrong interpolation (dense integration of the trilinear interpolant), or an
adjoint that is not the exact transpose (inner products, dense matrix, gather).
"""
import math

import numpy as np
import pytest

from paper_2512_21180_gb300 import inputs as I


def world_rays(g, k_angles=None):
    """Source and pixel-centre positions in mm, written from the geometry's
    definition (Sec. 2.2 setup: source on a circle of radius SID about z, flat panel
    at SDD facing it, panel axis e_u along the direction of rotation)."""
    na = g["n_angles"]
    ks = range(na) if k_angles is None else k_angles
    out = []
    for k in ks:
        th = 2 * math.pi * k / na
        src = np.array([g["sid"] * math.cos(th), g["sid"] * math.sin(th), 0.0])
        towards = -np.array([math.cos(th), math.sin(th), 0.0])
        eu = np.array([-math.sin(th), math.cos(th), 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        iu = np.arange(g["nu"])
        iv = np.arange(g["nv"])
        u = (iu - (g["nu"] - 1) / 2) * g["du"] + g["u_offset"]
        v = (iv - (g["nv"] - 1) / 2) * g["dv"] + g.get("v_offset", 0.0)
        det = src + g["sdd"] * towards
        pix = det[None, None, :] + v[:, None, None] * ev + u[None, :, None] * eu
        out.append((src, pix))
    return out


def ellipsoid_chord(src, pix, c, axes, rot):
    """Length of the segment of the line src->pix inside the ellipsoid
    (x-c)^T M (x-c) <= 1, M = R^T diag(1/a^2) R: roots of A t^2 + 2 B t + C = 0."""
    M = rot.T @ np.diag(1.0 / np.asarray(axes) ** 2) @ rot
    r = pix - src
    s = src - c
    A = np.einsum("...i,ij,...j->...", r, M, r)
    B = np.einsum("...i,ij,...j->...", r, M, s[None, None, :].repeat(r.shape[0], 0).repeat(r.shape[1], 1))
    C = s @ M @ s - 1.0
    disc = np.maximum(B * B - A * C, 0.0)
    return 2 * np.sqrt(disc) / A * np.linalg.norm(r, axis=-1)


def test_philox_known_answers(O):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        assert list(O.philox(v[0:4], v[4:6])) == v[6:10]
        n += 1
    assert n == 3


@pytest.mark.parametrize("k,axis", [(0, 0), (1, 1), (2, 0), (3, 1)])
@pytest.mark.parametrize("shift", [(0, 0), (2, -3), (-5, 4)])
def test_axis_aligned_central_ray(O, k, axis, shift):
    """A ray along a grid line through voxel centres: every bilinear weight is 1 or
    0, so the sum is exactly vox * (sum of the voxels on that line)."""
    g = dict(I.geometry("tiny16"))
    g.update(n=(15, 15, 15), nu=25, nv=17, n_angles=4)  # odd sizes: centre pixel/voxel exist
    # shift the volume so that a different voxel row lies on the central ray
    g["center"] = (0.0, shift[0] * 4.0, shift[1] * 4.0) if axis == 0 else (shift[0] * 4.0, 0.0, shift[1] * 4.0)
    G = O.Geom(g)
    vol = I.random_volume(G.vol_shape, 5).astype(np.float64)
    proj = O.forward(G, vol)
    val = proj[k, 8, 12]
    if axis == 0:   # ray along x at y index 7 - shift0, z index 7 - shift1
        expect = 4.0 * vol[7 - shift[1], 7 - shift[0], :].sum()
    else:
        expect = 4.0 * vol[7 - shift[1], :, 7 - shift[0]].sum()
    assert abs(val - expect) <= 1e-12 * abs(expect)


def test_constant_volume_step_count(O):
    """Constant 1: a ray whose in-plane points stay inside [0, n-1] on every plane
    collects exactly n_a samples of weight 1, i.e. n_a * (world step length)."""
    g = I.geometry("small64")
    G = O.Geom(g)
    proj = O.forward(G, np.ones(G.vol_shape))
    checked = 0
    for k in range(0, g["n_angles"], 5):
        S, D0S, EU, EV = np.split(O.frame(G, k), 4)
        for iv in range(0, g["nv"], 7):
            for iu in range(0, g["nu"], 5):
                R = D0S + iu * EU + iv * EV
                a = O.principal_axis(G, k, iu, iv)
                others = [c for c in range(3) if c != a]
                ok = True
                for i in (0, G.n[a] - 1):
                    t = (i - S[a]) / R[a]
                    for c in others:
                        q = S[c] + t * R[c]
                        ok &= 0.0 <= q <= G.n[c] - 1
                if not ok:
                    continue
                step = np.linalg.norm(R * np.array(g["vox"])) / abs(R[a])
                assert abs(proj[k, iv, iu] - G.n[a] * step) <= 1e-12 * G.n[a] * step
                checked += 1
    assert checked > 50


@pytest.mark.parametrize("offset", [0.0, 40.0])
def test_closed_form_ellipsoid_chords(O, offset):
    """Projection of a supersampled voxelised ellipsoid vs mu * exact chord length,
    and the error shrinks when the voxel size is halved (first-order convergence)."""
    errs = []
    for n, vox in ((32, 8.0), (64, 4.0)):
        g = dict(I.geometry("small64"))
        g.update(n=(n, n, n), vox=(vox, vox, vox), n_angles=16, nu=160, nv=120, du=1.6, dv=1.6,
                 u_offset=offset)
        G = O.Geom(g)
        c = np.array([18.0, -25.0, 12.0])
        axes = np.array([70.0, 45.0, 55.0])
        th = 0.4
        rot = np.array([[math.cos(th), math.sin(th), 0], [-math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
        mu = 0.02
        ell = np.concatenate([c, axes, rot.reshape(-1), [mu, 0]])[None, :]
        vol = O.phantom(G, ell, ss=4)
        proj = O.forward(G, vol)
        ref = np.stack([mu * ellipsoid_chord(s, p, c, axes, rot) for s, p in world_rays(g)])
        errs.append(np.linalg.norm(proj - ref) / np.linalg.norm(ref))
        # total attenuation (integral over the panel) is preserved to well below 1 %
        assert abs(proj.sum() / ref.sum() - 1.0) < 5e-3
    # the error is dominated by the blurred ellipsoid rim and halves with the voxel
    # size (first order): 5.5 % at 8 mm, 2.8 % at 4 mm, 1.4 % at 2 mm
    assert errs[1] <= 3e-2
    assert 0.4 < errs[1] / errs[0] < 0.6


def _trilinear(vol, p):
    """Zero-padded trilinear interpolation of vol[z, y, x] at index points p[..., (x, y, z)]."""
    nz, ny, nx = vol.shape
    pad = np.zeros((nz + 2, ny + 2, nx + 2))
    pad[1:-1, 1:-1, 1:-1] = vol
    q = p + 1.0
    ok = np.all((q >= 0) & (q <= np.array([nx + 1, ny + 1, nz + 1])), axis=-1)
    q = np.clip(q, 0, np.array([nx + 1, ny + 1, nz + 1]) - 1e-9)
    i0 = np.floor(q).astype(int)
    f = q - i0
    val = np.zeros(q.shape[:-1])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                wgt = (f[..., 0] if dx else 1 - f[..., 0]) * (f[..., 1] if dy else 1 - f[..., 1]) * \
                      (f[..., 2] if dz else 1 - f[..., 2])
                ix = np.minimum(i0[..., 0] + dx, nx + 1)
                iy = np.minimum(i0[..., 1] + dy, ny + 1)
                iz = np.minimum(i0[..., 2] + dz, nz + 1)
                val += wgt * pad[iz, iy, ix]
    return val * ok


def test_dense_integration_of_trilinear_interpolant(O):
    """16^3 smooth volume: the Joseph sum agrees with a fine midpoint-rule line
    integral of the zero-padded trilinear interpolant (computed here in mm)."""
    g = I.geometry("tiny16")
    G = O.Geom(g)
    vol = I.smooth_volume(G.n, 3)
    proj = O.forward(G, vol)
    ref = np.zeros_like(proj)
    vox = np.array(g["vox"])
    n = np.array(G.n)
    for k, (src, pix) in enumerate(world_rays(g)):
        r = pix - src
        L = np.linalg.norm(r, axis=-1)
        # the volume (with its one-voxel zero margin) lies in t in [t0, t1] for every ray
        t0 = (g["sid"] - 1.5 * n.max() * vox.max()) / g["sdd"]
        t1 = (g["sid"] + 1.5 * n.max() * vox.max()) / g["sdd"]
        m = 6000
        t = t0 + (np.arange(m) + 0.5) / m * (t1 - t0)
        pts = src[None, None, None, :] + t[None, None, :, None] * r[:, :, None, :]
        idx = pts / vox + (n - 1) / 2.0
        ref[k] = _trilinear(vol, idx).sum(-1) * (t1 - t0) / m * L
    err = np.linalg.norm(proj - ref) / np.linalg.norm(ref)
    assert err <= 1e-2, err


@pytest.mark.parametrize("name,offset", [("tiny16", 0.0), ("tiny16", 12.0), ("small64", 30.0)])
def test_adjoint_identity(O, name, offset):
    g = dict(I.geometry(name))
    g["u_offset"] = offset
    G = O.Geom(g)
    x = I.random_volume(G.vol_shape, 11).astype(np.float64)
    y = I.random_volume(G.proj_shape, 12).astype(np.float64)
    lhs = np.vdot(O.forward(G, x), y)
    rhs = np.vdot(x, O.adjoint(G, y))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_dense_matrix_columns_equal_adjoint_rows(O):
    """16^3 / 8 angles / 24x16: the 3072 x 4096 matrix built column by column from the
    forward equals the one built row by row from the adjoint, and the brute-force
    voxel gather reproduces the adjoint."""
    g = I.geometry("tiny16")
    G = O.Geom(g)
    nvox, nray = int(np.prod(G.vol_shape)), int(np.prod(G.proj_shape))
    A = np.zeros((nray, nvox))
    e = np.zeros(nvox)
    for j in range(nvox):
        e[j] = 1.0
        A[:, j] = O.forward(G, e).ravel()
        e[j] = 0.0
    assert np.count_nonzero(A) > 0.005 * A.size
    rows = np.random.default_rng(0).choice(nray, 256, replace=False)
    er = np.zeros(nray)
    for r in rows:
        er[r] = 1.0
        np.testing.assert_allclose(O.adjoint(G, er).ravel(), A[r], rtol=0, atol=1e-12 * np.abs(A).max())
        er[r] = 0.0
    y = I.random_volume(G.proj_shape, 3).astype(np.float64)
    full = A.T @ y.ravel()
    np.testing.assert_allclose(O.adjoint(G, y).ravel(), full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    ids = np.arange(nvox)
    np.testing.assert_allclose(O.adjoint_voxels(G, y, ids), full, rtol=1e-11, atol=1e-12 * np.abs(full).max())


def test_rotation_by_90_degrees(O):
    """Square grid centred at the isocentre, n_angles divisible by 4: rotating the
    volume by +90 deg about z equals advancing the angle index by n_angles/4."""
    g = dict(I.geometry("tiny16"))
    g.update(n_angles=12, u_offset=6.0)
    G = O.Geom(g)
    vol = I.random_volume(G.vol_shape, 21).astype(np.float64)
    # +90 deg about z maps (x, y) -> (-y, x): new[z, y, x] = old[z, n-1-x, y]
    rot = np.transpose(vol, (0, 2, 1))[:, :, ::-1]
    p0 = O.forward(G, vol)
    p1 = O.forward(G, rot)
    np.testing.assert_allclose(p1[3:], p0[:-3], rtol=1e-10, atol=1e-10 * np.abs(p0).max())


def test_linearity_batch_zero(O):
    G = O.Geom(I.geometry("tiny16"))
    x = I.random_volume(G.vol_shape, 1).astype(np.float64)
    y = I.random_volume(G.vol_shape, 2).astype(np.float64)
    lhs = O.forward(G, 2.5 * x - 0.75 * y)
    rhs = 2.5 * O.forward(G, x) - 0.75 * O.forward(G, y)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    assert not np.any(O.forward(G, np.zeros(G.vol_shape)))
    assert not np.any(O.adjoint(G, np.zeros(G.proj_shape)))


def test_sample_count_small64(O):
    """The small64 workload takes ~25 M samples per projection (the throughput unit)."""
    G = O.Geom(I.geometry("small64"))
    _, ns = O.forward(G, np.zeros(G.vol_shape), return_count=True)
    assert 20e6 < ns < 30e6

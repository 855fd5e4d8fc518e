"""GPU projector pair (forward_project / back_project through the C ABI) against
the FP64 oracle: element-wise on small and ragged cases, sampled rays and voxels
at the clinical size, the adjoint identity, the FP64 instantiation, autograd."""
import math

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L2 bar of the FP32 projector pair against the FP64 oracle


@pytest.fixture(scope="module")
def P():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import projector
    return projector


CASES = {
    "small64": I.geometry("small64"),
    "tiny16": I.geometry("tiny16"),
    "tiny16_offset": I.scaled(I.geometry("tiny16"), u_offset=14.0, v_offset=-3.0),
    "ragged": I.scaled(I.geometry("tiny16"), n=(19, 13, 11), nu=37, nv=23, du=3.1, dv=2.7,
                       u_offset=21.0, n_angles=13),
    "aniso": I.scaled(I.geometry("tiny16"), n=(24, 20, 12), vox=(3.0, 4.0, 5.5), nu=40, nv=20,
                      center=(7.0, -5.0, 3.0), n_angles=9),
    "diag_angles": I.scaled(I.geometry("tiny16"), nu=41, nv=9, du=2.0, n_angles=8),
}


def angles_for(name):
    if name == "diag_angles":   # exactly 45-degree multiples and near-ties
        return np.array([math.pi / 4, 3 * math.pi / 4, -math.pi / 4, 5 * math.pi / 4,
                         math.pi / 4 + 1e-7, math.pi / 4 - 3e-4, 0.3, 2.0])
    return None


@pytest.mark.parametrize("name", list(CASES))
def test_forward_and_adjoint_match_oracle(O, P, name):
    g = CASES[name]
    ang = angles_for(name)
    G = O.Geom(g, angles=ang)
    geom = P.Geometry(g, angles=ang)
    x = I.random_volume(G.vol_shape, 101)
    y = I.random_volume(G.proj_shape, 102)
    pf = to_np(P.forward_project(geom, to_gpu(x)))
    pr = O.forward(G, x.astype(np.float64))
    assert rel_l2(pf, pr) <= TOL
    assert np.abs(pf - pr).max() <= 1e-5 * np.abs(pr).max()
    vb = to_np(P.back_project(geom, to_gpu(y)))
    vr = O.adjoint(G, y.astype(np.float64))
    assert rel_l2(vb, vr) <= TOL
    assert np.abs(vb - vr).max() <= 1e-5 * np.abs(vr).max()


@pytest.mark.parametrize("name", ["tiny16_offset", "ragged", "diag_angles"])
def test_fp64_instantiation_matches_oracle(O, P, name):
    g = CASES[name]
    ang = angles_for(name)
    G = O.Geom(g, angles=ang)
    geom = P.Geometry(g, angles=ang)
    x = I.random_volume(G.vol_shape, 7).astype(np.float64)
    y = I.random_volume(G.proj_shape, 8).astype(np.float64)
    pf = to_np(P.forward_project(geom, to_gpu(x, torch.float64)))
    np.testing.assert_allclose(pf, O.forward(G, x), rtol=1e-12, atol=1e-12 * np.abs(pf).max())
    vb = to_np(P.back_project(geom, to_gpu(y, torch.float64)))
    np.testing.assert_allclose(vb, O.adjoint(G, y), rtol=1e-12, atol=1e-12 * np.abs(vb).max())


@pytest.mark.parametrize("name", ["small64", "clinical"])
def test_adjoint_identity_gpu(P, name):
    g = I.geometry(name)
    geom = P.Geometry(g)
    x = to_gpu(I.random_volume(geom.vol_shape, 1))
    y = to_gpu(I.random_volume(geom.proj_shape, 2))
    lhs = torch.dot(P.forward_project(geom, x).double().ravel(), y.double().ravel()).item()
    rhs = torch.dot(x.double().ravel(), P.back_project(geom, y).double().ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_clinical_sampled_rays_and_voxels(O, P):
    """Full clinical size (256x256x192, 400 angles, 512x384, +160 mm offset) in the
    benchmark's launch configuration: 3000 random rays and 6 voxels recomputed one
    by one by the oracle."""
    g = I.geometry("clinical")
    G = O.Geom(g)
    geom = P.Geometry(g)
    vol = O.phantom(G, I.phantom_params("clinical", 2))
    pf = to_np(P.forward_project(geom, to_gpu(vol))).ravel()
    rng = np.random.default_rng(5)
    rays = rng.choice(pf.size, 3000, replace=False)
    ref = O.forward_rays(G, vol, rays)
    assert rel_l2(pf[rays], ref) <= TOL
    assert np.all(np.abs(pf[rays] - ref) <= 1e-5 * np.abs(ref).max())
    y = I.random_volume(G.proj_shape, 9)
    vb = to_np(P.back_project(geom, to_gpu(y))).ravel()
    nz, ny, nx = G.vol_shape
    pts = [(nx // 2, ny // 2, nz // 2), (10, 200, 31), (128, 3, 100), (255, 255, 191), (60, 140, 0), (200, 90, 150)]
    ids = np.array([(z * ny + yy) * nx + xx for xx, yy, z in pts])
    ref = O.adjoint_voxels(G, y, ids)
    np.testing.assert_allclose(vb[ids], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


def test_clinical_full_volume_on_eight_angles(O, P):
    """Clinical volume and panel (256x256x192 at 2 mm, 512x384 at 0.8 mm, +160 mm offset)
    on 8 of its 400 angles, including exact 45-degree views: every ray of the forward and
    every voxel of the adjoint against the oracle. Bricks of 16x16x16 and no angle split,
    the launch shape of the full 400-angle backprojection."""
    g = I.geometry("clinical")
    k = np.array([0, 37, 50, 99, 150, 201, 250, 333])
    ang = 2 * np.pi * k / 400.0
    gs = I.scaled(g, n_angles=len(k))
    G = O.Geom(gs, angles=ang)
    geom = P.Geometry(gs, angles=ang)
    vol = O.phantom(G, I.phantom_params("clinical", 2))
    pf = to_np(P.forward_project(geom, to_gpu(vol)))
    pr = O.forward(G, vol)
    assert rel_l2(pf, pr) <= TOL, rel_l2(pf, pr)
    y = I.random_volume(G.proj_shape, 19)
    vb = to_np(P.back_project(geom, to_gpu(y)))
    vr = O.adjoint(G, y.astype(np.float64))
    assert rel_l2(vb, vr) <= TOL, rel_l2(vb, vr)
    assert np.abs(vb - vr).max() <= 1e-5 * np.abs(vr).max()


def test_sample_count_matches_oracle(O, P):
    g = I.geometry("small64")
    _, ns = O.forward(O.Geom(g), np.zeros((64, 64, 64)), return_count=True)
    got = P.Geometry(g).count_samples()
    assert abs(got - ns) <= 1e-6 * ns


@pytest.mark.parametrize("name", ["ragged", "small64"])
def test_batch_and_accumulate(P, name):
    """Batch independence and accumulate = 1, on a panel whose rows take the forward's
    per-ray stores (37 columns) and one whose rows take its four-ray vector stores (96).
    The forward's batch items equal single calls bit for bit. The adjoint splits the
    angles of small volumes into partial sums by the size of the grid, which grows with
    the batch, so its items equal single calls up to FP32 summation order, and repeat
    calls of one batch bit for bit."""
    g = CASES[name]
    geom = P.Geometry(g)
    x = to_gpu(I.random_volume((3,) + geom.vol_shape, 4))
    pb = P.forward_project(geom, x)
    for b in range(3):
        assert torch.equal(pb[b], P.forward_project(geom, x[b]))
    acc = pb.clone()
    P.forward_project(geom, x, out=acc, accumulate=True)
    torch.testing.assert_close(acc, 2 * pb, rtol=1e-6, atol=1e-6)
    y = to_gpu(I.random_volume((2,) + geom.proj_shape, 5))
    vb = P.back_project(geom, y)
    assert torch.equal(vb, P.back_project(geom, y))
    for b in range(2):
        v1 = P.back_project(geom, y[b])
        torch.testing.assert_close(vb[b], v1, rtol=1e-6, atol=1e-6 * v1.abs().max().item())
    zero = P.forward_project(geom, torch.zeros_like(x))
    assert not zero.any()


def test_gradcheck_fp64(P):
    g = I.geometry("tiny16")
    geom = P.Geometry(g)
    x = torch.rand((1,) + geom.vol_shape, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: P.project(geom, v), (x,), eps=1e-6, atol=1e-8, fast_mode=False)
    y = torch.rand((1,) + geom.proj_shape, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: P.backproject(geom, v), (y,), eps=1e-6, atol=1e-8, fast_mode=True)


def test_autograd_fp32_matches_oracle_adjoint(O, P):
    """Batch of 2 at 128^3 / 200 angles / 256x192 / +80 mm: the gradient of a random
    linear loss <w, P x> is P* w, compared with the oracle's adjoint."""
    g = I.geometry("diff128")
    G = O.Geom(g)
    geom = P.Geometry(g)
    x = to_gpu(I.random_volume((2,) + geom.vol_shape, 3)).requires_grad_(True)
    w = I.random_normal((2,) + geom.proj_shape, 4)
    loss = (P.project(geom, x) * to_gpu(w)).sum()
    loss.backward()
    gx = to_np(x.grad)
    for b in range(2):
        assert rel_l2(gx[b], O.adjoint(G, w[b].astype(np.float64))) <= TOL


def test_normalized_operators(O, P):
    g = I.geometry("tiny16")
    geom = P.Geometry(g, normalize=True)
    nrm = O.opnorm_P(O.Geom(g), iters=100)
    assert abs(geom.scale * nrm - 1.0) < 1e-3
    x = to_gpu(I.random_volume(geom.vol_shape, 1))
    ref = P.Geometry(g)
    torch.testing.assert_close(P.forward_project(geom, x), geom.scale * P.forward_project(ref, x),
                               rtol=1e-6, atol=1e-7)


def test_invalid_arguments_raise(P):
    from paper_2512_21180_gb300._lib import CbctError
    with pytest.raises(CbctError):
        P.Geometry(I.scaled(I.geometry("tiny16"), sdd=60.0, sid=40.0, nv=200))   # z-principal rays
    with pytest.raises(CbctError):
        P.Geometry(I.scaled(I.geometry("tiny16"), du=-1.0))

"""Multiscale scheme on the GPU: resampling kernels and the two-level learned
primal-dual (outputs and parameter gradients of both levels) against the FP64
reference with the same weights."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import rel_l2, to_gpu, to_np

GEOM = I.scaled(I.geometry("tiny16"), n=(24, 24, 16), vox=(8.0, 8.0, 8.0), nu=40, nv=16, du=4.0, dv=4.0,
                n_angles=12, u_offset=20.0)


def test_module_coarse_geometry_matches_reference():
    from oracle import multiscale_ref as S
    from paper_2512_21180_gb300 import multiscale as MS
    for g in (GEOM, I.geometry("clinical")):
        assert MS.coarse_geometry(g) == S.coarse_geometry(g)
    with pytest.raises(ValueError):
        MS.coarse_geometry(I.scaled(GEOM, nu=41))


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import lpd, multiscale, ops, projector
    return projector, lpd, multiscale, ops


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(3, 6, 10, 14), (1, 12, 16, 40), (2, 4, 2, 8)])
def test_resampling_matches_reference(M, shape):
    from oracle import multiscale_ref as S
    _, _, MS, ops = M
    x = I.random_normal(shape, 5).astype(np.float64)
    xg = to_gpu(x)
    assert rel_l2(to_np(MS.vol_down(xg)), S.vol_down(x)) <= 1e-6
    assert rel_l2(to_np(MS.proj_down(xg)), S.proj_down(x)) <= 1e-6
    assert np.array_equal(to_np(MS.up(xg)), S.up(x.astype(np.float32)))
    # adjoint of the upsampling
    y = I.random_normal(tuple(shape[:-3]) + tuple(2 * s for s in shape[-3:]), 6).astype(np.float64)
    assert rel_l2(to_np(MS.up_adjoint(to_gpu(y))), 8.0 * S.vol_down(y)) <= 1e-6
    with pytest.raises(Exception):
        ops.resample_down(to_gpu(np.zeros((3, 5, 4))))   # 3 is not divisible by 2


def oracle_params(flat, shapes):
    out, o = [], 0
    for cout, taps, cin in shapes:
        w = torch.tensor(flat[o:o + cout * taps * cin], dtype=torch.float64).reshape(cout, taps, cin)
        o += cout * taps * cin
        b = torch.tensor(flat[o:o + cout], dtype=torch.float64)
        o += cout
        k = (3, 3, 3) if taps == 27 else (3, 3)
        out.append((w.permute(0, 2, 1).reshape((cout, cin) + k).contiguous().requires_grad_(True),
                    b.clone().requires_grad_(True)))
    return out


def flat_grads(prm):
    return np.concatenate([np.concatenate([w.grad.permute(0, *range(2, w.dim()), 1).reshape(-1).numpy(),
                                           b.grad.numpy()]) for w, b in prm])


@pytest.mark.gpu
def test_two_level_lpd_matches_reference(O, M):
    from oracle import multiscale_ref as S
    P, L, MS, _ = M
    n_iter, mu, bps = 1, 0.02, 2e-3
    model = MS.MultiscaleLPD(GEOM, n_iter=(n_iter, n_iter), mu_ref=mu, bp_scale=bps)
    shapes = L.layer_shapes(n_iter)
    flat_c = I.lpd_weights(shapes, seed=3, last_scale=0.5)
    flat_f = I.lpd_weights(shapes, seed=4, last_scale=0.5)
    model.coarse.set_params(flat_c)
    model.fine.set_params(flat_f)
    Gf, Gc = O.Geom(GEOM), O.Geom(S.coarse_geometry(GEOM))
    x_true = O.phantom(Gf, I.ellipsoids(GEOM, 5, n_soft=6, axes_mm=(15.0, 60.0)))
    y = O.forward(Gf, x_true) + 0.01 * I.random_normal(Gf.proj_shape, 6).astype(np.float64)
    x0 = 0.8 * x_true + 0.002 * I.random_normal(Gf.vol_shape, 7).astype(np.float64)
    r = I.random_normal(Gf.vol_shape, 8).astype(np.float64)
    rc = I.random_normal(Gc.vol_shape, 9).astype(np.float64)

    xg, xcg = model.forward(to_gpu(y), to_gpu(x0), save_for_backward=True)
    pc, pf = oracle_params(flat_c, shapes), oracle_params(flat_f, shapes)
    split = lambda p: ([p[6 * n:6 * n + 3] for n in range(n_iter)], [p[6 * n + 3:6 * n + 6] for n in range(n_iter)])
    x, xc = S.lpd_multiscale(Gc, Gf, torch.tensor(y), torch.tensor(x0), torch.tensor(O.redundancy(Gc)),
                             torch.tensor(O.redundancy(Gf)), split(pc), split(pf), n_mem=5, mu_ref=mu,
                             bp_c=bps, bp_f=bps, round_grads=True)
    assert rel_l2(to_np(xcg), xc.detach().numpy()) <= 1e-2
    assert rel_l2(to_np(xg), x.detach().numpy()) <= 1e-2
    assert rel_l2(x.detach().numpy(), S.up(xc.detach().numpy())) > 1e-3   # the fine level acted

    ((x * torch.tensor(r)).sum() + (xc * torch.tensor(rc)).sum()).backward()
    model.zero_grad()
    model.backward(to_gpu(r), to_gpu(rc))
    e_f = rel_l2(model.fine.grads().astype(np.float64), flat_grads(pf))
    e_c = rel_l2(model.coarse.grads().astype(np.float64), flat_grads(pc))
    print(f"two-level gradient parity: fine {e_f:.2e}, coarse {e_c:.2e}")
    assert e_f <= 1e-2, e_f
    assert e_c <= 1e-2, e_c

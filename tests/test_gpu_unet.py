"""P4 U-Net primal blocks on the GPU (six P4 3x3x3 layers, 2 x 2 x 2 pooling, nearest
upsampling, skip by concatenation, group average): the network's output and gradients
against the FP64 reference with the same base filters, and equivariance end to end."""
import math

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import grad_tol, rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

GEOM = I.scaled(I.geometry("tiny16"), n=(24, 24, 16), vox=(8.0, 8.0, 8.0), nu=40, nv=16, du=4.0, dv=4.0,
                n_angles=12, u_offset=20.0)
F = 4  # base filters of the full-resolution layers


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import lpd, projector
    return projector, lpd


def unet_layers(cin, cout):
    """(co, g, ci, fan-in of the full layer) of the U-Net's six layers (g = 1: lift)."""
    return [(F, 1, cin, cin * 27), (F, 4, F, 4 * F * 27), (2 * F, 4, F, 4 * F * 27), (2 * F, 4, 2 * F, 8 * F * 27),
            (F, 4, 3 * F, 12 * F * 27), (cout, 4, F, 4 * F * 27)]


def unet_flat(n_iter, n_mem, seed, last_scale=0.1):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_iter):
        for i, (co, t, ci) in enumerate([(32, 9, n_mem + 2), (32, 9, 32), (n_mem, 9, 32)]):
            sd = math.sqrt(2.0 / (ci * t)) * (last_scale if i == 2 else 1.0)
            out += [rng.standard_normal(co * t * ci) * sd, rng.standard_normal(co) * 0.01]
        for i, (co, g, ci, fan) in enumerate(unet_layers(n_mem + 1, n_mem)):
            sd = math.sqrt(2.0 / fan) * (last_scale if i == 5 else 1.0)
            out += [rng.standard_normal(co * g * 27 * ci) * sd, rng.standard_normal(co) * 0.01]
    return np.concatenate(out).astype(np.float32)


def oracle_params(flat, n_iter, n_mem):
    dual, prim, o = [], [], 0

    def take(k):
        nonlocal o
        t = torch.tensor(flat[o:o + k], dtype=torch.float64)
        o += k
        return t
    for _ in range(n_iter):
        d = []
        for co, t, ci in [(32, 9, n_mem + 2), (32, 9, 32), (n_mem, 9, 32)]:
            w = take(co * t * ci).reshape(co, t, ci).permute(0, 2, 1).reshape(co, ci, 3, 3).contiguous()
            d.append((w.requires_grad_(True), take(co).requires_grad_(True)))
        p = []
        for co, g, ci, _ in unet_layers(n_mem + 1, n_mem):
            w = take(co * g * 27 * ci).reshape(co, g, 27, ci).permute(0, 3, 1, 2).reshape(co, ci, g, 3, 3, 3)
            w = w[:, :, 0].contiguous() if g == 1 else w.contiguous()
            p.append((w.requires_grad_(True), take(co).requires_grad_(True)))
        dual.append(d)
        prim.append(p)
    assert o == flat.size
    return dual, prim


def flat_grads(dual, prim):
    g = []
    for d, p in zip(dual, prim):
        for w, b in d:
            g += [w.grad.permute(0, 2, 3, 1).reshape(-1).numpy(), b.grad.numpy()]
        for i, (w, b) in enumerate(p):
            ww = w.grad.unsqueeze(2) if i == 0 else w.grad
            g += [ww.permute(0, 2, 3, 4, 5, 1).reshape(-1).numpy(), b.grad.numpy()]
    return np.concatenate(g)


def test_unet_lpd_matches_oracle(O, M):
    from oracle import lpd_ref as R
    P, L = M
    G = O.Geom(GEOM)
    geom = P.Geometry(GEOM)
    n_iter, n_mem, mu, bps = 2, 5, 0.02, 2e-3
    model = L.LPD(geom, n_iter=n_iter, n_mem=n_mem, mu_ref=mu, bp_scale=bps, unet=True)
    flat = unet_flat(n_iter, n_mem, 41)
    assert flat.size == model.nparams
    model.set_params(flat)
    x_true = O.phantom(G, I.ellipsoids(GEOM, 5, n_soft=6, axes_mm=(15.0, 60.0)))
    y = O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 6).astype(np.float64)
    x0 = 0.8 * x_true + 0.002 * I.random_normal(G.vol_shape, 7).astype(np.float64)
    r = I.random_normal(G.vol_shape, 8).astype(np.float64)
    w = torch.tensor(O.redundancy(G))
    xg = model.forward(to_gpu(y), to_gpu(x0), save_for_backward=True)
    model.zero_grad()
    gy, g0 = model.backward(to_gpu(r), want_y=True, want_x0=True)
    gg = model.grads().astype(np.float64)

    def reference(x0_scale=1.0):
        dual, prim = oracle_params(flat, n_iter, n_mem)
        yt = torch.tensor(y, requires_grad=True)
        x0t = torch.tensor(x0 * x0_scale, requires_grad=True)
        out = R.lpd(G, yt, x0t, w, dual, prim, n_mem=n_mem, mu_ref=mu, bp_scale=bps, round_grads=True, p4=True,
                    unet=True)
        (out * torch.tensor(r)).sum().backward()
        return out.detach().numpy(), flat_grads(dual, prim), yt.grad.numpy(), x0t.grad.numpy()

    xr, gr, gyr, g0r = reference()
    _, gp, gyp, g0p = reference(1.0 + 1e-6)
    assert rel_l2(to_np(xg), xr) <= 1e-2
    assert rel_l2(xr, x0) > 1e-4
    e_w, e_y, e_x = rel_l2(gg, gr), rel_l2(to_np(gy), gyr), rel_l2(to_np(g0), g0r)
    print(f"U-Net LPD gradient parity: params {e_w:.2e} (tol {grad_tol(gr, gp):.2e}), y {e_y:.2e}, x0 {e_x:.2e}")
    assert e_w <= grad_tol(gr, gp) and e_y <= grad_tol(gyr, gyp) and e_x <= grad_tol(g0r, g0p)
    # an inference pass runs the same arithmetic
    assert np.array_equal(to_np(model.forward(to_gpu(y), to_gpu(x0))), to_np(xg))


def test_unet_lpd_is_equivariant_end_to_end(M):
    from oracle import lpd_ref as R
    P, L = M
    geom = P.Geometry(GEOM)
    rng = np.random.default_rng(3)
    x = torch.tensor(I.smooth_volume(GEOM["n"], 4), dtype=torch.float32, device="cuda")
    rot = lambda v: R.rot_vol(v)
    y = P.forward_project(geom, x)
    y_rot = P.forward_project(geom, rot(x))
    q = GEOM["n_angles"] // 4
    errs = {s: rel_l2(to_np(y_rot), to_np(torch.roll(y, s, dims=0))) for s in (q, -q)}
    shift = min(errs, key=errs.get)
    assert errs[shift] <= 1e-5, errs
    y = y + 0.01 * torch.tensor(rng.standard_normal(tuple(y.shape)), dtype=torch.float32, device="cuda")
    y_rot = torch.roll(y, shift, dims=0).contiguous()
    x0 = 0.8 * x
    model = L.LPD(geom, n_iter=2, unet=True, seed=5, mu_ref=0.5, bp_scale=2e-3)
    model.set_params(model.get_params() * 3.0)
    out = model.forward(y, x0)
    out_rot = model.forward(y_rot, rot(x0).contiguous())
    ratio = rel_l2(to_np(out_rot), to_np(rot(out))) / rel_l2(to_np(out), to_np(x0))
    print(f"U-Net equivariance defect relative to the network's change: {ratio:.2e}")
    assert rel_l2(to_np(out), to_np(x0)) > 1e-3
    assert ratio <= 1e-4, ratio


def test_unet_needs_p4_grid_and_even_sizes(M):
    P, L = M
    odd = I.scaled(GEOM, n=(24, 24, 15))
    with pytest.raises(Exception):
        L.LPD(P.Geometry(odd), n_iter=1, unet=True)

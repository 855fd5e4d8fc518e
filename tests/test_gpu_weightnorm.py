"""Forced weight normalisation on the GPU: the network with normalised filters (a
learnable gain per layer after each bias) against the FP64 reference built from
weight_norm(), for plain blocks and for the P4 U-Net primal block (base filters
normalised before the rotation expansion); and the forced step after Adam, which
re-projects every raw filter without changing the network."""
import math

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import grad_tol, rel_l2, to_gpu, to_np
from test_gpu_unet import unet_layers

pytestmark = pytest.mark.gpu

GEOM = I.scaled(I.geometry("tiny16"), n=(24, 24, 16), vox=(8.0, 8.0, 8.0), nu=40, nv=16, du=4.0, dv=4.0,
                n_angles=12, u_offset=20.0)
N_ITER, N_MEM, MU, BPS = 2, 5, 0.02, 2e-3


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import lpd, projector
    return projector, lpd


def layers(unet):
    """Per iteration: (co, g, t, ci) of each layer, g = 0 for plain layers (weights
    [co][t][ci]), else base filters [co][g][27][ci]."""
    dual = [(32, 0, 9, N_MEM + 2), (32, 0, 9, 32), (N_MEM, 0, 9, 32)]
    prim = ([(co, g, 27, ci) for co, g, ci, _ in unet_layers(N_MEM + 1, N_MEM)] if unet else
            [(32, 0, 27, N_MEM + 1), (32, 0, 27, 32), (N_MEM, 0, 27, 32)])
    return dual + prim


def flat_params(unet, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(N_ITER):
        for co, g, t, ci in layers(unet):
            out += [rng.standard_normal(co * max(g, 1) * t * ci) * 0.1, rng.standard_normal(co) * 0.01,
                    [0.2 + 0.6 * rng.random()]]
    return np.concatenate(out).astype(np.float32)


def oracle_params(flat, unet):
    from oracle import lpd_ref as R
    dual, prim, raw, o = [], [], [], 0

    def take(k):
        nonlocal o
        t = torch.tensor(flat[o:o + k], dtype=torch.float64)
        o += k
        return t.requires_grad_(True)
    for _ in range(N_ITER):
        blk = []
        for co, g, t, ci in layers(unet):
            w = take(co * max(g, 1) * t * ci)
            b, gain = take(co), take(1)
            raw.append((w, b, gain))
            if g == 0:
                k = (3, 3, 3) if t == 27 else (3, 3)
                ww = w.reshape(co, t, ci).permute(0, 2, 1).reshape((co, ci) + k)
            else:
                ww = w.reshape(co, g, 27, ci).permute(0, 3, 1, 2).reshape(co, ci, g, 3, 3, 3)
                if g == 1:
                    ww = ww[:, :, 0]
            blk.append((R.weight_norm(ww, gain[0]), b))
        dual.append(blk[:3])
        prim.append(blk[3:])
    assert o == flat.size
    return dual, prim, raw


def case(O, M, unet):
    from oracle import lpd_ref as R
    P, L = M
    G = O.Geom(GEOM)
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=N_ITER, n_mem=N_MEM, mu_ref=MU, bp_scale=BPS, unet=unet, weight_norm=True)
    flat = flat_params(unet, 51 + unet)
    assert flat.size == model.nparams
    model.set_params(flat)
    x_true = O.phantom(G, I.ellipsoids(GEOM, 5, n_soft=6, axes_mm=(15.0, 60.0)))
    y = O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 6).astype(np.float64)
    x0 = 0.8 * x_true + 0.002 * I.random_normal(G.vol_shape, 7).astype(np.float64)
    r = I.random_normal(G.vol_shape, 8).astype(np.float64)
    w = torch.tensor(O.redundancy(G))

    def reference(x0_scale=1.0):
        dual, prim, raw = oracle_params(flat, unet)
        x0t = torch.tensor(x0 * x0_scale)
        out = R.lpd(G, torch.tensor(y), x0t, w, dual, prim, n_mem=N_MEM, mu_ref=MU, bp_scale=BPS, round_grads=True,
                    p4=unet, unet=unet)
        (out * torch.tensor(r)).sum().backward()
        return out.detach().numpy(), np.concatenate([t.grad.numpy().reshape(-1) for lay in raw for t in lay])
    return model, (y, x0, r), reference


@pytest.mark.parametrize("unet", [False, True])
def test_weight_normalised_lpd_matches_oracle(O, M, unet):
    model, (y, x0, r), reference = case(O, M, unet)
    xg = model.forward(to_gpu(y), to_gpu(x0), save_for_backward=True)
    model.zero_grad()
    model.backward(to_gpu(r))
    gg = model.grads().astype(np.float64)
    xr, gr = reference()
    _, gp = reference(1.0 + 1e-6)
    assert rel_l2(to_np(xg), xr) <= 1e-2
    assert rel_l2(xr, x0) > 1e-4
    e = rel_l2(gg, gr)
    print(f"weight-normalised LPD (U-Net {unet}): output {rel_l2(to_np(xg), xr):.2e}, params {e:.2e} "
          f"(tol {grad_tol(gr, gp):.2e})")
    assert e <= grad_tol(gr, gp)


def test_forced_step_keeps_the_network(O, M):
    """Adam with lr = 0 changes nothing but the forced re-projection: every raw filter then
    has zero mean and norm sqrt(fan-in), and the network's output is unchanged."""
    model, (y, x0, _), _ = case(O, M, False)
    before = to_np(model.forward(to_gpu(y), to_gpu(x0)))
    model.zero_grad()
    model.adam_step(0.0)
    theta = model.get_params().astype(np.float64)
    o = 0
    for _ in range(N_ITER):
        for co, g, t, ci in layers(False):
            n = t * ci
            wr = theta[o:o + co * n].reshape(co, n)
            assert np.abs(wr.mean(1)).max() <= 1e-6
            assert np.allclose(np.linalg.norm(wr, axis=1), math.sqrt(n), rtol=1e-5)
            o += co * n + co + 1
    assert o == theta.size
    after = to_np(model.forward(to_gpu(y), to_gpu(x0)))
    assert rel_l2(after, before) <= 1e-5

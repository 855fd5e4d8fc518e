"""GPU FDK_w, operator norm, PDHG-TV and Landweber against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import ops, projector
    return projector, ops


FDK_CASES = {
    "centred": I.scaled(I.geometry("small64"), n=(48, 48, 40), nu=160, nv=96, n_angles=90),
    "offset": I.scaled(I.geometry("small64"), n=(48, 48, 40), nu=112, nv=96, u_offset=50.0, n_angles=90),
}


@pytest.mark.parametrize("name", list(FDK_CASES))
def test_fdk_matches_oracle(O, M, name):
    P, ops = M
    g = FDK_CASES[name]
    G = O.Geom(g)
    geom = P.Geometry(g)
    vol = O.phantom(G, I.phantom_params("small64", 4))
    proj = O.forward(G, vol)
    got = to_np(ops.fdk(geom, to_gpu(proj)))[0]
    ref = O.fdk(G, proj)
    err = rel_l2(got, ref)
    # FP32 positions (~1e-5 pixel at 160 columns) inside a sharp filtered row
    assert err <= 1e-4, err
    assert ops.fdk(geom, to_gpu(proj)).shape == (1,) + G.vol_shape


@pytest.mark.parametrize("gamma", [0.0, 5.0])
def test_opnorm_matches_oracle(O, M, gamma):
    P, ops = M
    g = I.scaled(I.geometry("tiny16"), u_offset=9.0)
    got = ops.opnorm(P.Geometry(g), gamma=gamma, iters=200)
    ref = O.opnorm_K(O.Geom(g), iters=200, gamma=gamma) if gamma else O.opnorm_P(O.Geom(g), iters=200)
    assert abs(got / ref - 1.0) < 1e-4


def test_pdhg_matches_oracle(O, M):
    """Same data, start, lam, gamma, sigma, tau: 60 iterations agree to 1e-4."""
    P, ops = M
    g = I.scaled(I.geometry("tiny16"), n=(20, 20, 12), u_offset=6.0, n_angles=24)
    G = O.Geom(g)
    geom = P.Geometry(g)
    x_true = O.phantom(G, I.ellipsoids(g, 3, n_soft=5, axes_mm=(8.0, 30.0)))
    y = O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 5).astype(np.float64)
    gam = O.opnorm_P(G) / math.sqrt(12.0)
    L = O.opnorm_K(G, gamma=gam)
    sig = tau = 0.99 / L
    lam = 0.05
    ref = O.pdhg(G, y, np.zeros(G.vol_shape), 60, lam, sig, tau, gamma=gam)
    got = to_np(ops.pdhg(geom, to_gpu(y), torch.zeros((1,) + G.vol_shape, device="cuda"), 60, lam, gam, sig, tau))[0]
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)


def test_landweber_matches_oracle(O, M):
    P, ops = M
    g = I.scaled(I.geometry("tiny16"), u_offset=6.0)
    G = O.Geom(g)
    geom = P.Geometry(g)
    y = O.forward(G, I.random_volume(G.vol_shape, 2).astype(np.float64))
    tau = 1.0 / O.opnorm_P(G) ** 2
    x = np.zeros(G.vol_shape)
    for _ in range(10):
        x = x - tau * O.adjoint(G, O.forward(G, x) - y)
    got = to_np(ops.landweber(geom, to_gpu(y), torch.zeros((1,) + G.vol_shape, device="cuda"), 10, tau))[0]
    assert rel_l2(got, x) <= 1e-5

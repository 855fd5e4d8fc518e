"""Pins of the oracle's field-of-view tensor, redundancy weight, FDK, PDHG,
Poisson sampler, log transform and phantom voxeliser against closed forms,
library routines on special cases, and statistics."""
import math

import numpy as np
import pytest
from scipy import optimize, stats

from paper_2512_21180_gb300 import inputs as I

from test_oracle_projector import ellipsoid_chord, world_rays


def _fraction_u_above(c, r, sid, sdd):
    """Fraction of orbit angles at which a point at radius r (mid-plane) projects to
    u' >= c on a flat panel at sdd: u' = sdd r sin(psi) / (sid - r cos(psi)) >= c
    <=> r sqrt(sdd^2 + c^2) sin(psi + phi) >= c sid."""
    s = c * sid / (r * math.sqrt(sdd * sdd + c * c))
    if s >= 1:
        return 0.0
    if s <= -1:
        return 1.0
    return (math.pi - 2 * math.asin(s)) / (2 * math.pi)


@pytest.mark.parametrize("offset", [0.0, 115.0])
def test_fov_closed_form(O, offset):
    """Mid-plane voxels: V equals the fraction of the orbit during which the voxel
    projects onto the panel, from the closed form above, within the angular
    sampling error."""
    g = dict(I.geometry("tiny16"))
    g.update(n=(41, 41, 1), vox=(7.0, 7.0, 7.0), nu=256, nv=8, du=1.6, dv=1.6, u_offset=offset,
             n_angles=720)
    G = O.Geom(g)
    V = O.fov(G)[0]
    lo, hi = offset - 128 * 1.6, offset + 128 * 1.6
    errs = []
    for iy in range(41):
        for ix in range(41):
            x, y = (ix - 20) * 7.0, (iy - 20) * 7.0
            r = math.hypot(x, y)
            if r < 1e-9:
                exp = 1.0
            else:
                exp = _fraction_u_above(lo, r, 1000.0, 1536.0) - _fraction_u_above(hi, r, 1000.0, 1536.0)
            errs.append(abs(V[iy, ix] - exp))
    assert max(errs) <= 3.0 / 720


def test_redundancy_weight(O):
    """w(u') + w(-u') = 1 on conjugate columns; 0 / 1 outside the overlap band;
    monotone; a centred panel gets 1/2 everywhere; a mirrored offset mirrors w."""
    g = dict(I.geometry("lpd128"))
    g.update(u_offset=40 * 1.6)   # conjugate of column i is column nu - 1 - i - 80
    G = O.Geom(g)
    w = O.redundancy(G)
    nu = g["nu"]
    u = (np.arange(nu) - (nu - 1) / 2) * g["du"] + g["u_offset"]
    pairs = 0
    for i in range(nu):
        j = nu - 1 - i - 80
        if 0 <= j < nu:
            assert abs(w[i] + w[j] - 1.0) < 1e-14
            pairs += 1
    assert pairs > 50
    D = nu * g["du"] / 2 - g["u_offset"]
    assert np.all(w[u > D] == 1.0)
    assert np.all(np.diff(w) >= 0)
    assert np.all(w[u < -D] == 0.0) and np.all((w > 0)[u > -D])
    gc = dict(g)
    gc["u_offset"] = 0.0
    assert np.all(O.redundancy(O.Geom(gc)) == 0.5)
    gm = dict(g)
    gm["u_offset"] = -g["u_offset"]
    np.testing.assert_allclose(O.redundancy(O.Geom(gm)), w[::-1], atol=1e-14)


def _ball_projection(g, radius, mu):
    c = np.zeros(3)
    ax = np.full(3, radius)
    return np.stack([mu * ellipsoid_chord(s, p, c, ax, np.eye(3)) for s, p in world_rays(g)])


@pytest.mark.parametrize("offset", [0.0, 80.0])
def test_fdk_reconstructs_uniform_ball(O, offset):
    """FDK of exact (closed-form) projections of a uniform ball recovers its value
    in the interior and ~0 outside: pins the ramp-filter scaling, the cosine and
    distance weights and the redundancy weight."""
    g = dict(I.geometry("small64"))
    g.update(nu=256 if offset == 0 else 160, nv=128, du=1.6, dv=1.6, u_offset=offset, n_angles=180)
    G = O.Geom(g)
    mu, radius = 0.02, 60.0
    rec = O.fdk(G, _ball_projection(g, radius, mu))
    n = 64
    idx = (np.arange(n) - (n - 1) / 2) * 4.0
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    R = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    inner = R < 40.0
    outer = (R > 80.0) & (np.sqrt(X ** 2 + Y ** 2) < 110.0) & (np.abs(Z) < 20.0)
    assert abs(rec[inner].mean() / mu - 1.0) < 0.02
    assert np.abs(rec[inner] / mu - 1.0).max() < 0.08
    assert np.abs(rec[outer]).mean() < 0.03 * mu


def test_grad_div_adjoint(O):
    x = I.random_volume((5, 6, 7), 1).astype(np.float64)
    g3 = I.random_volume((3, 5, 6, 7), 2).astype(np.float64)
    assert abs(np.vdot(O.grad(x), g3) + np.vdot(x, O.div(g3))) < 1e-12 * abs(np.vdot(O.grad(x), g3))
    # forward differences of a linear ramp in x: 1 except on the last column
    ramp = np.broadcast_to(np.arange(7.0), (5, 6, 7)).copy()
    gr = O.grad(ramp)
    assert np.all(gr[0][..., :-1] == 1.0) and np.all(gr[0][..., -1] == 0.0) and not gr[1:].any()


def _tiny_pdhg_geom():
    g = dict(I.geometry("tiny16"))
    g.update(n=(8, 8, 8), vox=(8.0, 8.0, 8.0), nu=16, nv=12, du=6.0, dv=6.0, n_angles=16)
    return g


def test_pdhg_without_tv_matches_nnls(O):
    """lam = 0 removes the TV term: PDHG must converge to the non-negative least
    squares solution, computed here by scipy's NNLS on the dense matrix."""
    g = _tiny_pdhg_geom()
    G = O.Geom(g)
    nvox = int(np.prod(G.vol_shape))
    A = np.zeros((int(np.prod(G.proj_shape)), nvox))
    e = np.zeros(nvox)
    for j in range(nvox):
        e[j] = 1.0
        A[:, j] = O.forward(G, e).ravel()
        e[j] = 0.0
    xt = np.maximum(I.random_normal(G.vol_shape, 4).astype(np.float64), 0.0) * 0.02
    y = A @ xt.ravel() + 0.02 * I.random_normal(A.shape[0], 5).astype(np.float64)
    x_nnls, _ = optimize.nnls(A, y, maxiter=50 * nvox)
    gam = O.opnorm_P(G) / math.sqrt(12.0)
    L = O.opnorm_K(G, gamma=gam)
    x = O.pdhg(G, y.reshape(G.proj_shape), np.zeros(G.vol_shape), 3000, 0.0, 0.99 / L, 0.99 / L, gamma=gam)
    assert np.linalg.norm(x.ravel() - x_nnls) <= 2e-3 * np.linalg.norm(x_nnls)


def test_pdhg_huge_tv_gives_best_constant(O):
    """lam -> infinity forces grad x = 0: the minimiser is the best non-negative
    constant c = max(0, <P1, y> / ||P1||^2)."""
    g = _tiny_pdhg_geom()
    G = O.Geom(g)
    y = O.forward(G, I.random_volume(G.vol_shape, 8).astype(np.float64))
    p1 = O.forward(G, np.ones(G.vol_shape))
    c = max(0.0, np.vdot(p1, y) / np.vdot(p1, p1))
    gam = O.opnorm_P(G) / math.sqrt(12.0)
    L = O.opnorm_K(G, gamma=gam)
    x = O.pdhg(G, y, np.zeros(G.vol_shape), 10000, 1e6, 0.99 / L, 0.99 / L, gamma=gam)
    # TV-dominated problems converge at the O(1/k) rate: 0.35 % spread after 1e4 steps
    assert abs(x.mean() / c - 1.0) < 1e-3
    assert x.std() < 1e-2 * c


def test_opnorm_by_power_iteration_matches_dense_svd(O):
    g = _tiny_pdhg_geom()
    G = O.Geom(g)
    nvox = int(np.prod(G.vol_shape))
    K = []
    e = np.zeros(nvox)
    for j in range(nvox):
        e[j] = 1.0
        v = e.reshape(G.vol_shape)
        K.append(np.concatenate([O.forward(G, v).ravel(), 7.0 * O.grad(v).ravel()]))
        e[j] = 0.0
    s = np.linalg.norm(np.array(K).T, 2)
    assert abs(O.opnorm_K(G, iters=200, gamma=7.0) / s - 1.0) < 1e-6


@pytest.mark.parametrize("lam", [0.7, 2.5, 9.99, 10.0, 25.0, 300.0])
def test_poisson_distribution_chi2(O, lam):
    """Counts follow the Poisson(lam) pmf (chi-square goodness of fit, 2e5 draws),
    on both the inversion (lam < 10) and the PTRS (lam >= 10) branch."""
    n = 200_000
    k = O.poisson_lam(np.full(n, lam), seed=1234 + int(lam * 100))
    lo, hi = int(max(0, lam - 6 * math.sqrt(lam) - 2)), int(lam + 6 * math.sqrt(lam) + 3)
    edges = np.arange(lo, hi + 1)
    obs = np.array([np.sum(k <= lo)] + [np.sum(k == v) for v in edges[1:-1]] + [np.sum(k >= hi)])
    pm = stats.poisson(lam)
    exp = np.array([pm.cdf(lo)] + [pm.pmf(v) for v in edges[1:-1]] + [pm.sf(hi - 1)]) * n
    keep = exp > 5
    chi2 = (((obs - exp) ** 2)[keep] / exp[keep]).sum()
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4


@pytest.mark.parametrize("lam", [1.0, 10.0, 1e3, 1e5])
def test_poisson_mean_variance(O, lam):
    n = 1_000_000
    k = O.poisson_lam(np.full(n, lam), seed=99).astype(np.float64)
    assert abs(k.mean() - lam) < 5 * math.sqrt(lam / n)
    assert abs(k.var() / lam - 1.0) < 5 * math.sqrt(2.0 / n) + 2e-3


def test_poisson_from_line_integrals_is_deterministic(O):
    p = I.line_integrals(50_000, 3)
    a = O.poisson(p, 1e5, seed=7)
    b = O.poisson(p, 1e5, seed=7)
    c = O.poisson(p, 1e5, seed=8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a >= 0)


def test_neglog(O):
    I0 = 1000.0 * math.e ** 2
    y = O.neglog(np.array([1000, 0, 10 ** 6, int(I0) + 1], dtype=np.int32), I0)
    assert abs(y[0] - 2.0) < 1e-12
    assert abs(y[1] - math.log(I0)) < 1e-12    # zero counts clamped to one
    assert y[2] == 0.0 and y[3] == 0.0          # min(., 1)


def test_phantom_volume_and_overwrite(O):
    g = I.geometry("small64")
    G = O.Geom(g)
    c = np.array([10.0, -20.0, 5.0])
    ax = np.array([60.0, 40.0, 30.0])
    body = np.concatenate([c, ax, np.eye(3).ravel(), [0.02, 0]])
    hole = np.concatenate([c, [10.0, 10.0, 10.0], np.eye(3).ravel(), [0.0, 1]])
    v = O.phantom(G, body[None], ss=4)
    vol_mm3 = v.sum() * 4.0 ** 3
    assert abs(vol_mm3 / (0.02 * 4 / 3 * math.pi * ax.prod()) - 1.0) < 5e-3
    v2 = O.phantom(G, np.stack([body, hole]), ss=1)
    ic = np.round(c / 4.0 + 31.5).astype(int)
    assert v2[ic[2], ic[1], ic[0]] == 0.0
    assert abs(v2[ic[2], ic[1], ic[0] + 5] - 0.02) < 1e-15

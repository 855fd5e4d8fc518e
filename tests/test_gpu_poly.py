"""Polychromatic primary simulation (Sec. 2.1, primary model; Sec. 2.4,
normalised primary data) through the C ABI against the oracle: the water-bone
split, per-energy Poisson counts from seeded line integrals (bit-exact integers),
the expected and noisy readings, and the whole simulation (split, two
projections, reading, log) against the oracle's per-energy projections in the
paper's order, on small volumes, ragged panels and sampled clinical rays."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import rel_l2, to_gpu

MU_W = I.MU_WATER_60


def test_detector_response_matches_oracle(O):
    """Host-only entry point (no GPU needed): resp at the paper's bins and beyond."""
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import ops
    E = np.array(list(I.POLY_ENERGIES_KEV) + [10.0, 20.0, 60.0, 120.0, 131.0, 47.3])
    got = ops.detector_response(E)
    ref = np.array([O.resp(e) for e in E])
    np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import ops, projector
    return projector, ops


@pytest.mark.gpu
def test_water_bone_matches_oracle(O, M):
    _, ops = M
    rng = np.random.default_rng(4)
    mu = rng.uniform(-0.1, 4.2, size=(2, 7, 9, 13)) * MU_W
    mu[0, 0, 0, :6] = np.array([0.0, 1.2, 1.6, 1.2 - 1e-7, 1.6 + 1e-7, -0.0]) * MU_W
    mu32 = mu.astype(np.float32)
    rho = ops.water_bone(to_gpu(mu32), MU_W).cpu().numpy()
    w, b = O.water_bone(mu32.astype(np.float64), MU_W)
    assert rho.shape == (2, 2, 7, 9, 13)
    np.testing.assert_allclose(rho[:, 0], w, rtol=0, atol=2e-6)
    np.testing.assert_allclose(rho[:, 1], b, rtol=0, atol=2e-6)


def _tables(ne):
    E, mw, mb, _ = I.poly_tables()
    if ne <= len(E):
        return E[:ne], mw[:ne], mb[:ne]
    k = ne - len(E)
    return (np.concatenate([E, 120.0 + 5.0 * np.arange(k)]), np.concatenate([mw, np.full(k, 0.016)]),
            np.concatenate([mb, np.full(k, 0.037)]))


@pytest.mark.gpu
@pytest.mark.parametrize("ne,nv,nu,na,batch", [(10, 17, 29, 3, 2), (1, 8, 8, 2, 1), (16, 5, 33, 4, 1)])
def test_poly_counts_bit_exact(O, M, ne, nv, nu, na, batch):
    """Counts of every bin equal the oracle's integer draws on the same seeded line
    integrals; readings and normalised data agree to FP32 rounding."""
    _, ops = M
    E, mw, mb = _tables(ne)
    rng = np.random.default_rng(100 + ne)
    L = np.empty((batch, 2, na, nv, nu), dtype=np.float32)
    L[:, 0] = rng.uniform(0.0, 420.0, size=(batch, na, nv, nu))     # water path, mm of rho_w
    L[:, 1] = rng.uniform(0.0, 70.0, size=(batch, na, nv, nu))      # bone path
    L[0, 0, 0, 0, :3] = 0.0
    L[0, 1, 0, 0, :3] = 0.0
    g = dict(nu=nu, nv=nv, du=1.6, dv=1.6, u_offset=20.0)
    I0 = I.poly_intensity(g, photons_per_mm2=40000.0)
    if ne != len(I0):
        I0 = np.ascontiguousarray(np.resize(I0, (ne, nv, nu)))
    reading, y, counts = ops.poly_reading(to_gpu(L), to_gpu(I0), E, mw, mb, seed=99, noise=True, want_counts=True)
    lam = O.poly_lam(L[:, 0], L[:, 1], mw, mb, I0)
    ref, ref_counts = O.poly_reading(lam, E, seed=99, noise=True, return_counts=True)
    assert np.array_equal(counts.cpu().numpy().reshape(-1, ne), ref_counts)
    ref = ref.reshape(batch, na, nv, nu)
    np.testing.assert_allclose(reading.cpu().numpy(), ref.astype(np.float32), rtol=1e-7, atol=0)
    air = O.poly_air(E, I0)
    np.testing.assert_allclose(y.cpu().numpy(), O.poly_neglog(ref, air, E), rtol=1e-6, atol=1e-6)
    # expected reading (no draws)
    r0, y0, _ = ops.poly_reading(to_gpu(L), to_gpu(I0), E, mw, mb, seed=99, noise=False)
    ref0 = O.poly_reading(lam, E, seed=0, noise=False).reshape(batch, na, nv, nu)
    np.testing.assert_allclose(r0.cpu().numpy(), ref0, rtol=2e-7, atol=0)
    np.testing.assert_allclose(y0.cpu().numpy(), O.poly_neglog(ref0, air, E), rtol=1e-6, atol=1e-6)


def _phantom_mu(O, g, seed):
    """mu_60 phantom with soft tissue, dense bone and air (values in every branch
    of the water-bone split), made by the oracle's voxeliser, rounded to FP32."""
    G = O.Geom(g)
    ell = I.ellipsoids(g, seed=seed, n_soft=8, n_bone=3, n_air=2, body=True)
    return O.phantom(G, ell).astype(np.float32)


@pytest.mark.gpu
@pytest.mark.parametrize("name,kw", [("small64", {}),
                                     ("small64", dict(n=(37, 45, 29), nu=71, nv=53, n_angles=11, u_offset=30.0))])
def test_poly_simulate_matches_paper_order(O, M, name, kw):
    """Noise-free simulation (split, two projections, reading, log) against the
    oracle's per-energy projections of mu_tilde_e; the line integrals against the
    oracle's projections of rho_w and rho_b. Tolerance: the projector's 1e-5."""
    P, ops = M
    g = I.scaled(I.geometry(name), **kw)
    G = O.Geom(g)
    geom = P.Geometry(g)
    mu = _phantom_mu(O, g, seed=31)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    L, y = ops.poly_simulate(geom, to_gpu(mu), to_gpu(I0), E, mw, mb, MU_W, seed=3, noise=False)
    rw, rb = O.water_bone(mu.astype(np.float64), MU_W)
    assert rb.max() > 0.3 and rw.max() > 0.5
    Lc = L.cpu().numpy()
    assert rel_l2(Lc[0, 0], O.forward(G, rw)) <= 1e-5
    assert rel_l2(Lc[0, 1], O.forward(G, rb)) <= 1e-5
    _, yref = O.poly_primary(G, mu.astype(np.float64), MU_W, E, mw, mb, I0, seed=3, noise=False)
    yc = y.cpu().numpy()[0]
    assert rel_l2(yc, yref) <= 1e-5
    assert np.max(np.abs(yc - yref)) <= 1e-5 * max(1.0, yref.max())


@pytest.mark.gpu
def test_poly_simulate_noise_batch_and_reading_agree(O, M):
    """The noisy simulation of a batch equals cbct_poly_reading on its own line
    integrals (same counters: batch item b, angle, pixel in order), and the noisy
    data scatter around the expected ones with the Poisson spread."""
    P, ops = M
    g = I.geometry("small64")
    geom = P.Geometry(g)
    mu = np.stack([_phantom_mu(O, g, seed=s) for s in (5, 6)])
    E, mw, mb, _ = I.poly_tables()
    I0 = to_gpu(I.poly_intensity(g, photons_per_mm2=66000.0))
    L, y = ops.poly_simulate(geom, to_gpu(mu), I0, E, mw, mb, MU_W, seed=17, noise=True)
    _, y2, _ = ops.poly_reading(L, I0, E, mw, mb, seed=17, noise=True)
    assert torch.equal(y, y2)
    _, y0, _ = ops.poly_reading(L, I0, E, mw, mb, seed=17, noise=False)
    assert bool(torch.isfinite(y).all())
    y0c = y0.cpu().numpy()
    d = (y.cpu().numpy() - y0c)[y0c < 4.0]           # rays that keep hundreds of photons
    assert abs(d.mean()) < 2e-3 and 1e-4 < d.std() < 5e-2


@pytest.mark.gpu
def test_poly_simulate_clinical_sampled_rays(O, M):
    """Clinical size (256 x 256 x 192, 400 angles, 512 x 384 offset panel): noise-free
    normalised data on 400 sampled rays, the oracle walking each ray once per bin."""
    P, ops = M
    g = I.geometry("clinical")
    G = O.Geom(g)
    geom = P.Geometry(g)
    mu = _phantom_mu(O, g, seed=44)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    _, y = ops.poly_simulate(geom, to_gpu(mu), to_gpu(I0), E, mw, mb, MU_W, seed=1, noise=False)
    rng = np.random.default_rng(8)
    n_rays = g["n_angles"] * g["nv"] * g["nu"]
    ids = rng.choice(n_rays, size=400, replace=False)
    rw, rb = O.water_bone(mu.astype(np.float64), MU_W)
    lw, lb = O.forward_rays(G, rw, ids), O.forward_rays(G, rb, ids)
    pix = ids % (g["nv"] * g["nu"])
    i0 = I0.reshape(len(E), -1)[:, pix].astype(np.float64)
    resp = np.array([O.resp(e) for e in E])
    # per-energy line integrals of mu_tilde_e along each ray, walked by the oracle
    lam = np.stack([i0[j] * np.exp(-O.forward_rays(G, rw * mw[j] + rb * mb[j], ids)) for j in range(len(E))])
    yref = O.poly_neglog((resp[:, None] * lam).sum(0), (resp[:, None] * i0).sum(0), E)
    got = y.cpu().numpy().reshape(-1)[ids]
    assert lw.max() > 10 and lb.max() > 1
    assert np.max(np.abs(got - yref)) <= 1e-5 * max(1.0, yref.max())

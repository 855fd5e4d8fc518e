"""Pins of the oracle's polychromatic primary simulation (Sec. 2.1, "Primary
simulation", and the normalised primary data of Sec. 2.4): the water-bone split,
the detector response, the resp-weighted sum of per-energy Poisson draws and the
log normalisation, against what the paper states (continuity, key points),
special cases that reduce to the pinned monochromatic sampler and projector,
a first-order expansion, beam hardening, and statistics."""
import numpy as np
import pytest

from paper_2512_21180_gb300 import inputs as I

MU_W = I.MU_WATER_60
TAU = (0.0, 1.2, 1.6)


def _split(O, rho_hat):
    return O.water_bone(np.asarray(rho_hat, dtype=np.float64) * MU_W, MU_W)


def test_water_bone_continuous_at_every_breakpoint(O):
    """The paper calls both densities continuous functions of rho_hat: at each
    breakpoint the two one-sided values agree (a dropped tau factor or swapped
    thresholds breaks this)."""
    for t in TAU:
        lo = _split(O, [t - 1e-9])
        hi = _split(O, [t + 1e-9])
        for a, b in zip(lo, hi):
            assert abs(a[0] - b[0]) < 1e-8, t


def test_water_bone_piecewise_linear_and_its_anchor_values(O):
    """Inside each interval both densities are linear in rho_hat (second
    differences vanish); the middle pieces are then fixed by continuity with the
    outer ones: rho_w runs from tau1 to 0 and rho_b from 0 to kappa_b tau2."""
    pieces = [(0.05, 1.15), (1.22, 1.58), (1.62, 4.0)]
    for a, b in pieces:
        r = np.linspace(a, b, 41)
        for d in _split(O, r):
            assert np.max(np.abs(np.diff(d, 2))) < 1e-12
    w, b = _split(O, [1.2, 1.6 - 1e-12, 1.6])
    assert w[0] == pytest.approx(1.2, abs=1e-9) and w[1] == pytest.approx(0.0, abs=1e-9) and w[2] == 0.0
    assert b[0] == pytest.approx(0.0, abs=1e-12) and b[1] == pytest.approx(0.409 * 1.6, abs=1e-9)


def test_water_bone_reproduces_soft_tissue_at_60_kev(O):
    """Below tau1 a voxel is pure water at relative density rho_hat, so
    rho_w mu_w(60) gives back the CT value exactly; air and negative values carry
    no material."""
    mu = np.linspace(0.0, 1.19 * MU_W, 200)
    w, b = O.water_bone(mu, MU_W)
    assert np.max(np.abs(w * MU_W - mu)) < 1e-15
    assert np.all(b == 0.0)
    w, b = O.water_bone(np.array([-0.01, -1e-6]), MU_W)
    assert np.all(w == 0.0) and np.all(b == 0.0)


def test_detector_response_key_points_and_linearity(O):
    """resp(20) = 5, resp(60) = 20, resp(120) = 10 (the paper's key points), linear
    in between; constant outside."""
    assert O.resp(20.0) == 5.0 and O.resp(60.0) == 20.0 and O.resp(120.0) == 10.0
    for a, b in [(20.0, 60.0), (60.0, 120.0)]:
        e = np.linspace(a, b, 13)
        r = np.array([O.resp(x) for x in e])
        assert np.max(np.abs(np.diff(r, 2))) < 1e-12
    assert O.resp(40.0) == pytest.approx(12.5) and O.resp(90.0) == pytest.approx(15.0)
    assert O.resp(5.0) == 5.0 and O.resp(150.0) == 10.0


def test_one_bin_reduces_to_the_monochromatic_sampler(O):
    """With one energy bin, unit water attenuation and no bone, the counts are the
    monochromatic sampler's (same counter of each element) and the reading is
    resp(e) times them."""
    p = I.line_integrals((4, 6, 5), seed=3, lo=0.0, hi=9.0)
    I0 = np.full((1, 6, 5), 3.0e4, dtype=np.float32)
    lam = O.poly_lam(p, np.zeros_like(p), [1.0], [0.0], I0)
    reading, counts = O.poly_reading(lam, [60.0], seed=77, noise=True, return_counts=True)
    ref = O.poisson(p, 3.0e4, seed=77).reshape(-1)
    assert np.array_equal(counts[:, 0], ref)
    assert np.array_equal(reading, 20.0 * ref)


def test_counter_of_bin_j_is_element_times_bins_plus_j(O):
    """Bin j of element i draws from the counter of element i ne + j: the counts
    equal the plain sampler run over the flattened [n][ne] means."""
    rng = np.random.default_rng(5)
    lam = rng.uniform(0.5, 3e4, size=(50, 10))
    lam[:, 3] = rng.uniform(0.1, 9.0, size=50)       # inversion branch too
    _, counts = O.poly_reading(lam, I.POLY_ENERGIES_KEV, seed=11, noise=True, return_counts=True)
    assert np.array_equal(counts.reshape(-1), O.poisson_lam(lam.reshape(-1), seed=11))


def _small_geom(O):
    g = dict(I.geometry("tiny16"))
    return O.Geom(g), g


def test_air_scan_normalises_to_zero(O):
    """An empty volume reads exactly the air reading: y_primary = 0."""
    G, g = _small_geom(O)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    _, y = O.poly_primary(G, np.zeros(G.vol_shape), MU_W, E, mw, mb, I0, seed=1, noise=False)
    assert np.max(np.abs(y)) == 0.0


def test_no_photons_read_as_one_photon_of_the_least_responsive_bin(O):
    """A reading of zero (every bin absorbed) is raised to min resp (one photon in
    the least responsive bin), so y = log(air / min resp) stays finite; readings
    above that floor are untouched."""
    E = I.POLY_ENERGIES_KEV
    air = np.array([[1.0e5, 3.0e4]])
    floor = min(O.resp(e) for e in E)
    y = O.poly_neglog(np.array([[0.0, 2.0 * floor]]), air, E)
    assert y[0, 0] == pytest.approx(np.log(1.0e5 / floor), rel=1e-15)
    assert y[0, 1] == pytest.approx(np.log(3.0e4 / (2.0 * floor)), rel=1e-15)
    assert floor == O.resp(25.0) and floor < O.resp(115.0)


def test_monochromatic_limit_is_the_projection(O):
    """One bin whose water attenuation is mu_w(60): for a soft-tissue volume the
    expected normalised data equal the cone-beam projection P(mu) of the pinned
    projector (exp / log, the gain, the split and the per-energy projection all
    cancel)."""
    G, g = _small_geom(O)
    v = I.smooth_volume(g["n"], seed=4).astype(np.float64)
    mu = 0.02 * v / v.max()
    assert mu.max() < 1.19 * MU_W
    I0 = I.poly_intensity(g)[4:5]
    _, y = O.poly_primary(G, mu, MU_W, [65.0], [MU_W], [0.07], I0, seed=1, noise=False)
    p = O.forward(G, mu)
    assert np.max(np.abs(y - p)) < 1e-12 * max(1.0, p.max())


def test_monochromatic_limit_with_bone(O):
    """Above tau2 a voxel is bone of relative density kappa_b rho_hat; with one bin
    whose bone attenuation is mu_w(60) / kappa_b such voxels again give back mu, so
    a volume of soft tissue and dense bone (no mixed voxels) projects to P(mu)."""
    G, g = _small_geom(O)
    v = I.smooth_volume(g["n"], seed=8).astype(np.float64)
    mu = 0.02 * v / v.max()
    mu[5:9, 6:11, 3:12] = 2.0 * MU_W
    mu[10:13, 2:5, 9:14] = 3.1 * MU_W
    I0 = I.poly_intensity(g)[2:3]
    _, y = O.poly_primary(G, mu, MU_W, [45.0], [MU_W], [MU_W / 0.409], I0, seed=1, noise=False)
    p = O.forward(G, mu)
    assert np.max(np.abs(y - p)) < 1e-12 * max(1.0, p.max())


def test_two_projections_equal_the_per_energy_projections(O):
    """P is linear, so mu_w(e) P(rho_w) + mu_b(e) P(rho_b) (two projections, the
    GPU's route) gives the per-energy projections' mean counts up to the FP32
    rounding of the two line integrals."""
    G, g = _small_geom(O)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    mu = O.phantom(G, I.ellipsoids(g, seed=12, n_soft=6, n_bone=2, n_air=1))
    rw, rb = O.water_bone(mu, MU_W)
    assert rb.max() > 0.5 and rw.max() > 0.5
    lam = O.poly_lam(O.forward(G, rw), O.forward(G, rb), mw, mb, I0)
    ref = np.stack([I0[j] * np.exp(-O.forward(G, rw * mw[j] + rb * mb[j])) for j in range(len(E))], -1)
    assert np.max(np.abs(lam - ref.reshape(lam.shape)) / ref.reshape(lam.shape)) < 1e-5


def test_thin_limit_is_the_weighted_mean_attenuation(O):
    """First order in the thickness: y = sum_e w_e P(mu_tilde_e) with
    w_e = resp(e) I0_e / sum resp I0, so for a thin water volume
    y / P(rho_w) -> sum_e w_e mu_w(e) (catches a missing resp weight, or tables
    paired with the wrong bins)."""
    G, g = _small_geom(O)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    eps = 1e-7
    rho = eps * (0.5 + I.smooth_volume(g["n"], seed=6).astype(np.float64))
    _, y = O.poly_primary(G, rho * MU_W, MU_W, E, mw, mb, I0, seed=1, noise=False)
    L = O.forward(G, rho)
    wts = np.array([O.resp(e) for e in E])[:, None, None] * I0.astype(np.float64)
    mean_mu = (wts * mw[:, None, None]).sum(0) / wts.sum(0)
    m = L > 1e-3 * L.max()
    rel = np.abs(y[m] / L[m] - np.broadcast_to(mean_mu, L.shape)[m]) / mean_mu.max()
    assert rel.max() < 1e-5


def test_beam_hardening(O):
    """Polychromatic data are sub-linear in the amount of water (the soft bins are
    absorbed first): y(2 mu) < 2 y(mu) wherever the ray meets the object, and the
    effective attenuation lies between the hardest and the softest bin's."""
    G, g = _small_geom(O)
    E, mw, mb, _ = I.poly_tables()
    I0 = I.poly_intensity(g)
    mu = np.zeros(G.vol_shape)
    mu[4:12, 4:12, 4:12] = 0.5 * MU_W     # half-density water; doubled it stays water
    _, y1 = O.poly_primary(G, mu, MU_W, E, mw, mb, I0, seed=1, noise=False)
    _, y2 = O.poly_primary(G, 2 * mu, MU_W, E, mw, mb, I0, seed=1, noise=False)
    L = O.forward(G, mu / MU_W)
    m = L > 1.0
    assert np.all(y2[m] < 2 * y1[m] * (1 - 1e-6))
    assert np.all(y1[m] >= mw.min() * L[m] * (1 - 1e-9))
    assert np.all(y1[m] <= mw.max() * L[m] * (1 + 1e-9))


def test_noisy_reading_moments(O):
    """Mean and variance of the reading over many pixels with equal means:
    E = sum resp lam, Var = sum resp^2 lam (independent Poisson draws per bin)."""
    E, _, _, s = I.poly_tables()
    lam_row = 2.0e4 * s
    lam_row[0] = 4.0                      # one bin on the inversion branch
    n = 40000
    lam = np.tile(lam_row, (n, 1))
    r = O.poly_reading(lam, E, seed=2024, noise=True)
    resp = np.array([O.resp(e) for e in E])
    mean, var = (resp * lam_row).sum(), (resp ** 2 * lam_row).sum()
    assert abs(r.mean() - mean) < 4.0 * np.sqrt(var / n)
    assert abs(r.var() / var - 1.0) < 0.04

"""Pins of the multiscale reference (coarse level, pooling, upsampling) against closed
forms, exact identities and the projector physics."""
import numpy as np
import torch

from paper_2512_21180_gb300 import inputs as I


def test_pool_of_upsampled_is_identity_and_adjoint():
    from oracle import multiscale_ref as S
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 6))
    assert np.array_equal(S.vol_down(S.up(x)), x)
    y = rng.standard_normal((3, 8, 10, 12))
    # <up x, y> = <x, up^T y> with up^T = 8 x (2x2x2 mean)
    assert abs(np.vdot(S.up(x), y) - np.vdot(x, 8.0 * S.vol_down(y))) <= 1e-12 * np.abs(y).sum()


def test_pool_closed_forms():
    from oracle import multiscale_ref as S
    i, j, k = np.meshgrid(np.arange(8.0), np.arange(6.0), np.arange(4.0), indexing="ij")
    x = 3.0 * i - 2.0 * j + 0.5 * k + 1.0
    ic, jc, kc = np.meshgrid(np.arange(4.0), np.arange(3.0), np.arange(2.0), indexing="ij")
    # the mean of a linear function over a 2x2x2 block is its value at the block centre
    assert np.allclose(S.vol_down(x), 3.0 * (2 * ic + 0.5) - 2.0 * (2 * jc + 0.5) + 0.5 * (2 * kc + 0.5) + 1.0,
                       atol=1e-12)
    # projections: every second angle, 2x2 pixel means
    a, v, u = np.meshgrid(np.arange(6.0), np.arange(4.0), np.arange(8.0), indexing="ij")
    y = 100.0 * a + 10.0 * v + u
    ac, vc, uc = np.meshgrid(np.arange(3.0), np.arange(2.0), np.arange(4.0), indexing="ij")
    assert np.allclose(S.proj_down(y), 100.0 * (2 * ac) + 10.0 * (2 * vc + 0.5) + (2 * uc + 0.5), atol=1e-12)
    y2 = y.copy()
    y2[1::2] = -7.0        # odd angles are not used
    assert np.array_equal(S.proj_down(y2), S.proj_down(y))


def test_coarse_level_sees_the_same_object(O):
    """The coarse geometry's projection of the pooled volume equals the fine projection
    binned 2x2 at every second angle, up to the two discretisations (smooth object):
    a wrong panel offset, pixel centre or angle pairing breaks it by far more."""
    from oracle import multiscale_ref as S
    gf = I.scaled(I.geometry("lpd128"), n=(64, 64, 48), n_angles=40, nu=128, nv=96, du=3.2, dv=3.2)
    gc = S.coarse_geometry(gf)
    Gf, Gc = O.Geom(gf), O.Geom(gc)
    x = I.smooth_volume(gf["n"], 3).astype(np.float64)
    pf = O.forward(Gf, x)
    pc = O.forward(Gc, S.vol_down(x))
    d = S.proj_down(pf)
    rel = np.linalg.norm(pc - d) / np.linalg.norm(d)
    assert rel < 0.05, rel
    # controls: a mismatched angle pairing or a shifted panel is far off
    assert np.linalg.norm(pc - S.proj_down(pf[np.r_[1:40, 0]])) / np.linalg.norm(d) > 3 * rel
    gs = dict(gc, u_offset=gc["u_offset"] + gc["du"])
    ps = O.forward(O.Geom(gs), S.vol_down(x))
    assert np.linalg.norm(ps - d) / np.linalg.norm(d) > 3 * rel


def test_two_level_reference_runs_and_uses_the_coarse_state(O):
    """With zero fine-level weights the fine level passes its initial state through, so
    the two-level output equals the upsampled coarse output."""
    from oracle import multiscale_ref as S
    gf = I.scaled(I.geometry("tiny16"), n=(8, 8, 8), nu=12, nv=8, du=6.0, dv=6.0, n_angles=8, u_offset=4.0)
    gc = S.coarse_geometry(gf)
    Gf, Gc = O.Geom(gf), O.Geom(gc)
    rng = np.random.default_rng(2)
    y = torch.tensor(rng.random(Gf.proj_shape))
    x0 = torch.tensor(rng.random(Gf.vol_shape))

    def params(shapes, seed, scale):
        r = np.random.default_rng(seed)
        return [(torch.tensor(r.standard_normal(s) * scale), torch.tensor(r.standard_normal(s[0]) * scale))
                for s in shapes]
    pc = ([params([(4, 5, 3, 3), (4, 4, 3, 3), (3, 4, 3, 3)], 1, 0.1)],
          [params([(4, 4, 3, 3, 3), (4, 4, 3, 3, 3), (3, 4, 3, 3, 3)], 2, 0.1)])
    pz = ([params([(4, 5, 3, 3), (4, 4, 3, 3), (3, 4, 3, 3)], 3, 0.0)],
          [params([(4, 4, 3, 3, 3), (4, 4, 3, 3, 3), (3, 4, 3, 3, 3)], 4, 0.0)])
    wc, wf = torch.tensor(O.redundancy(Gc)), torch.tensor(O.redundancy(Gf))
    x, xc = S.lpd_multiscale(Gc, Gf, y, x0, wc, wf, pc, pz, n_mem=3, mu_ref=0.5)
    assert torch.allclose(x, S.up(xc), atol=1e-12)
    assert torch.linalg.norm(xc - S.vol_down(x0)) > 1e-3   # the coarse level did something

"""The seeded workload recipes match the configurations they stand for: volume and
panel sizes, pitches, offsets, orbit, phantom composition and the field of view the
offset panels cover."""
import math

import numpy as np
import pytest

from paper_2512_21180_gb300 import inputs as I


def fov_radius(g):
    """Radius of the cylinder every angle sees, for a centred or offset flat panel: the
    far panel edge at u_max subtends asin(u_max / |(SDD, u_max)|) at the source."""
    u_max = g["u_offset"] + 0.5 * g["nu"] * g["du"]
    u_min = -g["u_offset"] + 0.5 * g["nu"] * g["du"]
    u = max(u_max, u_min) if g["u_offset"] else u_max
    return g["sid"] * u / math.hypot(g["sdd"], u)


@pytest.mark.parametrize("name,n,vox,nu,nv,du,off,na,batch", [
    ("small64", (64, 64, 64), 4.0, 96, 64, 1.6, 0.0, 64, 1),
    ("clinical", (256, 256, 192), 2.0, 512, 384, 0.8, 160.0, 400, 1),
    ("diff128", (128, 128, 128), 4.0, 256, 192, 1.6, 80.0, 200, 2),
    ("lpd128", (128, 128, 128), 4.0, 256, 192, 1.6, 80.0, 200, 1),
    ("coarse128", (128, 128, 96), 4.0, 256, 192, 1.6, 160.0, 200, 1),
])
def test_geometries(name, n, vox, nu, nv, du, off, na, batch):
    g = I.geometry(name)
    assert tuple(g["n"]) == n and tuple(g["vox"]) == (vox,) * 3
    assert (g["nu"], g["nv"], g["du"], g["dv"]) == (nu, nv, du, du)
    assert g["u_offset"] == off and g["v_offset"] == 0.0 and tuple(g["center"]) == (0.0, 0.0, 0.0)
    assert (g["sid"], g["sdd"], g["n_angles"], g["batch"]) == (1000.0, 1536.0, na, batch)


def test_multiscale_coarse_level_is_the_clinical_scan_halved():
    c, f = I.geometry("coarse128"), I.geometry("clinical")
    assert tuple(2 * v for v in c["n"]) == tuple(f["n"])
    assert c["vox"][0] == 2 * f["vox"][0]
    assert (2 * c["nu"], 2 * c["nv"], c["du"], c["n_angles"] * 2) == (f["nu"], f["nv"], 2 * f["du"], f["n_angles"])
    assert c["u_offset"] == f["u_offset"]


def test_fields_of_view():
    # half-fan panels: clinical covers ~231 mm, the 128^3 workloads ~182 mm
    assert fov_radius(I.geometry("clinical")) == pytest.approx(231.1, abs=0.2)
    assert fov_radius(I.geometry("lpd128")) == pytest.approx(182.3, abs=0.2)
    # the centred 96-column panel of the operator-test workload sees only ~50 mm
    assert fov_radius(I.geometry("small64")) == pytest.approx(49.9, abs=0.2)


def test_clinical_phantom_composition():
    p = I.phantom_params("clinical", 2)
    assert p.shape == (40, I.ELL_COLS)
    value, mode = p[:, 15], p[:, 16]
    assert mode[0] == 0 and value[0] == pytest.approx(0.02)                     # body
    soft = p[1:32]
    assert np.all(soft[:, 16] == 0) and np.all((soft[:, 15] >= 0.01) & (soft[:, 15] <= 0.03))
    assert np.all(mode[32:] == 1)                                                # overwrite inserts
    assert np.allclose(value[32:36], 0.04) and np.allclose(value[36:40], 0.0)    # 4 bone, 4 air


def test_small_phantom_ranges_and_rotations():
    p = I.phantom_params("small64", 1)
    assert p.shape == (10, I.ELL_COLS)
    axes = p[:, 3:6]
    assert np.all((axes >= 10.0) & (axes <= 100.0))
    assert np.all((p[:, 15] >= 0.01) & (p[:, 15] <= 0.03)) and np.all(p[:, 16] == 0)
    for row in p:
        R = row[6:15].reshape(3, 3)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)


def test_learned_workload_body_inside_the_field_of_view():
    g = I.geometry("lpd128")
    p = I.phantom_params("lpd128", 30_000)
    body = p[0]
    assert max(body[3], body[4]) < fov_radius(g)
    # every insert centre lies inside the cylinder it is drawn from (half-width x 0.5)
    r = np.hypot(p[1:, 0], p[1:, 1])
    assert np.all(r <= 0.5 * 0.5 * g["n"][0] * g["vox"][0] + 1e-9)


def test_seeded_draws_are_deterministic():
    a, b = I.phantom_params("clinical", 7), I.phantom_params("clinical", 7)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, I.phantom_params("clinical", 8))
    assert np.array_equal(I.random_normal((5, 7), 3), I.random_normal((5, 7), 3))

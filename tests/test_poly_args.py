"""Host-side argument checks of the polychromatic entry points (no GPU needed: every
case is rejected with CBCT_EINVAL before anything is launched or dereferenced on the
device)."""
import ctypes

import numpy as np
import pytest

EINVAL = -1
FAKE = ctypes.c_void_p(256)   # a device pointer that is never dereferenced


@pytest.fixture(scope="module")
def lib():
    from paper_2512_21180_gb300 import _lib, build
    build.build()
    return _lib.load()


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tables(ne=10):
    E = np.linspace(25.0, 115.0, ne)
    return E, np.full(ne, 0.02), np.full(ne, 0.05)


def test_detector_response_host_only(lib):
    E = np.array([20.0, 40.0, 60.0, 90.0, 120.0])
    out = np.zeros(5)
    assert lib.cbct_detector_response(_p(E), 5, _p(out)) == 0
    assert np.allclose(out, [5.0, 12.5, 20.0, 15.0, 10.0])
    assert lib.cbct_detector_response(_p(E), -1, _p(out)) == EINVAL
    assert lib.cbct_detector_response(None, 5, _p(out)) == EINVAL


@pytest.mark.parametrize("case", ["no_bins", "too_many_bins", "negative_energy", "nan_attenuation",
                                  "negative_attenuation", "null_tables", "null_input", "null_maps",
                                  "no_outputs", "counts_without_noise", "ragged_pixels", "zero_batch"])
def test_poly_reading_rejects(lib, case):
    ne = {"no_bins": 0, "too_many_bins": 17}.get(case, 10)
    E, mw, mb = _tables(max(ne, 1))
    if case == "negative_energy":
        E[3] = -1.0
    if case == "nan_attenuation":
        mw[2] = np.nan
    if case == "negative_attenuation":
        mb[0] = -0.01
    tabs = (None, None, None) if case == "null_tables" else (_p(E), _p(mw), _p(mb))
    L = None if case == "null_input" else FAKE
    I0 = None if case == "null_maps" else FAKE
    reading = None if case == "no_outputs" else FAKE
    y = None if case == "no_outputs" else FAKE
    counts = FAKE if case == "counts_without_noise" else None
    noise = 0 if case == "counts_without_noise" else 1
    npix = 7 if case == "ragged_pixels" else 12
    batch = 0 if case == "zero_batch" else 1
    rc = lib.cbct_poly_reading(L, batch, 3 * 12, npix, ne, *tabs, I0, 1, noise, reading, y, counts, None)
    assert rc == EINVAL, case
    assert lib.cbct_last_error()


def test_water_bone_rejects(lib):
    assert lib.cbct_water_bone(FAKE, 100, 1, 0.0, FAKE, None) == EINVAL      # mu_water60 must be > 0
    assert lib.cbct_water_bone(FAKE, 100, 1, float("nan"), FAKE, None) == EINVAL
    assert lib.cbct_water_bone(FAKE, 100, 0, 0.02, FAKE, None) == EINVAL     # batch >= 1
    assert lib.cbct_water_bone(None, 100, 1, 0.02, FAKE, None) == EINVAL
    assert lib.cbct_water_bone(FAKE, -1, 1, 0.02, FAKE, None) == EINVAL


def test_poly_simulate_rejects(lib):
    E, mw, mb = _tables()
    tabs = (_p(E), _p(mw), _p(mb))
    assert lib.cbct_poly_simulate(None, FAKE, 1, 0.02, 10, *tabs, FAKE, 1, 1, FAKE, FAKE, None) == EINVAL
    assert lib.cbct_poly_simulate(None, FAKE, 1, 0.02, 0, *tabs, FAKE, 1, 1, FAKE, FAKE, None) == EINVAL
    assert lib.cbct_poly_simulate(None, FAKE, 1, 0.02, 10, None, None, None, FAKE, 1, 1, FAKE, FAKE, None) == EINVAL

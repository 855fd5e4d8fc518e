"""back_project_noalloc: backprojection for callers that cannot allocate device
memory during the call (a framework that owns the whole device budget, or a
latency-critical loop that must stay out of the CUDA allocator). Called through
the C ABI and compared with back_project on two calls in a row.

Named to be collected last, so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the projector pair's relative-L2 bar used by every GPU test


@pytest.fixture(scope="module")
def env():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import _lib, projector
    return _lib, projector


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_noalloc_matches_back_project_twice(env):
    _lib, P = env
    lib = _lib.load()
    g = I.geometry("lpd128")          # 200 angles of 256 x 192: two chunks of the fixed scratch
    geom = P.Geometry(g)
    y = torch.tensor(I.random_volume((2,) + geom.proj_shape, 31), device="cuda")
    ref = P.back_project(geom, y)
    st = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((2,) + geom.vol_shape, float("nan"), device="cuda")
        _lib.check(lib.back_project_noalloc(geom.handle, y.data_ptr(), out.data_ptr(), 2, 0, st),
                   "back_project_noalloc")
        torch.cuda.synchronize()
        assert _rel(out, ref) <= TOL, (call, _rel(out, ref))
    # accumulate = 1 adds to what is there
    out2 = ref.clone()
    _lib.check(lib.back_project_noalloc(geom.handle, y.data_ptr(), out2.data_ptr(), 2, 1, st), "noalloc accumulate")
    torch.cuda.synchronize()
    assert _rel(out2, 2 * ref) <= TOL


def test_noalloc_rejects_oversized_projection(env):
    _lib, P = env
    lib = _lib.load()
    g = I.scaled(I.geometry("tiny16"), nu=4096, nv=2100, du=0.05, dv=0.05, n_angles=1)
    geom = P.Geometry(g)
    y = torch.zeros((1,) + geom.proj_shape, device="cuda")
    out = torch.zeros((1,) + geom.vol_shape, device="cuda")
    rc = lib.back_project_noalloc(geom.handle, y.data_ptr(), out.data_ptr(), 1, 0,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"exceeds the fixed scratch" in lib.cbct_last_error()

"""Failure handling of the pipelined kernels: a bounded wait that runs out sets the
device status word, the kernel returns, and reading the word with clear resets it.
The wait is made to expire on a barrier that nothing completes (no fault, no hang:
the limit is 1 ms of the GPU's global timer)."""
import time

import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TIMEOUT_CODE = 1   # the status value a kernel writes when its wait gives up


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import _lib, projector
    return _lib, projector


def test_bounded_wait_expires_and_status_clears(M):
    L, P = M
    geom = P.Geometry(I.geometry("tiny16"))
    assert geom.device_status(clear=True) == 0
    waited = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.check(L.load().cbct_wait_probe(geom.handle, 1_000_000, waited.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream), "cbct_wait_probe")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert waited.item() == 0            # no wait completed: the barrier never flipped
    assert dt < 1.0                      # the kernel returned after its short limit
    assert geom.device_status(clear=True) == TIMEOUT_CODE
    assert geom.device_status() == 0     # the clear reset the word
    # the context is still usable: a projection after the expired wait is correct
    x = torch.ones((1,) + geom.vol_shape, device="cuda")
    p = P.forward_project(geom, x)
    assert torch.isfinite(p).all() and p.max().item() > 0


def test_wait_probe_rejects_bad_limits(M):
    L, P = M
    geom = P.Geometry(I.geometry("tiny16"))
    waited = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for lim in (0, -5, 10 ** 9):
        assert L.load().cbct_wait_probe(geom.handle, lim, waited.data_ptr(), st) == -1
    assert L.load().cbct_wait_probe(geom.handle, 1000, None, st) == -1

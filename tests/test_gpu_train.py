"""Training-step kernels against the FP64 reference: the FoV-masked loss and its
gradient (cbct_masked_mse) element by element, and lpd_adam_step / lpd_clip_grads
over several steps on gradients the network's own backward produced."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

GEOM = I.scaled(I.geometry("tiny16"), n=(24, 24, 16), vox=(8.0, 8.0, 8.0), nu=40, nv=16, du=4.0, dv=4.0,
                n_angles=12, u_offset=20.0)


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import lpd, ops, projector
    return projector, lpd, ops


@pytest.mark.parametrize("n,thr", [(1, 0.5), (1000, 0.5), (128 ** 3, 0.5), (128 ** 3 + 77, 0.25), (4096, 2.0)])
def test_masked_mse_matches_reference(M, n, thr):
    """Loss and gradient over the voxels with V >= thr, sizes from one element to a
    128^3 volume with a ragged tail; thr 2 leaves the mask empty (loss and gradient 0)."""
    from oracle import train_ref as T
    _, L, _ = M
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    r = rng.standard_normal(n).astype(np.float32)
    V = rng.random(n).astype(np.float32)
    V[: max(1, n // 3)] = 1.0                 # a block of fully visible voxels
    loss, grad = L.masked_mse(to_gpu(x), to_gpu(r), to_gpu(V), thr)
    l_ref, g_ref = T.masked_mse(x, r, V, thr)
    if l_ref == 0.0:
        assert loss.item() == 0.0 and not torch.any(grad)
        return
    assert abs(loss.item() - l_ref) <= 1e-6 * l_ref
    assert rel_l2(to_np(grad), g_ref) <= 1e-6
    # no mask: every element counts
    loss_all, _ = L.masked_mse(to_gpu(x), to_gpu(r), None, thr, want_grad=False)
    assert abs(loss_all.item() - T.masked_mse(x, r)[0]) <= 1e-6 * T.masked_mse(x, r)[0]


def test_adam_and_clipping_match_reference(M):
    """Three steps of clip + Adam on the gradients of three backward passes: the
    parameters after each step equal the FP64 reference's element by element."""
    from oracle import train_ref as T
    P, L, _ = M
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=2, seed=5)
    theta = model.get_params().astype(np.float64)
    opt = T.Adam(model.nparams)
    lr, b1, b2, eps, scale, clip = 2e-3, 0.9, 0.99, 1e-8, 0.5, None
    for step in range(3):
        y = torch.tensor(I.random_volume(geom.proj_shape, 40 + step), device="cuda")
        x0 = torch.tensor(I.random_volume(geom.vol_shape, 50 + step), device="cuda")
        model.zero_grad()
        model.forward(y, x0, save_for_backward=True)
        model.backward(torch.tensor(I.random_normal(geom.vol_shape, 60 + step), device="cuda"))
        g = model.grads().astype(np.float64)
        if step == 1:
            # clip to half the current norm before the step (the library scales in place)
            n_ref, _ = T.clip_grads(g, 1.0, scale)
            clip = 0.5 * n_ref
            n_gpu = model.clip_grads(clip, grad_scale=scale)
            assert abs(n_gpu - n_ref) <= 1e-6 * n_ref
            g_clip = model.grads().astype(np.float64)
            _, g_ref = T.clip_grads(g, clip, scale)
            assert rel_l2(g_clip, g_ref) <= 1e-6
            g = g_clip
        model.adam_step(lr, b1, b2, eps, grad_scale=scale)
        new_ref = opt.step(theta, g, lr, b1, b2, eps, grad_scale=scale)
        got = model.get_params().astype(np.float64)
        assert rel_l2(got, new_ref) <= 1e-6, (step, rel_l2(got, new_ref))
        assert rel_l2(got - theta, new_ref - theta) <= 1e-4, (step, rel_l2(got - theta, new_ref - theta))
        theta = got

"""Learned primal-dual on the GPU (tcgen05 convs + projector pair) against the FP64
reference network with the same weights; gradients; a short training run."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

from gpu_util import grad_tol, rel_l2, to_gpu, to_np

pytestmark = pytest.mark.gpu

GEOM = I.scaled(I.geometry("tiny16"), n=(24, 24, 16), vox=(8.0, 8.0, 8.0), nu=40, nv=16, du=4.0, dv=4.0,
                n_angles=12, u_offset=20.0)


@pytest.fixture(scope="module")
def M():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import lpd, projector
    return projector, lpd


def oracle_params(flat, shapes):
    out, o = [], 0
    for cout, taps, cin in shapes:
        w = torch.tensor(flat[o:o + cout * taps * cin], dtype=torch.float64).reshape(cout, taps, cin)
        o += cout * taps * cin
        b = torch.tensor(flat[o:o + cout], dtype=torch.float64)
        o += cout
        k = (3, 3, 3) if taps == 27 else (3, 3)
        out.append((w.permute(0, 2, 1).reshape((cout, cin) + k).contiguous().requires_grad_(True),
                    b.clone().requires_grad_(True)))
    return out


# a larger, anisotropic case: 72 x 56 x 24 volume, 24 angles, 96 x 24 panel, 3 iterations
GEOM_L = I.scaled(I.geometry("tiny16"), n=(72, 56, 24), vox=(5.0, 5.0, 5.0), nu=96, nv=24, du=4.0, dv=4.0,
                  n_angles=24, u_offset=30.0)


def _lpd_case(O, M, last_scale, seed_w=3, width=32, gd=GEOM, n_iter=2):
    """GPU forward/backward and the FP64 reference (BF16 operands in both passes) on the
    24x24x16 / 12-angle case with 2 iterations (or the geometry and iteration count
    given); returns both sides' output and gradients and a function that re-evaluates the
    reference's gradients for a perturbed x0."""
    from oracle import lpd_ref as R
    P, L = M
    G = O.Geom(gd)
    geom = P.Geometry(gd)
    mu, bps = 0.02, 2e-3
    model = L.LPD(geom, n_iter=n_iter, mu_ref=mu, bp_scale=bps, width=width)
    shapes = L.layer_shapes(n_iter, width=width)
    flat = I.lpd_weights(shapes, seed=seed_w, last_scale=last_scale)
    model.set_params(flat)
    x_true = O.phantom(G, I.ellipsoids(gd, 5, n_soft=6, axes_mm=(15.0, 60.0)))
    y = O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 6).astype(np.float64)
    x0 = 0.8 * x_true + 0.002 * I.random_normal(G.vol_shape, 7).astype(np.float64)
    r = I.random_normal(G.vol_shape, 8).astype(np.float64)
    xg = model.forward(to_gpu(y), to_gpu(x0), save_for_backward=True)
    model.zero_grad()
    gy, g0 = model.backward(to_gpu(r), want_y=True, want_x0=True)
    gpu = (to_np(xg), model.grads().astype(np.float64), to_np(gy), to_np(g0))

    def reference(x0_scale=1.0):
        prm = oracle_params(flat, shapes)
        dual = [prm[6 * n:6 * n + 3] for n in range(n_iter)]
        prim = [prm[6 * n + 3:6 * n + 6] for n in range(n_iter)]
        yt = torch.tensor(y, requires_grad=True)
        x0t = torch.tensor(x0 * x0_scale, requires_grad=True)
        ref = R.lpd(G, yt, x0t, torch.tensor(O.redundancy(G)), dual, prim, n_mem=5, round_bf16=True, mu_ref=mu,
                    bp_scale=bps, round_grads=True)
        (ref * torch.tensor(r)).sum().backward()
        gref = np.concatenate([np.concatenate([w.grad.permute(0, *range(2, w.dim()), 1).reshape(-1).numpy(),
                                               b.grad.numpy()]) for w, b in prm])
        return ref.detach().numpy(), gref, yt.grad.numpy(), x0t.grad.numpy()
    return model, gpu, reference, (y, x0)


def test_lpd_forward_and_gradients_match_oracle(O, M):
    """Blocks at the library's initialisation scale (last layer of each block x 0.1):
    output, parameter gradient, dL/dy and dL/dx0 within the 1e-2 bar of BF16 blocks."""
    model, (xg, gg, gy, g0), reference, (y, x0) = _lpd_case(O, M, 0.1)
    ref, gref, gyr, g0r = reference()
    _, gp, gyp, g0p = reference(1.0 + 1e-6)
    assert rel_l2(xg, ref) <= 1e-2
    assert rel_l2(ref, x0) > 1e-4          # the network changed its input: the check is not vacuous
    e_w, e_y, e_x = rel_l2(gg, gref), rel_l2(gy, gyr), rel_l2(g0, g0r)
    print(f"LPD gradient parity: params {e_w:.2e}, y {e_y:.2e} (tol {grad_tol(gyr, gyp):.2e}), x0 {e_x:.2e}")
    assert e_w <= 1e-2, e_w
    assert e_x <= 1e-2, e_x
    assert e_y <= grad_tol(gyr, gyp), e_y
    # an inference pass (no stored states; the zero initial dual memory is never read)
    # runs the same arithmetic as the training pass above
    xi = model.forward(to_gpu(y), to_gpu(x0))
    assert np.array_equal(to_np(xi), xg)


def test_lpd_larger_case_matches_oracle(O, M):
    """72 x 56 x 24 voxels, 24 angles of a 96 x 24 panel, 3 iterations: projection images
    and volume rows of several widths, more angles per dual launch; output and gradients
    within the same bars."""
    model, (xg, gg, gy, g0), reference, _ = _lpd_case(O, M, 0.1, gd=GEOM_L, n_iter=3)
    ref, gref, gyr, g0r = reference()
    _, gp, gyp, g0p = reference(1.0 + 1e-6)
    assert rel_l2(xg, ref) <= 1e-2
    e_w, e_y, e_x = rel_l2(gg, gref), rel_l2(gy, gyr), rel_l2(g0, g0r)
    print(f"LPD 72x56x24 gradient parity: params {e_w:.2e} (tol {grad_tol(gref, gp):.2e}), y {e_y:.2e} "
          f"(tol {grad_tol(gyr, gyp):.2e}), x0 {e_x:.2e} (tol {grad_tol(g0r, g0p):.2e})")
    assert e_w <= grad_tol(gref, gp) and e_x <= grad_tol(g0r, g0p) and e_y <= grad_tol(gyr, gyp)


def test_lpd_width64_matches_oracle(O, M):
    """Blocks of width 64 (64-slot activations: 3x3 dual and 3x3x3 primal convolutions on
    64 input slots, each hidden layer as two launches of 32 outputs, weight gradients in
    32 x 32 blocks): output and gradients within the same bars as width 32."""
    _, (xg, gg, gy, g0), reference, _ = _lpd_case(O, M, 0.1, width=64)
    ref, gref, gyr, g0r = reference()
    _, gp, gyp, g0p = reference(1.0 + 1e-6)
    assert rel_l2(xg, ref) <= 1e-2
    e_w, e_y, e_x = rel_l2(gg, gref), rel_l2(gy, gyr), rel_l2(g0, g0r)
    print(f"LPD width 64 gradient parity: params {e_w:.2e}, y {e_y:.2e} (tol {grad_tol(gyr, gyp):.2e}), "
          f"x0 {e_x:.2e}")
    assert e_w <= grad_tol(gref, gp) and e_x <= grad_tol(g0r, g0p) and e_y <= grad_tol(gyr, gyp)


def test_lpd_strong_blocks_within_reference_conditioning(O, M):
    """Blocks five times stronger (last layer x 0.5): BF16 roundings of activations then
    decide the gradient at the FP32 rounding scale — the FP64 reference's own gradient
    moves by s under a 1e-6 relative change of x0. The GPU output keeps the 1e-2 bar; its
    gradients must agree within max(1e-2, 2 s)."""
    _, (xg, gg, gy, g0), reference, _ = _lpd_case(O, M, 0.5)
    ref, gref, gyr, g0r = reference()
    _, gp, gyp, g0p = reference(1.0 + 1e-6)
    assert rel_l2(xg, ref) <= 1e-2
    for name, got, want, pert in (("params", gg, gref, gp), ("y", gy, gyr, gyp), ("x0", g0, g0r, g0p)):
        e = rel_l2(got, want)
        print(f"strong blocks, {name}: GPU {e:.2e}, reference moved by {rel_l2(pert, want):.2e} under 1e-6")
        assert e <= grad_tol(want, pert), (name, e)


def test_lpd_training_reduces_loss(O, M):
    """A few Adam steps on simulated phantoms reduce the FoV-masked loss."""
    P, L = M
    from paper_2512_21180_gb300 import ops
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=3, seed=1)
    V = ops.fov(geom)
    data = []
    for s in range(4):
        x = ops.phantom(geom, I.ellipsoids(GEOM, 100 + s, n_soft=6, axes_mm=(15.0, 60.0)))
        _, y = ops.simulate(geom, x, 1e5, seed=s)
        x0 = ops.fdk(geom, y)[0]
        data.append((x, y[0], x0))
    def loss_all():
        tot = 0.0
        for x, y, x0 in data:
            out = model.forward(y, x0)
            tot += L.masked_mse(out, x, V, want_grad=False)[0].item()
        return tot
    l0 = loss_all()
    for it in range(30):
        model.zero_grad()
        for x, y, x0 in data:
            out = model.forward(y, x0, save_for_backward=True)
            _, g = L.masked_mse(out, x, V)
            model.backward(g)
        model.adam_step(1e-3, grad_scale=1.0 / len(data))
    l1 = loss_all()
    assert np.isfinite(l1) and l1 < 0.7 * l0, (l0, l1)


def test_gradient_clipping(O, M):
    """lpd_clip_grads: the returned norm is ||scale g||, the clipped gradient has norm
    max_norm, a small gradient is untouched, a non-finite one becomes zero."""
    P, L = M
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=1, seed=2)
    model.zero_grad()
    x = torch.rand(geom.vol_shape, device="cuda")
    y = torch.rand(geom.proj_shape, device="cuda")
    model.forward(y, x, save_for_backward=True)
    model.backward(torch.rand(geom.vol_shape, device="cuda"))
    g0 = model.grads().astype(np.float64)
    scale = 0.25
    n0 = float(np.linalg.norm(g0) * scale)
    n = model.clip_grads(1e30, grad_scale=scale)
    assert abs(n - n0) <= 1e-6 * n0
    assert np.array_equal(model.grads(), g0.astype(np.float32))      # below the limit: unchanged
    n = model.clip_grads(0.5 * n0, grad_scale=scale)
    g1 = model.grads().astype(np.float64)
    assert abs(np.linalg.norm(g1) * scale - 0.5 * n0) <= 1e-5 * n0
    model_params = model.get_params()
    # a non-finite gradient: set through a backward of a non-finite upstream gradient
    model.zero_grad()
    model.forward(y, x, save_for_backward=True)
    gx = torch.rand(geom.vol_shape, device="cuda")
    gx[0, 0, 0] = float("inf")
    model.backward(gx)
    n = model.clip_grads(1.0)
    assert not np.isfinite(n)
    assert not np.any(model.grads())
    assert np.array_equal(model.get_params(), model_params)


def test_trained_network_gains_over_fdk(M):
    """The committed weights (8 iterations with the data-residual channel, trained on 512
    phantoms of the learned workload by `experiment_lpd`) reconstruct unseen test
    phantoms far better than the FDK_w start the network is given."""
    import math
    import os
    P, L = M
    from paper_2512_21180_gb300 import ops
    import json
    wdir = os.path.join(os.path.dirname(L.__file__), "weights")
    with open(os.path.join(wdir, "lpd128.json")) as f:
        meta = json.load(f)
    g = I.geometry("lpd128")
    geom = P.Geometry(g)
    model = L.LPD(geom, n_iter=meta["n_iter"], n_mem=meta["n_mem"], residual_input=meta["residual_input"])
    model.set_params(np.load(os.path.join(wdir, meta["file"])))
    full = ops.fov(geom) >= 0.5

    def psnr(a, ref):
        mse = torch.mean((a[full] - ref[full]).double() ** 2).item()
        return 10 * math.log10(ref[full].max().item() ** 2 / mse)
    gains = []
    for j, s in enumerate((30_000, 30_001, 30_002)):   # test seeds, disjoint from training (10_000+)
        x = ops.phantom(geom, I.phantom_params("lpd128", s))
        _, y = ops.simulate(geom, x, 1e5, seed=90_000 + j)
        x0 = ops.fdk(geom, y)[0]
        out = model.forward(y[0], x0)
        gains.append(psnr(out, x) - psnr(x0, x))
    assert min(gains) > 10.0, gains


def test_status_words_stay_clear(M):
    """After a forward and backward pass no kernel of the model or of its geometry
    gave up a bounded wait: both device status words read 0."""
    P, L = M
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=1, seed=2)
    y = torch.rand((1,) + geom.proj_shape, device="cuda")
    x0 = torch.rand((1,) + geom.vol_shape, device="cuda")
    out = model.forward(y[0], x0[0], save_for_backward=True)
    model.zero_grad()
    model.backward(torch.ones_like(out))
    assert model.device_status() == 0
    assert geom.device_status(clear=True) == 0


def test_lpd_batch_and_residual_channel_match_oracle(O, M):
    """A batch of two volumes through one lpd_forward / lpd_backward call, with the
    data-residual input channel: each volume's output, and the batch's summed
    parameter gradient, against two FP64 reference runs with the same weights."""
    from oracle import lpd_ref as R
    P, L = M
    G = O.Geom(GEOM)
    geom = P.Geometry(GEOM)
    n_iter, mu, bps = 2, 0.02, 2e-3
    model = L.LPD(geom, n_iter=n_iter, mu_ref=mu, bp_scale=bps, residual_input=True, max_batch=2)
    shapes = L.layer_shapes(n_iter, residual_input=True)
    assert shapes[0] == (32, 9, 8)
    flat = I.lpd_weights(shapes, seed=13, last_scale=0.1)
    model.set_params(flat)
    ys, x0s, rs = [], [], []
    for b in range(2):
        x_true = O.phantom(G, I.ellipsoids(GEOM, 21 + b, n_soft=6, axes_mm=(15.0, 60.0)))
        ys.append(O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 30 + b).astype(np.float64))
        x0s.append(0.8 * x_true + 0.002 * I.random_normal(G.vol_shape, 40 + b).astype(np.float64))
        rs.append(I.random_normal(G.vol_shape, 50 + b).astype(np.float64))
    xg = model.forward(to_gpu(np.stack(ys)), to_gpu(np.stack(x0s)), save_for_backward=True)
    assert tuple(xg.shape) == (2,) + G.vol_shape
    model.zero_grad()
    gy, g0 = model.backward(to_gpu(np.stack(rs)), want_y=True, want_x0=True)
    gg = model.grads().astype(np.float64)
    prm = oracle_params(flat, shapes)
    dual = [prm[6 * n:6 * n + 3] for n in range(n_iter)]
    prim = [prm[6 * n + 3:6 * n + 6] for n in range(n_iter)]
    w = torch.tensor(O.redundancy(G))
    def ref_run(b, x0_scale=1.0):
        yt = torch.tensor(ys[b], requires_grad=True)
        x0t = torch.tensor(x0s[b] * x0_scale, requires_grad=True)
        ref = R.lpd(G, yt, x0t, w, dual, prim, n_mem=5, round_bf16=True, mu_ref=mu, bp_scale=bps,
                    round_grads=True, residual_input=True)
        (ref * torch.tensor(rs[b])).sum().backward()
        return ref.detach().numpy(), yt.grad.numpy(), x0t.grad.numpy()
    for b in range(2):
        ref, gyr, g0r = ref_run(b)
        _, gyp, g0p = ref_run(b, 1.0 + 1e-6)
        e = rel_l2(to_np(xg[b]), ref)
        assert e <= 1e-2, (b, e)
        assert rel_l2(to_np(gy[b]), gyr) <= grad_tol(gyr, gyp), (b, rel_l2(to_np(gy[b]), gyr))
        assert rel_l2(to_np(g0[b]), g0r) <= grad_tol(g0r, g0p), b
    # the parameter gradient sums both volumes' reference runs (the first pair of calls)
    for p_ in prm:
        for t in p_:
            t.grad = None
    ref_run(0)
    ref_run(1)
    gref = np.concatenate([np.concatenate([wt.grad.permute(0, *range(2, wt.dim()), 1).reshape(-1).numpy(),
                                           bt.grad.numpy()]) for wt, bt in prm])
    e = rel_l2(gg, gref)
    print(f"batch-2 residual-channel gradient parity: {e:.2e}")
    assert e <= 1e-2, e
    # one volume of the batch alone gives the same output as in the batch
    x1 = model.forward(to_gpu(ys[1]), to_gpu(x0s[1]))
    assert rel_l2(to_np(x1), to_np(xg[1])) <= 1e-4

"""Reversible learned primal-dual (additive coupling + channel permutations) on the
GPU against the FP64 reference: output, gradients, the recovery of the initial states
by the backward pass (no stored iterates), the permutation table, and device memory
against the stored-iterate model at the learned workload's size."""
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


@pytest.mark.parametrize("n_mem,res", [(6, True), (8, False)])
def test_reversible_matches_oracle_and_inverts(O, M, n_mem, res):
    from oracle import lpd_ref as R
    P, L = M
    G = O.Geom(GEOM)
    geom = P.Geometry(GEOM)
    n_iter, mu, bps = 3, 0.02, 2e-3
    model = L.LPD(geom, n_iter=n_iter, n_mem=n_mem, mu_ref=mu, bp_scale=bps, residual_input=res, reversible=True,
                  seed=7)
    perms = model.perms()
    assert all(R.mixes_halves(p) for p in perms.reshape(-1, n_mem))
    shapes = L.layer_shapes(n_iter, n_mem, residual_input=res, reversible=True)
    flat = I.lpd_weights(shapes, seed=17, last_scale=0.1)
    model.set_params(flat)
    x_true = O.phantom(G, I.ellipsoids(GEOM, 5, n_soft=6, axes_mm=(15.0, 60.0)))
    y = O.forward(G, x_true) + 0.01 * I.random_normal(G.proj_shape, 6).astype(np.float64)
    x0 = 0.8 * x_true + 0.002 * I.random_normal(G.vol_shape, 7).astype(np.float64)
    r = I.random_normal(G.vol_shape, 8).astype(np.float64)

    xg = model.forward(to_gpu(y), to_gpu(x0), save_for_backward=True)
    fN, hN = model.state()
    prm = oracle_params(flat, shapes)
    dual = [prm[6 * n:6 * n + 3] for n in range(n_iter)]
    prim = [prm[6 * n + 3:6 * n + 6] for n in range(n_iter)]
    yt = torch.tensor(y, requires_grad=True)
    x0t = torch.tensor(x0, requires_grad=True)
    w = torch.tensor(O.redundancy(G))
    ref, f_ref, h_ref = R.lpd_reversible(G, yt, x0t, w, dual, prim, perms[:, 0], perms[:, 1], n_mem=n_mem,
                                         mu_ref=mu, bp_scale=bps, round_grads=True, residual_input=res,
                                         return_state=True)
    assert rel_l2(to_np(xg), ref.detach().numpy()) <= 1e-2
    assert rel_l2(to_np(fN), f_ref.detach().numpy()) <= 1e-2
    assert rel_l2(to_np(hN), h_ref.detach().numpy()) <= 1e-2
    assert rel_l2(ref.detach().numpy(), x0) > 1e-4

    (ref * torch.tensor(r)).sum().backward()
    model.zero_grad()
    gy, g0 = model.backward(to_gpu(r), want_y=True, want_x0=True)
    gg = model.grads().astype(np.float64)
    gref = np.concatenate([np.concatenate([wt.grad.permute(0, *range(2, wt.dim()), 1).reshape(-1).numpy(),
                                           bt.grad.numpy()]) for wt, bt in prm])
    e_w, e_y, e_x = rel_l2(gg, gref), rel_l2(to_np(gy), yt.grad.numpy()), rel_l2(to_np(g0), x0t.grad.numpy())
    # the reference's own y gradient under a 1e-6 relative change of x0 sets its tolerance
    yp = torch.tensor(y, requires_grad=True)
    prm2 = oracle_params(flat, shapes)
    refp = R.lpd_reversible(G, yp, torch.tensor(x0 * (1 + 1e-6)), w,
                            [prm2[6 * n:6 * n + 3] for n in range(n_iter)],
                            [prm2[6 * n + 3:6 * n + 6] for n in range(n_iter)],
                            perms[:, 0], perms[:, 1], n_mem=n_mem, mu_ref=mu, bp_scale=bps, round_grads=True,
                            residual_input=res)
    (refp * torch.tensor(r)).sum().backward()
    tol_y = grad_tol(yt.grad.numpy(), yp.grad.numpy())
    print(f"reversible n_mem {n_mem}: gradient parity params {e_w:.2e}, y {e_y:.2e} (tol {tol_y:.2e}), x0 {e_x:.2e}")
    assert e_w <= 1e-2 and e_x <= 1e-2 and e_y <= tol_y, (e_w, e_y, e_x)

    # the backward pass undid every iteration: the states are the initial ones again,
    # f_0 = x0 / mu_ref in every channel and h_0 = 0, up to the FP32 roundings of the updates
    f0, h0 = model.state()
    want = torch.tensor(x0 / mu, dtype=torch.float32, device="cuda").expand_as(f0)
    ef = float((f0 - want).abs().max() / want.abs().max())
    eh = float(h0.abs().max() / hN.abs().max())
    print(f"reversible n_mem {n_mem}: recovered f_0 max err {ef:.2e}, h_0 max err {eh:.2e} (relative)")
    assert ef <= 1e-5 and eh <= 1e-5, (ef, eh)


def test_permutation_table_round_trip_and_checks(M):
    P, L = M
    geom = P.Geometry(GEOM)
    model = L.LPD(geom, n_iter=2, n_mem=6, reversible=True, seed=3)
    p = model.perms()
    assert p.shape == (2, 2, 6)
    q = p[:, ::-1].copy()                      # swap the primal and dual tables
    model.set_params(model.get_params())
    model.set_perms(q)
    assert np.array_equal(model.perms(), q)
    bad = q.copy()
    bad[0, 0] = [1, 0, 2, 4, 3, 5]             # a permutation that keeps the halves apart
    with pytest.raises(Exception):
        model.set_perms(bad)
    bad[0, 0] = [0, 0, 1, 2, 3, 4]             # not a permutation
    with pytest.raises(Exception):
        model.set_perms(bad)
    with pytest.raises(Exception):
        L.LPD(geom, n_iter=1, n_mem=5, reversible=True)   # odd memory


def test_reversible_model_needs_less_device_memory(M):
    """At the learned workload's size (128^3, 200 angles of 256x192), 8 iterations: the
    reversible model keeps one state instead of n_iter + 1 iterates and their projector
    outputs: the saving must be at least 90 % of those stored arrays' size."""
    P, L = M
    geom = P.Geometry(I.geometry("lpd128"))
    torch.cuda.synchronize()
    used = {}
    for name, kw in (("stored", dict(n_mem=6)), ("reversible", dict(n_mem=6, reversible=True))):
        free0 = torch.cuda.mem_get_info()[0]
        m = L.LPD(geom, n_iter=8, **kw)
        torch.cuda.synchronize()
        used[name] = free0 - torch.cuda.mem_get_info()[0]
        m.close()
        torch.cuda.synchronize()
    print(f"LPD device memory at 128^3, 8 iterations: stored iterates {used['stored'] / 2**30:.2f} GiB, "
          f"reversible {used['reversible'] / 2**30:.2f} GiB")
    nvox, nproj = 128 ** 3, 200 * 192 * 256
    stored_arrays = 4 * (8 * 6 * (nvox + nproj) + 8 * (nvox + nproj))   # 8 more iterates + P f, P^T h per iteration
    assert used["stored"] - used["reversible"] >= 0.9 * stored_arrays, (used, stored_arrays)

"""Pins of the reversible (additive coupling + permutation) learned primal-dual
reference: running the iterations backwards recovers the initial states, the update
of each half reads only the other half, the permutations must mix the halves, and
the gradient matches finite differences."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I

GEO = I.scaled(I.geometry("tiny16"), n=(8, 8, 6), nu=10, nv=6, du=6.0, dv=6.0, n_angles=6, u_offset=4.0)
M = 6
PERMS_F = [[3, 1, 4, 0, 5, 2], [5, 0, 3, 2, 1, 4]]
PERMS_H = [[4, 2, 0, 5, 1, 3], [1, 3, 5, 0, 2, 4]]


def params(seed, res=False, scale=0.1):
    r = np.random.default_rng(seed)
    mk = lambda s: torch.tensor(r.standard_normal(s) * scale, requires_grad=True)
    K = M // 2
    dual = [[(mk((4, K + 2 + int(res), 3, 3)), mk(4)), (mk((4, 4, 3, 3)), mk(4)), (mk((K, 4, 3, 3)), mk(K))]
            for _ in range(2)]
    prim = [[(mk((4, K + 1, 3, 3, 3)), mk(4)), (mk((4, 4, 3, 3, 3)), mk(4)), (mk((K, 4, 3, 3, 3)), mk(K))]
            for _ in range(2)]
    return dual, prim


def setup(O):
    G = O.Geom(GEO)
    rng = np.random.default_rng(1)
    return G, torch.tensor(rng.random(G.proj_shape)), torch.tensor(rng.random(G.vol_shape)), \
        torch.tensor(O.redundancy(G))


def test_permutations_used_here_mix_halves():
    from oracle import lpd_ref as R
    assert all(R.mixes_halves(p) for p in PERMS_F + PERMS_H)
    assert not R.mixes_halves([1, 0, 2, 5, 3, 4])


@pytest.mark.parametrize("res", [False, True])
def test_inverse_recovers_initial_states(O, res):
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    dual, prim = params(2, res)
    mu, bps = 0.5, 0.05
    out, f, h = R.lpd_reversible(G, y, x0, w, dual, prim, PERMS_F, PERMS_H, n_mem=M, mu_ref=mu, bp_scale=bps,
                                 residual_input=res, return_state=True)
    f0, h0 = R.lpd_reversible_inverse(G, y, f.detach(), h.detach(), w, dual, prim, PERMS_F, PERMS_H, n_mem=M,
                                      mu_ref=mu, bp_scale=bps, residual_input=res)
    ref_f = (x0 / mu).unsqueeze(0).repeat(M, 1, 1, 1)
    assert torch.allclose(f0, ref_f, rtol=0, atol=1e-12 * ref_f.abs().max().item())
    assert h0.abs().max().item() <= 1e-12 * max(1.0, h.abs().max().item())
    # the network acted: the final states differ from the initial ones
    assert (f.detach() - ref_f[list(np.arange(M))]).abs().max().item() > 1e-3


def test_zero_blocks_and_half_updates(O):
    """Zero weights and biases leave the states untouched (output x0); a change to the
    dual weights does not alter the first dual half in the first iteration's update, only
    d2 (checked through the states before any permutation by using identity perms)."""
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    zero = lambda t: torch.zeros_like(t)
    dual, prim = params(3)
    dz = [[(zero(a), zero(b)) for a, b in blk] for blk in dual]
    pz = [[(zero(a), zero(b)) for a, b in blk] for blk in prim]
    out = R.lpd_reversible(G, y, x0, w, dz, pz, PERMS_F, PERMS_H, n_mem=M, mu_ref=0.5, bp_scale=0.05)
    assert torch.allclose(out, x0, rtol=0, atol=1e-15)
    ident = [list(range(M))] * 2
    _, f, h = R.lpd_reversible(G, y, x0, w, dual[:1], prim[:1], ident[:1], ident[:1], n_mem=M, mu_ref=0.5,
                               bp_scale=0.05, return_state=True)
    assert h[:M // 2].abs().max().item() == 0.0              # d1 untouched (starts at 0)
    assert h[M // 2:].abs().max().item() > 0.0               # d2 updated
    assert torch.equal(f[:M // 2], (x0 / 0.5).unsqueeze(0).repeat(M // 2, 1, 1, 1))   # p1 untouched


def test_reversible_gradient_by_finite_differences(O):
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    dual, prim = params(4, True)
    run = lambda: R.lpd_reversible(G, y, x0, w, dual, prim, PERMS_F, PERMS_H, n_mem=M, round_bf16=False,
                                   mu_ref=0.5, bp_scale=0.05, residual_input=True).pow(2).sum()
    run().backward()
    eps = 1e-6
    for t, i in ((prim[1][0][0], (1, 2, 1, 0, 2)), (dual[0][0][0], (2, 4, 1, 1)), (dual[1][2][1], (1,))):
        g = t.grad[i].item()
        with torch.no_grad():
            t[i] += eps
            lp = run().item()
            t[i] -= 2 * eps
            lm = run().item()
            t[i] += eps
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (fd, g)


def lire_params(seed, K, n_iter=2, scale=0.1):
    r = np.random.default_rng(seed)
    mk = lambda s: torch.tensor(r.standard_normal(s) * scale, requires_grad=True)
    dual = [[(mk((4, K + 4, 3, 3, 3)), mk(4)), (mk((4, 4, 3, 3, 3)), mk(4)), (mk((K, 4, 3, 3, 3)), mk(K))]
            for _ in range(n_iter)]
    prim = [[(mk((4, K + 4, 3, 3, 3)), mk(4)), (mk((4, 4, 3, 3, 3)), mk(4)), (mk((K, 4, 3, 3, 3)), mk(K))]
            for _ in range(n_iter)]
    out = [(mk((2 * K,)), mk((1,))) for _ in range(n_iter)]
    return dual, prim, out


def test_lire_zero_blocks_reduce_to_the_output_convolution(O):
    """With zero blocks the latents keep their initial values (f alternating x0 / mu and
    s P^T(w y)), so each iteration adds mu (sum_c omega_c f_c + beta) to x: a closed form
    in terms of the initial channels, whatever the permutations."""
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    V = torch.tensor(O.fov(G))
    dual, prim, out = lire_params(5, M // 2)
    zero = lambda t: torch.zeros_like(t)
    dz = [[(zero(a), zero(b)) for a, b in blk] for blk in dual]
    pz = [[(zero(a), zero(b)) for a, b in blk] for blk in prim]
    mu, s = 0.5, 0.05
    got = R.lire(G, y, x0, w, V, dz, pz, out, PERMS_F, PERMS_H, n_mem=M, mu_ref=mu, bp_scale=s, round_bf16=False)
    xbp = s * torch.tensor(O.adjoint(G, (w.view(1, 1, -1) * y).numpy()))
    f = [x0 / mu if c % 2 == 0 else xbp for c in range(M)]
    perm = list(range(M))
    want = x0.clone()
    for n in range(2):
        om, be = out[n]
        want = want + mu * (sum(om[c].item() * f[perm[c]] for c in range(M)) + be.item())
        perm = [perm[p] for p in PERMS_F[n]]
    assert torch.allclose(got.detach(), want, rtol=1e-12, atol=1e-12)


def test_lire_landweber_term_is_the_data_gradient(O):
    """Only the primal block's Landweber input is nonzero (weight 1 from that channel to
    one hidden unit, identity-like path to p2[0], output conv reading that channel): the
    update is then a multiple of P^T(P x - y), the gradient of 1/2 ||P x - y||^2 — checked
    against the oracle's own operators applied by hand with a finite-difference gradient."""
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    V = torch.tensor(O.fov(G))
    K = M // 2
    dual, prim, out = lire_params(6, K, n_iter=1)
    zero = lambda t: torch.zeros_like(t)
    dz = [[(zero(a), zero(b)) for a, b in blk] for blk in dual]
    w1 = torch.zeros((4, K + 4, 3, 3, 3), dtype=torch.float64)
    w1[0, K + 2, 1, 1, 1] = 1.0                       # LW channel -> hidden unit 0 (centre tap)
    w2 = torch.zeros((4, 4, 3, 3, 3), dtype=torch.float64)
    w2[0, 0, 1, 1, 1] = 1.0
    w3 = torch.zeros((K, 4, 3, 3, 3), dtype=torch.float64)
    w3[0, 0, 1, 1, 1] = 1.0                           # -> p2[0]
    zb = lambda k: torch.zeros(k, dtype=torch.float64)
    prim = [[(w1, zb(4)), (w2, zb(4)), (w3, zb(K))]]
    om = torch.zeros(M, dtype=torch.float64)
    om[K] = 1.0                                        # x += mu * p2[0]
    out = [(om, zb(1))]
    mu, s = 0.5, 0.05
    ident = [list(range(M))]
    got = R.lire(G, y, x0, w, V, dz, prim, out, ident, ident, n_mem=M, mu_ref=mu, bp_scale=s, round_bf16=False)
    # by hand: LW = s P^T(P x0 - y); LeakyReLU keeps positive parts and scales negative ones
    lw = s * torch.tensor(O.adjoint(G, O.forward(G, x0.numpy()) - y.numpy()))
    act = lambda t: torch.where(t > 0, t, R.SLOPE * t)
    p2_0 = s * torch.tensor(O.adjoint(G, (w.view(1, 1, -1) * y).numpy())) if K % 2 == 1 else x0 / mu
    want = x0 + mu * (om[K] * (p2_0 + act(act(lw))))
    assert torch.allclose(got.detach(), want, rtol=1e-12, atol=1e-12)
    # and LW is the gradient of 1/2 ||P x - y||^2 (times s): central differences at one voxel
    i = (2, 3, 4)
    e = 1e-5
    xp, xm = x0.clone(), x0.clone()
    xp[i] += e
    xm[i] -= e
    phi = lambda v: 0.5 * float(np.sum((O.forward(G, v.numpy()) - y.numpy()) ** 2))
    assert abs((phi(xp) - phi(xm)) / (2 * e) * s - lw[i].item()) <= 1e-6 * max(1.0, abs(lw[i].item()))


def test_lire_gradient_by_finite_differences(O):
    from oracle import lpd_ref as R
    G, y, x0, w = setup(O)
    V = torch.tensor(O.fov(G))
    dual, prim, out = lire_params(7, M // 2)
    run = lambda: R.lire(G, y, x0, w, V, dual, prim, out, PERMS_F, PERMS_H, n_mem=M, round_bf16=False,
                         mu_ref=0.5, bp_scale=0.05).pow(2).sum()
    run().backward()
    eps = 1e-6
    for t, i in ((prim[1][0][0], (1, 2, 1, 0, 2)), (dual[0][0][0], (2, 4, 1, 1, 0)), (out[1][0], (3,)),
                 (out[0][1], (0,))):
        g = t.grad[i].item()
        with torch.no_grad():
            t[i] += eps
            lp = run().item()
            t[i] -= 2 * eps
            lm = run().item()
            t[i] += eps
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (fd, g)

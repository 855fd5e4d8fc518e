"""Pins of the FP64 learned-block reference: the library convolution is the
cross-correlation written out as a sum (brute force on small cases), and the
unrolled network's gradient agrees with finite differences."""
import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I


def brute_conv(x, w, b):
    """y[o, p] = b[o] + sum_{c, t} w[o, c, t] x[c, p + t - 1], zero outside."""
    spatial = x.shape[1:]
    xp = np.pad(x, [(0, 0)] + [(1, 1)] * len(spatial))
    y = np.zeros((w.shape[0],) + spatial)
    for o in range(w.shape[0]):
        y[o] = b[o]
        for idx in np.ndindex(*w.shape[2:]):
            sl = tuple(slice(i, i + n) for i, n in zip(idx, spatial))
            y[o] += np.tensordot(w[o][(slice(None),) + idx], xp[(slice(None),) + sl], axes=(0, 0))
    return y


@pytest.mark.parametrize("dims", [(5, 7), (4, 5, 6)])
def test_conv_is_cross_correlation(dims):
    from oracle import lpd_ref as R
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3,) + dims)
    w = rng.standard_normal((4, 3) + (3,) * len(dims))
    b = rng.standard_normal(4)
    got = R.conv(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b))[0].numpy()
    np.testing.assert_allclose(got, brute_conv(x, w, b), rtol=1e-12, atol=1e-12)


def test_bf16_rounding_is_round_to_nearest_even():
    from oracle import lpd_ref as R
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to even (1)
    v = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 3.0], dtype=torch.float64)
    assert R.bf16(v).tolist() == [1.0, 1.0 + 2.0 ** -6, 3.0]


def test_lpd_gradient_by_finite_differences(O):
    """The oracle network's parameter gradient (autograd through the FP64 projector
    pair) matches central differences on a tiny problem."""
    from oracle import lpd_ref as R
    g = I.scaled(I.geometry("tiny16"), n=(8, 8, 6), nu=10, nv=6, du=6.0, dv=6.0, n_angles=6, u_offset=4.0)
    G = O.Geom(g)
    rng = np.random.default_rng(1)
    y = torch.tensor(rng.random(G.proj_shape))
    x0 = torch.tensor(rng.random(G.vol_shape))
    w = torch.tensor(O.redundancy(G))

    def params(shapes, seed):
        r = np.random.default_rng(seed)
        return [(torch.tensor(r.standard_normal(s) * 0.1, requires_grad=True),
                 torch.tensor(r.standard_normal(s[0]) * 0.1, requires_grad=True)) for s in shapes]
    dual = [params([(4, 5, 3, 3), (4, 4, 3, 3), (3, 4, 3, 3)], 2)]
    prim = [params([(4, 4, 3, 3, 3), (4, 4, 3, 3, 3), (3, 4, 3, 3, 3)], 3)]
    loss = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=False, mu_ref=0.5, bp_scale=0.05).pow(2).sum()
    loss.backward()
    wt = prim[0][1][0]
    i = (1, 2, 1, 0, 2)
    eps = 1e-6
    with torch.no_grad():
        wt[i] += eps
        lp = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=False, mu_ref=0.5, bp_scale=0.05).pow(2).sum().item()
        wt[i] -= 2 * eps
        lm = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=False, mu_ref=0.5, bp_scale=0.05).pow(2).sum().item()
        wt[i] += eps
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - wt.grad[i].item()) <= 1e-6 * max(1.0, abs(fd))
    wd = dual[0][0][0]
    j = (2, 4, 1, 1)
    with torch.no_grad():
        wd[j] += eps
        lp = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=False, mu_ref=0.5, bp_scale=0.05).pow(2).sum().item()
        wd[j] -= 2 * eps
        lm = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=False, mu_ref=0.5, bp_scale=0.05).pow(2).sum().item()
        wd[j] += eps
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - wd.grad[j].item()) <= 1e-6 * max(1.0, abs(fd))


def test_residual_channel_is_the_data_residual(O):
    """The dual block's extra input is mu_ref P f_1 - y: with weights a, -a, +a on the
    residual, P f_1 and y channels its contribution cancels exactly (FP64, no rounding),
    and with zero residual weights the network equals the one without the channel."""
    from oracle import lpd_ref as R
    g = I.scaled(I.geometry("tiny16"), n=(8, 8, 6), nu=10, nv=6, du=6.0, dv=6.0, n_angles=6, u_offset=4.0)
    G = O.Geom(g)
    rng = np.random.default_rng(5)
    y = torch.tensor(rng.random(G.proj_shape))
    x0 = torch.tensor(rng.random(G.vol_shape))
    w = torch.tensor(O.redundancy(G))
    M = 3
    r = np.random.default_rng(6)
    mk = lambda s: torch.tensor(r.standard_normal(s) * 0.1)
    d_rest = [(mk((4, 4, 3, 3)), mk(4)), (mk((3, 4, 3, 3)), mk(3))]
    prim = [[(mk((4, 4, 3, 3, 3)), mk(4)), (mk((4, 4, 3, 3, 3)), mk(4)), (mk((3, 4, 3, 3, 3)), mk(3))]]
    w1, b1 = mk((4, M + 2, 3, 3)), mk(4)
    run = lambda first, res: R.lpd(G, y, x0, w, [[first] + d_rest], prim, n_mem=M, round_bf16=False, mu_ref=0.5,
                                   bp_scale=0.05, residual_input=res)
    base = run((w1, b1), False)
    # zero weights on the residual channel
    w1z = torch.cat([w1, torch.zeros((4, 1, 3, 3), dtype=torch.float64)], 1)
    assert torch.allclose(run((w1z, b1), True), base, rtol=0, atol=1e-13)
    # a (P f_1 - y) - a P f_1 + a y = 0
    a = mk((4, 1, 3, 3))
    w1c = torch.cat([w1[:, :M], w1[:, M:M + 1] - a, w1[:, M + 1:M + 2] + a, a], 1)
    assert torch.allclose(run((w1c, b1), True), base, rtol=0, atol=1e-12)
    # a wrong sign on y would not cancel
    w1x = torch.cat([w1[:, :M], w1[:, M:M + 1] - a, w1[:, M + 1:M + 2] - a, a], 1)
    assert (run((w1x, b1), True) - base).abs().max().item() > 1e-6

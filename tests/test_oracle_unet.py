"""Pins of the P4-equivariant U-Net primal block reference (p4_unet) and of the
weight-normalisation reference: exact equivariance (and its failure for untied
weights), the pooling / upsampling adjoint pair, the reduction to a plain layer chain
when the bottleneck is zero (which fixes the concatenation order), finite-difference
gradients, and closed-form properties of the normalisation."""
import numpy as np
import pytest
import torch

FB, K, CIN = 2, 3, 5


def unet_params(seed, scale=0.2, fb=FB, k=K, cin=CIN):
    g = torch.Generator().manual_seed(seed)
    mk = lambda *s: (torch.randn(*s, generator=g, dtype=torch.float64) * scale).requires_grad_(True)
    return [(mk(fb, cin, 3, 3, 3), mk(fb)), (mk(fb, fb, 4, 3, 3, 3), mk(fb)), (mk(2 * fb, fb, 4, 3, 3, 3), mk(2 * fb)),
            (mk(2 * fb, 2 * fb, 4, 3, 3, 3), mk(2 * fb)), (mk(fb, 3 * fb, 4, 3, 3, 3), mk(fb)),
            (mk(k, fb, 4, 3, 3, 3), mk(k))]


def vol(seed, shape=(2, CIN, 4, 6, 6)):
    return torch.tensor(np.random.default_rng(seed).standard_normal(shape))


@pytest.mark.parametrize("r", [1, 2, 3])
def test_unet_is_rotation_equivariant(r):
    from oracle import lpd_ref as R
    p = unet_params(1)
    x = vol(2)
    out = R.p4_unet(x, p, round_bf16=False)
    rot = R.p4_unet(R.rot_vol(x, r), p, round_bf16=False)
    assert (rot - R.rot_vol(out, r)).abs().max().item() <= 1e-12 * out.abs().max().item()
    assert (R.rot_vol(out, r) - out).abs().max().item() > 1e-3 * out.abs().max().item()   # not trivially symmetric


def test_untied_weights_break_equivariance(monkeypatch):
    """The same network with the group layers' full weights drawn freely (not tied by
    rotation) is not equivariant: the check above can fail."""
    from oracle import lpd_ref as R
    g = torch.Generator().manual_seed(9)
    real = R.p4_group

    def untied(w_base, b_base):
        w, b = real(w_base, b_base)
        return torch.randn(w.shape, generator=g, dtype=w.dtype) * 0.2, b
    monkeypatch.setattr(R, "p4_group", untied)
    x = vol(3)
    p = unet_params(4)
    out = R.p4_unet(x, p, round_bf16=False)
    g.manual_seed(9)
    rot = R.p4_unet(R.rot_vol(x), p, round_bf16=False)
    assert (rot - R.rot_vol(out)).abs().max().item() > 1e-3 * out.abs().max().item()


def test_pool_and_upsample_are_adjoint_up_to_the_block_size():
    from oracle import lpd_ref as R
    a = vol(5, (1, 3, 2, 3, 4))
    b = vol(6, (1, 3, 4, 6, 8))
    lhs = float((R.up2(a) * b).sum())
    rhs = 8.0 * float((a * R.pool2(b)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert torch.allclose(R.pool2(R.up2(a)), a, rtol=0, atol=1e-15)
    # pool2 is the plain mean of each 2 x 2 x 2 block
    assert abs(R.pool2(b)[0, 1, 1, 2, 3].item() - b[0, 1, 2:4, 4:6, 6:8].mean().item()) <= 1e-15


def test_zero_bottleneck_reduces_to_a_plain_chain():
    """With the half-resolution layers zero (weights and biases), up(r) = 0 and the block
    is lift -> g2 -> g5 -> avg6 with g5 reading only its last 4F inputs (the skip s): the
    concatenation puts up(r) first and s second."""
    from oracle import lpd_ref as R
    p = unet_params(7)
    with torch.no_grad():
        for i in (2, 3):
            p[i][0].zero_()
            p[i][1].zero_()
    x = vol(8)
    got = R.p4_unet(x, p, round_bf16=False)
    w5, b5 = R.p4_group(*p[4])
    chain = [R.p4_lift(*p[0]), R.p4_group(*p[1]), (w5[:, 8 * FB:], b5), R.p4_avg(*p[5])]
    want = R.block(x, chain, round_bf16=False)
    assert torch.allclose(got, want, rtol=1e-13, atol=1e-13)


def test_unet_gradient_by_finite_differences():
    from oracle import lpd_ref as R
    p = unet_params(10)
    x = vol(11)
    wr = vol(12, (2, K, 4, 6, 6))
    run = lambda: float((R.p4_unet(x, p, round_bf16=False) * wr).sum())
    (R.p4_unet(x, p, round_bf16=False) * wr).sum().backward()
    eps = 1e-6
    for t, i in ((p[0][0], (1, 2, 0, 1, 2)), (p[2][0], (3, 1, 2, 0, 1, 1)), (p[4][0], (1, 5, 3, 2, 2, 0)),
                 (p[3][1], (2,)), (p[5][0], (0, 1, 1, 1, 0, 2))):
        gval = t.grad[i].item()
        with torch.no_grad():
            t[i] += eps
            lp = run()
            t[i] -= 2 * eps
            lm = run()
            t[i] += eps
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gval) <= 1e-6 * max(1.0, abs(fd)), (fd, gval)


def test_weight_norm_closed_forms():
    """Each effective filter has zero mean and norm |gain|; shifting a filter by a constant
    or scaling it by a positive factor changes nothing; the gradient with respect to the raw
    filter sums to zero and is orthogonal to the centred filter; the forced step keeps the
    effective weights and sets every raw filter's norm to sqrt(fan-in)."""
    from oracle import lpd_ref as R
    g = torch.Generator().manual_seed(3)
    w = torch.randn(4, 6, 3, 3, 3, generator=g, dtype=torch.float64).requires_grad_(True)
    gain = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    e = R.weight_norm(w, gain)
    rows = e.reshape(4, -1)
    assert torch.allclose(rows.mean(1), torch.zeros(4, dtype=torch.float64), atol=1e-15)
    assert torch.allclose(rows.norm(dim=1), torch.full((4,), 0.7, dtype=torch.float64), rtol=1e-14)
    shifted = w.detach() * torch.tensor([2.0, 0.5, 3.0, 1.0], dtype=torch.float64).reshape(4, 1, 1, 1, 1) + 1.25
    assert torch.allclose(R.weight_norm(shifted, gain), e, rtol=1e-13, atol=1e-15)
    c = torch.randn(e.shape, generator=g, dtype=torch.float64)
    (e * c).sum().backward()
    gw = w.grad.reshape(4, -1)
    v = (w.detach() - w.detach().reshape(4, -1).mean(1).reshape(4, 1, 1, 1, 1)).reshape(4, -1)
    assert gw.sum(1).abs().max().item() <= 1e-12
    assert (gw * v).sum(1).abs().max().item() <= 1e-12 * gw.norm().item() * v.norm().item()
    assert abs(gain.grad.item() - float((e.detach() / 0.7 * c).sum())) <= 1e-12
    f = R.forced_renorm(w.detach())
    assert torch.allclose(f.reshape(4, -1).norm(dim=1), torch.full((4,), (6 * 27) ** 0.5, dtype=torch.float64))
    assert torch.allclose(R.weight_norm(f, gain.detach()), e.detach(), rtol=1e-13, atol=1e-15)

"""Pins of the training-step reference (Adam, FoV-masked loss, gradient clipping),
each against a closed form or a hand-computed case rather than the formula itself,
and of the bfloat16 rounding of gradient operands in the block reference."""
import math

import numpy as np
import pytest
import torch

from paper_2512_21180_gb300 import inputs as I


def test_adam_constant_gradient_moves_by_lr_each_step():
    """For a constant gradient the bias-corrected moments are exactly g and g^2, so
    every step moves each parameter by lr against the sign of its gradient. Without
    the bias correction step 1 would move by lr (1 - b1) / sqrt(1 - b2) = 3.16 lr."""
    from oracle import train_ref as T
    g = np.array([3.0, -0.5, 1e-3, -200.0])
    th = np.array([0.1, 0.2, -0.3, 0.0])
    opt = T.Adam(4)
    lr = 1e-3
    for t in range(1, 6):
        new = opt.step(th, g, lr, eps=0.0)
        np.testing.assert_allclose(new - th, -lr * np.sign(g), rtol=1e-12, atol=0)
        th = new


def test_adam_two_steps_by_hand():
    """g = +1 then -1 (beta1 0.9, beta2 0.999): step 1 moves by -lr; at step 2
    m = 0.09 - 0.1 = -0.01, v = 0.000999 + 0.001 = 0.001999, m_hat = -0.01 / 0.19 = -1/19,
    v_hat = 0.001999 / 0.001999 = 1, so step 2 moves by +lr / 19."""
    from oracle import train_ref as T
    opt = T.Adam(1)
    lr = 0.01
    th1 = opt.step(np.array([0.0]), np.array([1.0]), lr, eps=0.0)
    assert abs(th1[0] + lr) <= 1e-15
    th2 = opt.step(th1, np.array([-1.0]), lr, eps=0.0)
    assert abs((th2[0] - th1[0]) - lr / 19.0) <= 1e-14


def test_adam_zero_gradient_and_scale():
    from oracle import train_ref as T
    opt = T.Adam(2)
    th = np.array([1.0, -1.0])
    assert np.array_equal(opt.step(th, np.zeros(2), 0.1), th)          # eps keeps 0/0 at 0
    # grad_scale multiplies the gradient before both moments: sign-invariant at step 1
    a, b = T.Adam(2), T.Adam(2)
    g = np.array([2.0, -4.0])
    np.testing.assert_allclose(a.step(th, g, 0.1, eps=1e-8, grad_scale=0.25),
                               b.step(th, 0.25 * g, 0.1, eps=1e-8), rtol=0, atol=1e-15)


def test_masked_mse_closed_form_and_mask():
    """x - ref = c on the mask gives loss c^2 and gradient 2 c / count there; values
    off the mask (however wrong) change neither; an empty mask gives zeros."""
    from oracle import train_ref as T
    rng = np.random.default_rng(3)
    ref = rng.random((4, 5, 6))
    V = rng.random((4, 5, 6))
    mask = V >= 0.5
    c = 0.125
    x = ref + c
    x[~mask] += 1e3
    loss, grad = T.masked_mse(x, ref, V, 0.5)
    n = int(mask.sum())
    assert abs(loss - c * c) <= 1e-15
    assert np.allclose(grad.reshape(V.shape)[mask], 2 * c / n, rtol=1e-15, atol=0)
    assert not np.any(grad.reshape(V.shape)[~mask])
    l0, g0 = T.masked_mse(x, ref, np.zeros_like(V), 0.5)
    assert l0 == 0.0 and not np.any(g0)


def test_masked_mse_gradient_by_finite_differences():
    from oracle import train_ref as T
    rng = np.random.default_rng(4)
    x, ref, V = rng.random(50), rng.random(50), rng.random(50)
    _, g = T.masked_mse(x, ref, V, 0.3)
    h = 1e-6
    for i in (0, 7, 19, 33, 49):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (T.masked_mse(xp, ref, V, 0.3)[0] - T.masked_mse(xm, ref, V, 0.3)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-8


def test_clip_grads_norm_and_limit():
    from oracle import train_ref as T
    g = np.array([3.0, 4.0])                                       # norm 5
    n, c = T.clip_grads(g, 10.0, grad_scale=2.0)                   # ||2 g|| = 10: not above the limit
    assert n == 10.0 and np.array_equal(c, g)
    n, c = T.clip_grads(g, 1.0)
    assert n == 5.0 and np.allclose(c, [0.6, 0.8], rtol=1e-15)
    n, c = T.clip_grads(np.array([1.0, np.inf]), 1.0)
    assert not math.isfinite(n) and not np.any(c)


def test_round_grad_rounds_only_the_backward():
    """round_grad is the identity forward; its backward is the bfloat16 rounding of
    the incoming gradient (round to nearest even)."""
    from oracle import lpd_ref as R
    x = torch.tensor([0.3, -1.7, 2.5], dtype=torch.float64, requires_grad=True)
    c = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 0.1], dtype=torch.float64)
    y = R.round_grad(x)
    assert torch.equal(y.detach(), x.detach())
    (y * c).sum().backward()
    assert x.grad.tolist() == [1.0, 1.0 + 2.0 ** -6, R.bf16(torch.tensor(0.1, dtype=torch.float64)).item()]


def test_lpd_rounded_gradient_stays_near_exact_gradient(O):
    """With bfloat16 gradient operands the network's parameter gradient moves from the
    exact one only by the operand rounding (2^-9 relative per operand), far less than
    its own size: a dropped or misplaced rounding site that changed the gradient's
    structure would not."""
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

    def grads(round_grads):
        dual = [params([(4, 5, 3, 3), (4, 4, 3, 3), (3, 4, 3, 3)], 2)]
        prim = [params([(4, 4, 3, 3, 3), (4, 4, 3, 3, 3), (3, 4, 3, 3, 3)], 3)]
        out = R.lpd(G, y, x0, w, dual, prim, n_mem=3, round_bf16=True, mu_ref=0.5, bp_scale=0.05,
                    round_grads=round_grads)
        out.pow(2).sum().backward()
        return np.concatenate([t.grad.reshape(-1).numpy() for p in dual + prim for wb in p for t in wb])

    exact, rounded = grads(False), grads(True)
    rel = np.linalg.norm(rounded - exact) / np.linalg.norm(exact)
    assert 0 < rel <= 1e-2, rel


def test_bf16_operand_rounding_passes_the_gradient_through():
    """bf16() rounds the forward value only: the gradient reaches the master value
    unrounded (the GPU applies FP32 weight and input gradients to FP32 masters)."""
    from oracle import lpd_ref as R
    x = torch.tensor([0.3, 1.0 + 2.0 ** -8], dtype=torch.float64, requires_grad=True)
    y = R.bf16(x)
    assert y.tolist() == [R.bf16(torch.tensor(0.3, dtype=torch.float64)).item(), 1.0]
    (y * torch.tensor([1.001, -3.3], dtype=torch.float64)).sum().backward()
    assert x.grad.tolist() == [1.001, -3.3]

"""Pins of the P4-equivariant layers of the reference: the rotation is a rotation
(four of them are the identity, it moves voxels as written), a rotated filter on a
rotated volume gives the rotated result, and the three-layer block commutes with the
rotation exactly in FP64 while a block without the weight tying does not."""
import numpy as np
import torch


def test_rotation_moves_voxels_by_a_quarter_turn():
    from oracle import lpd_ref as R
    v = torch.arange(2 * 3 * 3, dtype=torch.float64).reshape(2, 3, 3)
    r = R.rot_vol(v)
    # (rho v)[z, y, x] = v[z, x, n - 1 - y]
    for z in range(2):
        for y in range(3):
            for x in range(3):
                assert r[z, y, x] == v[z, x, 2 - y]
    assert torch.equal(R.rot_vol(v, 4), v)
    assert not torch.equal(R.rot_vol(v, 2), v)


def test_rotated_filter_commutes_with_convolution():
    from oracle import lpd_ref as R
    rng = np.random.default_rng(0)
    v = torch.tensor(rng.standard_normal((1, 2, 5, 7, 7)))
    w = torch.tensor(rng.standard_normal((3, 2, 3, 3, 3)))
    lhs = R.conv(R.rot_vol(v), R.rot_filter(w, 1), None)
    rhs = R.rot_vol(R.conv(v, w, None))
    assert torch.allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_p4_block_is_equivariant():
    from oracle import lpd_ref as R
    rng = np.random.default_rng(1)
    mk = lambda *s: torch.tensor(rng.standard_normal(s) * 0.3)
    cin, c1, c2, cout = 6, 2, 2, 3
    params = [(mk(c1, cin, 3, 3, 3), mk(c1)), (mk(c2, c1, 4, 3, 3, 3), mk(c2)),
              (mk(cout, c2, 4, 3, 3, 3), mk(cout))]
    x = torch.tensor(rng.standard_normal((1, cin, 4, 6, 6)))
    y = R.p4_block(x, params, round_bf16=False)
    y_rot = R.p4_block(R.rot_vol(x), params, round_bf16=False)
    assert torch.allclose(y_rot, R.rot_vol(y), rtol=0, atol=1e-12)
    # the same layer sizes with untied weights are not equivariant
    full = [R.p4_lift(*params[0]), R.p4_group(*params[1]), R.p4_avg(*params[2])]
    untied = [(w + 0.1 * torch.tensor(rng.standard_normal(tuple(w.shape))), b) for w, b in full]
    z = R.block(x, untied, round_bf16=False)
    z_rot = R.block(R.rot_vol(x), untied, round_bf16=False)
    assert (z_rot - R.rot_vol(z)).abs().max().item() > 1e-3


def test_p4_group_layer_shifts_the_group_index():
    """A group layer maps rho (input with group index shifted by one) to rho (output with
    group index shifted by one): the defining property of the weight tying."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(2)
    ci, co = 2, 3
    w, b = R.p4_group(torch.tensor(rng.standard_normal((co, ci, 4, 3, 3, 3))), torch.zeros(co, dtype=torch.float64))
    u = torch.tensor(rng.standard_normal((1, ci * 4, 3, 5, 5)))
    shift = lambda t, c: t.reshape(1, c, 4, *t.shape[2:]).roll(1, dims=2).reshape(t.shape)   # (c, s) <- (c, s - 1)
    lhs = R.conv(R.rot_vol(shift(u, ci)), w, b)
    rhs = R.rot_vol(shift(R.conv(u, w, b), co))
    assert torch.allclose(lhs, rhs, rtol=0, atol=1e-12)

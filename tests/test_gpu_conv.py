"""Tensor-core convolutions (tcgen05) and their gradients against the FP64
reference on BF16-rounded operands."""
import zlib

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SLOPE = 0.2


@pytest.fixture(scope="module")
def L():
    from paper_2512_21180_gb300 import build
    build.build()
    from paper_2512_21180_gb300 import _lib
    return _lib


def to_cl(x, cp):
    """[N, C, *S] float64 -> BF16 row-blocked [N, *S[:-1], cp / 8, W, 8] on the GPU
    (channel slots >= C zero)."""
    n, c = x.shape[:2]
    y = torch.zeros((n,) + tuple(x.shape[2:]) + (cp,), dtype=torch.float64)
    y[..., :c] = x.movedim(1, -1)
    W = x.shape[-1]
    y = y.reshape(y.shape[:-2] + (W, cp // 8, 8)).transpose(-3, -2)
    return y.to(torch.bfloat16).cuda().contiguous()


def from_cl(y, c):
    """Inverse of to_cl: row-blocked [N, *S[:-1], cp / 8, W, 8] -> [N, c, *S] float64."""
    y = y.transpose(-3, -2)
    y = y.reshape(y.shape[:-2] + (-1,))
    return y[..., :c].double().movedim(-1, 1).cpu()


def run_conv(L, x_cl, dims, taps3d, w, b, cin, cout, flip, epi, cpout, mask=None, state=None):
    nimg = x_cl.shape[0]
    D, H, W = dims if taps3d else (1,) + dims
    n_out = cin if flip else cout
    W = x_cl.shape[-2]
    y = torch.zeros((nimg,) + tuple(x_cl.shape[1:-3]) + (cpout // 8, W, 8), dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sp = state.data_ptr() if state is not None else None
    ss = state[0].numel() if state is not None else 0
    rc = L.load().cbct_conv(x_cl.data_ptr(), nimg, D, H, W, x_cl.shape[-3] * 8, taps3d, w.data_ptr(),
                            b.data_ptr() if b is not None else None, cin, cout, flip, epi, SLOPE,
                            y.data_ptr(), cpout, mask.data_ptr() if mask is not None else None, sp, ss,
                            status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    L.check(rc, "cbct_conv")
    torch.cuda.synchronize()
    assert status.item() == 0
    return y


def rel(a, b):
    return float((a - b).norm() / b.norm())


CASES = [
    ("2d_7to32", (19, 37), 0, 7, 32, 3),
    ("2d_32to32", (16, 40), 0, 32, 32, 2),
    ("3d_6to32", (9, 10, 21), 1, 6, 32, 2),
    ("3d_32to32", (8, 12, 17), 1, 32, 32, 1),
]


@pytest.mark.parametrize("name,dims,taps3d,cin,cout,nimg", CASES)
def test_conv_forward_act(L, name, dims, taps3d, cin, cout, nimg):
    from oracle import lpd_ref as R
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 1000)
    x = torch.tensor(rng.standard_normal((nimg, cin) + dims))
    w = torch.tensor(rng.standard_normal((cout, cin) + (3,) * len(dims)) * 0.2)
    b = torch.tensor(rng.standard_normal(cout) * 0.1)
    cp = (cin + 7) // 8 * 8
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()   # [cout][taps][cin]
    y = run_conv(L, to_cl(x, cp), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 0, 32)
    ref = R.lrelu(R.conv(R.bf16(x), R.bf16(w), b.float().double()))
    got = from_cl(y, cout)
    assert rel(got, ref) <= 1e-2, rel(got, ref)
    assert rel(got, R.bf16(ref)) <= 4e-3


def test_conv_rejects_slope_outside_unit_interval(L):
    """The activation epilogue evaluates LeakyReLU as max(v, slope v), which needs
    0 <= slope <= 1: other slopes are refused before any launch."""
    x = torch.zeros((1, 4, 1, 16, 8), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(32 * 9 * 8, device="cuda")
    y = torch.zeros((1, 4, 4, 16, 8), dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for slope in (1.5, -0.1, float("nan")):
        rc = L.load().cbct_conv(x.data_ptr(), 1, 1, 4, 16, 8, 0, w.data_ptr(), None, 8, 32, 0, 0, slope,
                                y.data_ptr(), 32, None, None, 0, status.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        assert rc == -1
        assert b"slope" in L.load().cbct_last_error()
    torch.cuda.synchronize()
    assert float(y.float().abs().sum()) == 0.0


@pytest.mark.parametrize("cout,epi", [(32, 0), (5, 1)])
def test_conv_many_tiles_per_cta(L, cout, epi):
    """40 images of 64 x 256 give every persistent CTA several tiles, so the TMEM
    accumulators are reused and handed between the MMA issuer and the four epilogue
    warpgroups many times; images at both ends of the batch are checked."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(11 + cout)
    nimg, dims, cin = 40, (64, 256), 32
    x = torch.tensor(rng.standard_normal((nimg, cin) + dims))
    w = torch.tensor(rng.standard_normal((cout, cin, 3, 3)) * 0.1)
    b = torch.tensor(rng.standard_normal(cout) * 0.1)
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()
    pick = [0, 1, nimg - 2, nimg - 1]
    conv = R.conv(R.bf16(x[pick]), R.bf16(w), b.float().double())
    if epi == 0:
        y = run_conv(L, to_cl(x, 32), dims, 0, wg, b.float().cuda(), cin, cout, 0, 0, 32)
        got = from_cl(y[pick], cout)
        ref = R.lrelu(conv)
    else:
        state0 = torch.tensor(rng.standard_normal((cout, nimg) + dims))
        state = state0.float().cuda().contiguous()
        run_conv(L, to_cl(x, 32), dims, 0, wg, b.float().cuda(), cin, cout, 0, 1, 8, state=state)
        got = state.double().cpu()[:, pick]
        ref = state0[:, pick] + conv.movedim(1, 0)
    assert rel(got, ref) <= (1e-2 if epi == 0 else 1e-5), rel(got, ref)


@pytest.mark.parametrize("taps3d,dims", [(0, (21, 33)), (1, (7, 11, 13))])
def test_conv_residual_into_state(L, taps3d, dims):
    from oracle import lpd_ref as R
    rng = np.random.default_rng(7)
    cin, cout, nimg = 32, 5, 2
    x = torch.tensor(rng.standard_normal((nimg, cin) + dims))
    w = torch.tensor(rng.standard_normal((cout, cin) + (3,) * len(dims)) * 0.1)
    b = torch.tensor(rng.standard_normal(cout) * 0.1)
    state0 = torch.tensor(rng.standard_normal((cout, nimg) + dims))
    state = state0.float().cuda().contiguous()
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()
    run_conv(L, to_cl(x, 32), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 1, 8, state=state)
    ref = state0 + R.conv(R.bf16(x), R.bf16(w), b.float().double()).movedim(1, 0)
    assert rel(state.double().cpu(), ref) <= 1e-5


@pytest.mark.parametrize("taps3d,dims", [(0, (17, 26)), (1, (6, 9, 11))])
def test_conv_input_gradient_and_weight_gradient(L, taps3d, dims):
    """flip = 1 computes dL/dx of conv for upstream dL/dy, masked by the LeakyReLU
    derivative of a forward activation; wgrad matches autograd."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(11)
    cin, cout, nimg = 32, 32, 2
    x = R.bf16(torch.tensor(rng.standard_normal((nimg, cin) + dims)))
    w = R.bf16(torch.tensor(rng.standard_normal((cout, cin) + (3,) * len(dims)) * 0.1))
    dy = R.bf16(torch.tensor(rng.standard_normal((nimg, cout) + dims)))
    act = torch.tensor(rng.standard_normal((nimg, cin) + dims))        # sign pattern of a forward activation
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    br = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    (R.conv(xr, wr, br) * dy).sum().backward()
    ref_dx = xr.grad * torch.where(R.bf16(act) > 0, 1.0, SLOPE)
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()
    y = run_conv(L, to_cl(dy, 32), dims, taps3d, wg, None, cin, cout, 1, 2, 32, mask=to_cl(act, 32))
    got = from_cl(y, cin)
    assert rel(got, ref_dx) <= 1e-2, rel(got, ref_dx)
    # weight / bias gradient
    D, H, W = dims if taps3d else (1,) + dims
    dw = torch.zeros((cout, 27 if taps3d else 9, cin), device="cuda")
    db = torch.zeros(cout, device="cuda")
    x_cl, dy_cl = to_cl(x, 32), to_cl(dy, 32)   # keep both alive until the kernel has run
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.check(L.load().cbct_conv_wgrad(x_cl.data_ptr(), 32, cin, dy_cl.data_ptr(), 32, cout, nimg, D,
                                     H, W, taps3d, dw.data_ptr(), db.data_ptr(), 0, status.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream), "wgrad")
    torch.cuda.synchronize()
    assert status.item() == 0
    ref_dw = wr.grad.reshape(cout, cin, -1).permute(0, 2, 1)
    assert rel(dw.double().cpu(), ref_dw) <= 1e-5
    assert rel(db.double().cpu(), br.grad) <= 1e-5


@pytest.mark.parametrize("taps3d,dims,cin,cout,cpout,cpin", [
    (0, (9, 150), 20, 5, 8, 32), (0, (13, 37), 32, 12, 16, 32), (1, (5, 7, 9), 32, 5, 8, 32),
    (1, (4, 6, 130), 24, 32, 32, 32),
    # the production shapes: 3-D W = 128 full tiles (odd and even H), 2-D 192 x 256 images,
    # 8-slot inputs (the blocks' first layers) and 5 outputs in 8 slots (their last layers)
    (1, (4, 8, 128), 32, 32, 32, 32), (1, (3, 7, 128), 6, 32, 32, 8), (1, (4, 8, 128), 32, 5, 8, 32),
    (0, (192, 256), 32, 32, 32, 32), (0, (192, 256), 7, 32, 32, 8), (0, (191, 256), 32, 5, 8, 32)])
def test_conv_weight_gradient_shapes(L, taps3d, dims, cin, cout, cpout, cpin):
    """Weight and bias gradients for fewer input channels and 5 / 12 / 32 outputs
    (tensor-core path for 8 or 32 input slots), ragged W, odd H (the last tile's second
    output row outside the image), 2-D and 3-D."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(17)
    nimg = 2
    x = R.bf16(torch.tensor(rng.standard_normal((nimg, cin) + dims)))
    dy = R.bf16(torch.tensor(rng.standard_normal((nimg, cout) + dims)))
    wr = torch.zeros((cout, cin) + (3,) * len(dims), dtype=torch.float64, requires_grad=True)
    br = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    (R.conv(x, wr, br) * dy).sum().backward()
    D, H, W = dims if taps3d else (1,) + dims
    dw = torch.zeros((cout, 27 if taps3d else 9, cin), device="cuda")
    db = torch.zeros(cout, device="cuda")
    x_cl, dy_cl = to_cl(x, cpin), to_cl(dy, cpout)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.check(L.load().cbct_conv_wgrad(x_cl.data_ptr(), cpin, cin, dy_cl.data_ptr(), cpout, cout, nimg, D, H, W,
                                     taps3d, dw.data_ptr(), db.data_ptr(), 0, status.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream), "wgrad")
    torch.cuda.synchronize()
    assert status.item() == 0
    ref_dw = wr.grad.reshape(cout, cin, -1).permute(0, 2, 1)
    assert rel_l2_t(dw.double().cpu(), ref_dw) <= 1e-5
    assert rel_l2_t(db.double().cpu(), br.grad) <= 1e-5


def rel_l2_t(a, b):
    return float((a - b).norm() / b.norm())


FULL = [
    # the production tile widths: 3-D blocks at W = 128 (one full 128-pixel tile per row,
    # several row tiles with a ragged last one), 2-D blocks on 192 x 256 projection images
    ("3d_full_32to32", 1, (4, 8, 128), 32, 32, 1, "act"),
    ("3d_full_6to32", 1, (4, 8, 128), 6, 32, 1, "act"),
    ("3d_full_32to5", 1, (4, 8, 128), 32, 5, 1, "res"),
    ("3d_full_dx_5to32", 1, (4, 8, 128), 32, 5, 1, "dx"),
    ("3d_full_dx_32to32", 1, (4, 8, 128), 32, 32, 1, "dx"),
    ("3d_full_dx_32to6", 1, (4, 8, 128), 6, 32, 1, "dxres"),
    ("2d_full_7to32", 0, (192, 256), 7, 32, 2, "act"),
    ("2d_full_32to32", 0, (192, 256), 32, 32, 2, "act"),
    ("2d_full_32to5", 0, (192, 256), 32, 5, 2, "res"),
    ("2d_full_dx_32to32", 0, (192, 256), 32, 32, 2, "dx"),
    ("2d_full_dx_32to7", 0, (192, 256), 7, 32, 2, "dxres"),
]


@pytest.mark.parametrize("name,taps3d,dims,cin,cout,nimg,kind", FULL)
def test_conv_full_size_tiles(L, name, taps3d, dims, cin, cout, nimg, kind):
    """Forward (bias + LeakyReLU), residual update and masked input gradient at the
    tile shapes the learned blocks run: every output element compared with the FP64
    reference on BF16-rounded operands."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 10000)
    w = torch.tensor(rng.standard_normal((cout, cin) + (3,) * len(dims)) * 0.1)
    b = torch.tensor(rng.standard_normal(cout) * 0.1)
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()
    if kind in ("dx", "dxres"):
        # input gradient of a layer with cin inputs and cout outputs: dy has cout channels
        # (8 slots for 5, else 32), the result cin channels, masked by a forward activation
        # (BF16, 32 slots) or added to an FP32 channel-first state
        dy = R.bf16(torch.tensor(rng.standard_normal((nimg, cout) + dims)))
        xr = torch.zeros((nimg, cin) + dims, dtype=torch.float64, requires_grad=True)
        (R.conv(xr, R.bf16(w), None) * dy).sum().backward()
        dy_cl = to_cl(dy, 8 if cout <= 8 else 32)
        if kind == "dx":
            act = torch.tensor(rng.standard_normal((nimg, cin) + dims))
            y = run_conv(L, dy_cl, dims, taps3d, wg, None, cin, cout, 1, 2, 32, mask=to_cl(act, 32))
            ref = xr.grad * torch.where(R.bf16(act) > 0, 1.0, SLOPE)
            got = from_cl(y, cin)
            assert rel(got, ref) <= 1e-2, rel(got, ref)
        else:
            state0 = torch.tensor(rng.standard_normal((cin, nimg) + dims))
            state = state0.float().cuda().contiguous()
            run_conv(L, dy_cl, dims, taps3d, wg, None, cin, cout, 1, 1, 8, state=state)
            ref = state0 + xr.grad.movedim(1, 0)
            assert rel(state.double().cpu(), ref) <= 1e-5, rel(state.double().cpu(), ref)
        return
    x = torch.tensor(rng.standard_normal((nimg, cin) + dims))
    cp = 8 if cin <= 8 else 32
    conv = R.conv(R.bf16(x), R.bf16(w), b.float().double())
    if kind == "act":
        y = run_conv(L, to_cl(x, cp), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 0, 32)
        got, ref = from_cl(y, cout), R.lrelu(conv)
        assert rel(got, ref) <= 1e-2, rel(got, ref)
        assert rel(got, R.bf16(ref)) <= 4e-3
    else:
        state0 = torch.tensor(rng.standard_normal((cout, nimg) + dims))
        state = state0.float().cuda().contiguous()
        run_conv(L, to_cl(x, cp), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 1, 8, state=state)
        ref = state0 + conv.movedim(1, 0)
        assert rel(state.double().cpu(), ref) <= 1e-5, rel(state.double().cpu(), ref)


WIDE = [
    # 64-channel layers (the paper's dual block width): inputs of 64 slots on the channel
    # stride-64 kernels, more than 32 outputs as two launches into one 64-slot output
    ("2d_64to64", 0, (19, 150), 64, 64, 2, "act"),
    ("3d_64to64", 1, (5, 7, 130), 64, 64, 1, "act"),
    ("3d_8to64", 1, (5, 7, 130), 8, 64, 1, "act"),
    ("2d_12to40", 0, (19, 150), 12, 40, 2, "act"),
    ("3d_64to4", 1, (5, 7, 130), 64, 4, 1, "res"),
    ("2d_64to4", 0, (19, 150), 64, 4, 2, "res"),
    ("3d_dx_64to64", 1, (5, 7, 130), 64, 64, 1, "dx"),
    ("3d_dx_4to64", 1, (5, 7, 130), 64, 4, 1, "dx"),
    ("2d_dx_64to8", 0, (19, 150), 8, 64, 2, "dxres"),
]


def slots(c):
    return 8 if c <= 8 else (16 if c <= 16 else (32 if c <= 32 else 64))


@pytest.mark.parametrize("name,taps3d,dims,cin,cout,nimg,kind", WIDE)
def test_conv_wide_layers(L, name, taps3d, dims, cin, cout, nimg, kind):
    """Forward, residual update and masked input gradient with 64 input slots and with
    more than 32 outputs, every output element against the FP64 reference on
    BF16-rounded operands (ragged W over two column tiles, several row tiles)."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 10000)
    w = torch.tensor(rng.standard_normal((cout, cin) + (3,) * len(dims)) * 0.1)
    b = torch.tensor(rng.standard_normal(cout) * 0.1)
    wg = w.reshape(cout, cin, -1).permute(0, 2, 1).contiguous().float().cuda()
    if kind in ("dx", "dxres"):
        dy = R.bf16(torch.tensor(rng.standard_normal((nimg, cout) + dims)))
        xr = torch.zeros((nimg, cin) + dims, dtype=torch.float64, requires_grad=True)
        (R.conv(xr, R.bf16(w), None) * dy).sum().backward()
        dy_cl = to_cl(dy, slots(cout))
        if kind == "dx":
            act = torch.tensor(rng.standard_normal((nimg, cin) + dims))
            cp = max(32, slots(cin))
            y = run_conv(L, dy_cl, dims, taps3d, wg, None, cin, cout, 1, 2, cp, mask=to_cl(act, cp))
            ref = xr.grad * torch.where(R.bf16(act) > 0, 1.0, SLOPE)
            got = from_cl(y, cin)
            assert rel(got, ref) <= 1e-2, rel(got, ref)
        else:
            state0 = torch.tensor(rng.standard_normal((cin, nimg) + dims))
            state = state0.float().cuda().contiguous()
            run_conv(L, dy_cl, dims, taps3d, wg, None, cin, cout, 1, 1, 8, state=state)
            ref = state0 + xr.grad.movedim(1, 0)
            assert rel(state.double().cpu(), ref) <= 1e-5, rel(state.double().cpu(), ref)
        return
    x = torch.tensor(rng.standard_normal((nimg, cin) + dims))
    conv = R.conv(R.bf16(x), R.bf16(w), b.float().double())
    if kind == "act":
        cp = max(32, slots(cout))
        y = run_conv(L, to_cl(x, slots(cin)), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 0, cp)
        got, ref = from_cl(y, cout), R.lrelu(conv)
        assert rel(got, ref) <= 1e-2, rel(got, ref)
        assert rel(got, R.bf16(ref)) <= 4e-3
        # padding slots of the output (channels cout .. cp - 1) are zero
        if cout < cp:
            pad = y.transpose(-3, -2).reshape(y.shape[:-3] + (y.shape[-2], -1))[..., cout:]
            assert not torch.any(pad.float())
    else:
        state0 = torch.tensor(rng.standard_normal((cout, nimg) + dims))
        state = state0.float().cuda().contiguous()
        run_conv(L, to_cl(x, slots(cin)), dims, taps3d, wg, b.float().cuda(), cin, cout, 0, 1, 8, state=state)
        ref = state0 + conv.movedim(1, 0)
        assert rel(state.double().cpu(), ref) <= 1e-5, rel(state.double().cpu(), ref)


@pytest.mark.parametrize("taps3d,dims,cin,cout,cpin,cpout", [
    (1, (5, 7, 130), 64, 64, 64, 64), (0, (19, 150), 64, 64, 64, 64), (1, (5, 7, 130), 8, 64, 8, 64),
    (1, (5, 7, 130), 64, 4, 64, 8), (0, (19, 150), 40, 48, 64, 64)])
def test_conv_weight_gradient_wide(L, taps3d, dims, cin, cout, cpin, cpout):
    """Weight and bias gradients with 64 input or output slots (blocks of 32 x 32
    channels on the tensor cores, written into one [cout][taps][cin] array)."""
    from oracle import lpd_ref as R
    rng = np.random.default_rng(cin * 100 + cout + taps3d)
    nimg = 2
    x = R.bf16(torch.tensor(rng.standard_normal((nimg, cin) + dims)))
    dy = R.bf16(torch.tensor(rng.standard_normal((nimg, cout) + dims)))
    wr = torch.zeros((cout, cin) + (3,) * len(dims), dtype=torch.float64, requires_grad=True)
    br = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    (R.conv(x, wr, br) * dy).sum().backward()
    D, H, W = dims if taps3d else (1,) + dims
    dw = torch.full((cout, 27 if taps3d else 9, cin), 0.5, device="cuda")   # accumulate = 1 adds to it
    db = torch.full((cout,), 0.5, device="cuda")
    x_cl, dy_cl = to_cl(x, cpin), to_cl(dy, cpout)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.check(L.load().cbct_conv_wgrad(x_cl.data_ptr(), cpin, cin, dy_cl.data_ptr(), cpout, cout, nimg, D, H, W,
                                     taps3d, dw.data_ptr(), db.data_ptr(), 1, status.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream), "wgrad")
    torch.cuda.synchronize()
    assert status.item() == 0
    ref_dw = wr.grad.reshape(cout, cin, -1).permute(0, 2, 1) + 0.5
    assert rel_l2_t(dw.double().cpu(), ref_dw) <= 1e-5
    assert rel_l2_t(db.double().cpu(), br.grad + 0.5) <= 1e-5

"""FP64 reference of the learned primal-dual blocks (test infrastructure only).

Plain PyTorch CPU in float64. The convolution blocks of the paper's dual and primal
updates (Sec. 2.6, Algorithm 1: Gamma and Lambda; 3-layer blocks of any width with
LeakyReLU between layers, 2D over the detector plane or 3D; P4-equivariant blocks; the
P4 U-Net primal block of depth 1; centred forced weight normalisation), the unrolled
networks built from them (Adler-style memory, reversible coupling, the LIRE iteration),
with the projector pair taken from the FP64 C oracle through autograd functions.

BF16 operands are emulated by rounding the inputs and weights to bfloat16 before
the FP64 arithmetic, exactly where the GPU path rounds them. With round_grad the
backward pass does the same for the gradient operands of the tensor-core
contractions: the gradient reaching each convolution's output (the operand of the
input-gradient and weight-gradient convolutions) is rounded to bfloat16, and the
rest of the backward stays FP64.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

from . import adjoint as _adjoint
from . import forward as _forward

SLOPE = 0.2


def bf16(t: torch.Tensor) -> torch.Tensor:
    """Round to bfloat16 (round to nearest even) and back to float64. The rounded value
    is an operand copy of the FP32/FP64 master value, so the gradient passes through to
    the master unchanged (a plain dtype cast would round the gradient as well)."""
    r = t.detach().to(torch.bfloat16).to(torch.float64)
    if not t.requires_grad:
        return r
    return t + (r - t.detach())


class _RoundGrad(torch.autograd.Function):
    """Identity whose backward rounds the incoming gradient to bfloat16."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(torch.float64)


def round_grad(t: torch.Tensor) -> torch.Tensor:
    return _RoundGrad.apply(t)


def conv(x: torch.Tensor, w: torch.Tensor, b: torch.Tensor | None) -> torch.Tensor:
    """'Same' zero-padded 3x3 (2D, x [N, C, H, W]) or 3x3x3 (3D, x [N, C, D, H, W])
    cross-correlation: y[o, p] = b[o] + sum_{c, t} w[o, c, t] x[c, p + t - 1]."""
    if x.dim() == 4:
        return F.conv2d(x, w, b, padding=1)
    return F.conv3d(x, w, b, padding=1)


def lrelu(x: torch.Tensor) -> torch.Tensor:
    return torch.where(x > 0, x, SLOPE * x)


def block(x: torch.Tensor, params, round_bf16: bool = True, round_grads: bool = False) -> torch.Tensor:
    """conv -> LReLU -> conv -> LReLU -> conv; params = [(w1, b1), (w2, b2), (w3, b3)].
    With round_bf16 the conv inputs and weights are rounded to bfloat16 first (the
    GPU's operand precision); accumulation stays FP64. With round_grads the gradient
    with respect to each convolution's output is rounded to bfloat16 in the backward
    pass (the GPU's operand precision of its input- and weight-gradient convolutions)."""
    r = bf16 if round_bf16 else (lambda t: t)
    h = x
    for i, (w, b) in enumerate(params):
        h = conv(r(h), r(w), b)
        if round_grads:
            h = round_grad(h)
        if i < len(params) - 1:
            h = lrelu(h)
    return h


class _Proj(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, x):
        ctx.G = G
        return torch.from_numpy(_forward(G, x.detach().numpy()))

    @staticmethod
    def backward(ctx, g):
        return None, torch.from_numpy(_adjoint(ctx.G, g.detach().numpy()))


class _Back(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, y):
        ctx.G = G
        return torch.from_numpy(_adjoint(G, y.detach().numpy()))

    @staticmethod
    def backward(ctx, g):
        return None, torch.from_numpy(_forward(ctx.G, g.detach().numpy()))


def project(G, x):
    return _Proj.apply(G, x)


def backproject(G, y):
    return _Back.apply(G, y)


def lpd(G, y: torch.Tensor, x0: torch.Tensor | None, w_red: torch.Tensor, dual_params, primal_params,
        n_mem: int = 5, round_bf16: bool = True, mu_ref: float = 1.0, bp_scale: float = 1.0,
        f0: torch.Tensor | None = None, h0: torch.Tensor | None = None, return_state: bool = False,
        round_grads: bool = False, residual_input: bool = False, p4: bool = False, unet: bool = False):
    """Learned primal-dual (Adler-style memory of n_mem channels, the reading of the
    paper's primal/dual latents for this workload), in units of mu_ref:
        f <- x0 / mu_ref repeated (or the given f0), h <- 0 (or the given h0)
        h <- h + Gamma_n([h, mu_ref P f_1, y])                  (per projection image, 2D)
        f <- f + Lambda_n([f, bp_scale P^T (w h_1)])            (3D)
        output mu_ref f_0 (and the final f, h with return_state).
    y: [na, nv, nu]; x0: [nz, ny, nx]; w_red: [nu] redundancy weight. round_bf16 /
    round_grads: bfloat16 operands of the forward / backward convolutions (block).
    residual_input: the dual block also receives the data residual mu_ref P f_1 - y
    (the projection-domain form of the Landweber input of Algorithm 1):
        h <- h + Gamma_n([h, mu_ref P f_1, y, mu_ref P f_1 - y])."""
    na, nv, nu = y.shape
    f = (x0 / mu_ref).unsqueeze(0).repeat(n_mem, 1, 1, 1) if f0 is None else f0
    h = torch.zeros((n_mem, na, nv, nu), dtype=torch.float64) if h0 is None else h0
    for dp, pp in zip(dual_params, primal_params):
        pf = mu_ref * project(G, f[1])
        chans = [h, pf.unsqueeze(0), y.unsqueeze(0)]
        if residual_input:
            chans.append((pf - y).unsqueeze(0))                            # the data residual
        inp = torch.cat(chans, 0)                                          # [n_mem + 2 (+ 1), na, nv, nu]
        h = h + block(inp.permute(1, 0, 2, 3), dp, round_bf16, round_grads).permute(1, 0, 2, 3)
        bp = bp_scale * backproject(G, w_red.view(1, 1, -1) * h[1])
        inp = torch.cat([f, bp.unsqueeze(0)], 0).unsqueeze(0)             # [1, n_mem + 1, nz, ny, nx]
        f = f + primal_block(inp, pp, round_bf16, round_grads, p4, unet)[0]
    if return_state:
        return mu_ref * f[0], f, h
    return mu_ref * f[0]


def primal_block(x, params, round_bf16, round_grads, p4, unet=False):
    """The primal block: plain 3x3x3 layers, P4-equivariant ones (p4_block) whose params are
    base filters, or the P4 U-Net of depth 1 (p4_unet)."""
    if unet:
        return p4_unet(x, params, round_bf16, round_grads)
    return p4_block(x, params, round_bf16, round_grads) if p4 else block(x, params, round_bf16, round_grads)


def lpd_reversible(G, y: torch.Tensor, x0: torch.Tensor, w_red: torch.Tensor, dual_params, primal_params, perms_f,
                   perms_h, n_mem: int = 6, round_bf16: bool = True, mu_ref: float = 1.0, bp_scale: float = 1.0,
                   round_grads: bool = False, residual_input: bool = False, return_state: bool = False,
                   p4: bool = False, unet: bool = False):
    """Learned primal-dual with additive coupling and channel permutations (Algorithm 1:
    split, update the second half from the first, combine, permute), in units of mu_ref.
    With M = n_mem (even), f = [p1, p2] and h = [d1, d2] halves of M / 2 channels:
        f <- x0 / mu_ref in every channel, h <- 0
        per iteration n:
          d2 <- d2 + Gamma_n([d1, mu_ref P p2[0], y (, mu_ref P p2[0] - y)])
          p2 <- p2 + Lambda_n([p1, bp_scale P^T (w d2[0])])
          h <- (h[perms_h[n][c]])_c,   f <- (f[perms_f[n][c]])_c
        output mu_ref f[0].
    Each update reads only the half it does not change, so the iteration is inverted
    by undoing the permutations and subtracting the same block outputs in reverse order
    (lpd_reversible_inverse); the permutations mix the two halves."""
    M = n_mem
    K = M // 2
    na, nv, nu = y.shape
    f = (x0 / mu_ref).unsqueeze(0).repeat(M, 1, 1, 1)
    h = torch.zeros((M, na, nv, nu), dtype=torch.float64)
    for n, (dp, pp) in enumerate(zip(dual_params, primal_params)):
        d1, d2 = h[:K], h[K:]
        p1, p2 = f[:K], f[K:]
        pf = mu_ref * project(G, p2[0])
        chans = [d1, pf.unsqueeze(0), y.unsqueeze(0)]
        if residual_input:
            chans.append((pf - y).unsqueeze(0))
        d2 = d2 + block(torch.cat(chans, 0).permute(1, 0, 2, 3), dp, round_bf16, round_grads).permute(1, 0, 2, 3)
        bp = bp_scale * backproject(G, w_red.view(1, 1, -1) * d2[0])
        p2 = p2 + primal_block(torch.cat([p1, bp.unsqueeze(0)], 0).unsqueeze(0), pp, round_bf16, round_grads, p4, unet)[0]
        h = torch.cat([d1, d2], 0)[list(perms_h[n])]
        f = torch.cat([p1, p2], 0)[list(perms_f[n])]
    if return_state:
        return mu_ref * f[0], f, h
    return mu_ref * f[0]


def lpd_reversible_inverse(G, y: torch.Tensor, f: torch.Tensor, h: torch.Tensor, w_red: torch.Tensor, dual_params,
                           primal_params, perms_f, perms_h, n_mem: int = 6, round_bf16: bool = True,
                           mu_ref: float = 1.0, bp_scale: float = 1.0, residual_input: bool = False):
    """The initial states (f_0, h_0) recovered from the final ones by running
    lpd_reversible's iterations backwards: undo the permutations, then p2 -= Lambda_n(...)
    and d2 -= Gamma_n(...) with the same block inputs the forward pass used."""
    M = n_mem
    K = M // 2
    with torch.no_grad():
        for n in reversed(range(len(dual_params))):
            inv_f = np.argsort(perms_f[n])
            inv_h = np.argsort(perms_h[n])
            f = f[list(inv_f)]
            h = h[list(inv_h)]
            p1, p2 = f[:K], f[K:]
            d1, d2 = h[:K], h[K:]
            bp = bp_scale * backproject(G, w_red.view(1, 1, -1) * d2[0])
            p2 = p2 - block(torch.cat([p1, bp.unsqueeze(0)], 0).unsqueeze(0), primal_params[n], round_bf16)[0]
            pf = mu_ref * project(G, p2[0])
            chans = [d1, pf.unsqueeze(0), y.unsqueeze(0)]
            if residual_input:
                chans.append((pf - y).unsqueeze(0))
            d2 = d2 - block(torch.cat(chans, 0).permute(1, 0, 2, 3), dual_params[n], round_bf16).permute(1, 0, 2, 3)
            f = torch.cat([p1, p2], 0)
            h = torch.cat([d1, d2], 0)
    return f, h


def mixes_halves(perm) -> bool:
    """A permutation of 2K channels mixes the halves when the new first half takes at
    least one channel from the old second half (and so, by counting, the reverse)."""
    K = len(perm) // 2
    return any(p >= K for p in perm[:K])


def lire(G, y: torch.Tensor, x0: torch.Tensor, w_red: torch.Tensor, V: torch.Tensor, dual_params, primal_params,
         out_params, perms_f, perms_h, n_mem: int = 8, round_bf16: bool = True, mu_ref: float = 1.0,
         bp_scale: float = 1.0, round_grads: bool = False, return_state: bool = False, p4: bool = False,
         unet: bool = False):
    """The learned iterative scheme of Algorithm 1 (Sec. 2.6) at one resolution, in the
    reading used by the library (units: f in mu_ref, h and y in line-integral units):
        x <- x0                                              (FDK_w start)
        f <- [x / mu_ref, s P^T(w y), x / mu_ref, s P^T(w y), ...],  h <- y in every channel
        per iteration n, with halves of K = n_mem / 2 channels:
          d1, d2 = h[:K], h[K:];  p1, p2 = f[:K], f[K:]
          p_op = [mu_ref P p2[0], P x]                       (projections of p2 and x)
          d2 <- d2 + Gamma_n([d1, p_op, y, P x - y])         (3x3x3 convs over (angle, v, u))
          b_op = s P^T(w d2[0]);  LW = s P^T(P x - y)        (weighted backprojection, Landweber term)
          p2 <- p2 + Lambda_n([p1, b_op, x / mu_ref, LW, V]) (3x3x3 convs over the volume)
          f = [p1, p2];  x <- x + mu_ref (sum_c omega_n[c] f[c] + beta_n)   (1x1x1 output conv)
          h <- h[perms_h[n]];  f <- f[perms_f[n]]
        output x.
    out_params: per iteration (omega [n_mem], beta [1]); s = bp_scale; V the FoV tensor."""
    M = n_mem
    K = M // 2
    na, nv, nu = y.shape
    x = x0
    xbp = bp_scale * backproject(G, w_red.view(1, 1, -1) * y)
    f = torch.stack([x0 / mu_ref if c % 2 == 0 else xbp for c in range(M)], 0)
    h = y.unsqueeze(0).repeat(M, 1, 1, 1)
    for n, (dp, pp, (om, be)) in enumerate(zip(dual_params, primal_params, out_params)):
        d1, d2 = h[:K], h[K:]
        p1, p2 = f[:K], f[K:]
        pp2 = mu_ref * project(G, p2[0])
        px = project(G, x)
        res = px - y
        inp = torch.cat([d1, pp2.unsqueeze(0), px.unsqueeze(0), y.unsqueeze(0), res.unsqueeze(0)], 0)
        d2 = d2 + block(inp.unsqueeze(0), dp, round_bf16, round_grads)[0]          # [K, na, nv, nu]
        bop = bp_scale * backproject(G, w_red.view(1, 1, -1) * d2[0])
        lw = bp_scale * backproject(G, res)
        inp = torch.cat([p1, bop.unsqueeze(0), (x / mu_ref).unsqueeze(0), lw.unsqueeze(0), V.unsqueeze(0)], 0)
        p2 = p2 + primal_block(inp.unsqueeze(0), pp, round_bf16, round_grads, p4, unet)[0]
        f = torch.cat([p1, p2], 0)
        h = torch.cat([d1, d2], 0)
        x = x + mu_ref * ((om.view(-1, 1, 1, 1) * f).sum(0) + be)
        h = h[list(perms_h[n])]
        f = f[list(perms_f[n])]
    if return_state:
        return x, f, h
    return x


# ---- P4-equivariant convolutions (Sec. 2.6: the primal block's P4-equivariant layers) ----
#
# rho rotates a volume [.., z, y, x] by 90 degrees about z on a square x-y grid:
# (rho v)[z, y, x] = v[z, x, n - 1 - y]; on a 3x3x3 tap (dz, dy, dx) it acts as
# (dz, dy, dx) -> (dz, dx, -dy). A lifting layer's output group channel (co, r) uses the
# base filter rotated r times; a group layer's weight from input channel (ci, s) to
# output (co, r) is the base filter of relative rotation (s - r) mod 4, rotated r times;
# the last layer averages its group outputs. Each layer then commutes with rho (the group
# index of a group-channel tensor shifts by one under rho).


def rot_vol(v: torch.Tensor, r: int = 1) -> torch.Tensor:
    """rho^r applied to the last three axes [z, y, x] (square x-y grid)."""
    for _ in range(r % 4):
        v = torch.flip(v, dims=[-1]).transpose(-1, -2)   # (rho v)[z, y, x] = v[z, x, n - 1 - y]
    return v


def rot_filter(w: torch.Tensor, r: int) -> torch.Tensor:
    """The filter w[..., dz, dy, dx] rotated r times: W_r[t] = W[rho^-r t], i.e. the filter
    of the rotated volume, so that conv(rho v, W_r) = rho conv(v, W_{r-1})."""
    return rot_vol(w, r)


def p4_lift(w_base: torch.Tensor, b_base: torch.Tensor):
    """Full weights [4 co, cin, 3, 3, 3] of a lifting layer (output group channel
    (co, r) at index co * 4 + r) from base [co, cin, 3, 3, 3]; bias shared over r."""
    co = w_base.shape[0]
    w = torch.stack([rot_filter(w_base, r) for r in range(4)], 1).reshape((co * 4,) + tuple(w_base.shape[1:]))
    return w, b_base.repeat_interleave(4)


def p4_group(w_base: torch.Tensor, b_base: torch.Tensor):
    """Full weights [4 co, 4 ci, 3, 3, 3] of a group layer from base [co, ci, 4, 3, 3, 3]
    (relative rotation g): W[(co, r), (ci, s)] = rot_r(base[co, ci, (s - r) mod 4])."""
    co, ci = w_base.shape[:2]
    rows = []
    for r in range(4):
        blocks = [rot_filter(w_base[:, :, (s - r) % 4], r) for s in range(4)]   # each [co, ci, 3, 3, 3]
        rows.append(torch.stack(blocks, 2).reshape(co, ci * 4, 3, 3, 3))      # input index ci * 4 + s
    w = torch.stack(rows, 1).reshape(co * 4, ci * 4, 3, 3, 3)
    return w, b_base.repeat_interleave(4)


def p4_avg(w_base: torch.Tensor, b: torch.Tensor):
    """Weights [co, 4 ci, 3, 3, 3] of the last layer: the group layer's outputs (co, r)
    averaged over r, from base [co, ci, 4, 3, 3, 3]; bias per output channel."""
    w, _ = p4_group(w_base, torch.zeros(w_base.shape[0], dtype=w_base.dtype))
    co = w_base.shape[0]
    return w.reshape(co, 4, -1, 3, 3, 3).mean(1), b


def p4_block(x: torch.Tensor, params, round_bf16: bool = True, round_grads: bool = False) -> torch.Tensor:
    """The primal block with P4-equivariant layers: lift -> LReLU -> group -> LReLU ->
    group averaged over rotations. params = [(w_lift [c1, cin, 3, 3, 3], b [c1]),
    (w_group [c2, c1, 4, 3, 3, 3], b [c2]), (w_avg [cout, c2, 4, 3, 3, 3], b [cout])]; the
    hidden widths are 4 c1 and 4 c2 group channels."""
    full = [p4_lift(*params[0]), p4_group(*params[1]), p4_avg(*params[2])]
    return block(x, full, round_bf16, round_grads)


def pool2(x: torch.Tensor) -> torch.Tensor:
    """Mean over 2 x 2 x 2 blocks of the last three axes (even sizes)."""
    assert all(s % 2 == 0 for s in x.shape[-3:])
    return F.avg_pool3d(x, 2)


def up2(x: torch.Tensor) -> torch.Tensor:
    """Nearest upsampling by 2 along the last three axes."""
    for d in (-3, -2, -1):
        x = x.repeat_interleave(2, dim=d)
    return x


def p4_unet(x: torch.Tensor, params, round_bf16: bool = True, round_grads: bool = False) -> torch.Tensor:
    """The primal block as a U-Net of depth 1 (Sec. 2.6): six P4-equivariant 3x3x3 layers,
    LeakyReLU after all but the last, the last averaged over the rotations.
        a = L(lift(x)),  s = L(g2(a))                      full resolution, 4F group channels
        q = L(g3(pool(s))),  r = L(g4(q))                 half resolution, 8F group channels
        t = L(g5([up(r), s])),  out = avg6(t)             skip by concatenation, 12F -> 4F -> K
    params: (w [F, cin, 3,3,3], b [F]) for the lift, then base filters w [co, ci, 4, 3,3,3]
    with biases for g2 (F, F), g3 (2F, F), g4 (2F, 2F), g5 (F, 3F) and avg6 (K, F). BF16
    rounding as in block(): conv inputs and weights rounded; the pooled mean is a conv input."""
    r = bf16 if round_bf16 else (lambda t: t)
    full = [p4_lift(*params[0]), p4_group(*params[1]), p4_group(*params[2]), p4_group(*params[3]),
            p4_group(*params[4]), p4_avg(*params[5])]

    def layer(h, i, act=True):
        w, b = full[i]
        o = conv(r(h), r(w), b)
        if round_grads:
            o = round_grad(o)
        return lrelu(o) if act else o

    a = layer(x, 0)
    s = layer(a, 1)
    q = layer(pool2(r(s)), 2)
    rr = layer(q, 3)
    t = layer(torch.cat([up2(r(rr)), s], 1), 4)
    return layer(t, 5, act=False)


def weight_norm(w: torch.Tensor, gain: torch.Tensor) -> torch.Tensor:
    """Centred weight normalisation per output filter (the reading of forced weight
    normalisation): w_eff[c] = gain (w[c] - mean w[c]) / ||w[c] - mean w[c]||, over all
    other axes of w."""
    v = w - w.reshape(w.shape[0], -1).mean(1).reshape((-1,) + (1,) * (w.dim() - 1))
    n = v.reshape(v.shape[0], -1).norm(dim=1).reshape((-1,) + (1,) * (w.dim() - 1))
    return gain * v / n


def forced_renorm(w: torch.Tensor) -> torch.Tensor:
    """The forced step after an optimiser update: each filter replaced by its centred,
    normalised version scaled to norm sqrt(fan-in), which leaves weight_norm unchanged."""
    fan = w[0].numel()
    return weight_norm(w, torch.tensor(float(fan) ** 0.5, dtype=w.dtype))

"""Host-side tile planning of the tensor-core convolutions (cbct_conv_plan, no GPU
call): the invariants the kernel relies on, over a grid of shapes, and the packed
weight size against the row-unit definition restated here."""
import ctypes
import itertools

import pytest

SMEM_LIMIT = 227 * 1024


@pytest.fixture(scope="module")
def lib():
    from paper_2512_21180_gb300 import _lib, build
    build.build()
    return _lib.load()


def plan(lib, taps3d, H, cpin, cin, cout, flip=0):
    r, st, acc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb = ctypes.c_longlong()
    rc = lib.cbct_conv_plan(taps3d, H, cpin, cin, cout, flip, ctypes.byref(r), ctypes.byref(nb), ctypes.byref(st),
                            ctypes.byref(acc))
    assert rc == 0
    return r.value, nb.value, st.value, acc.value


def packed_bytes(taps3d, cpin, n_out, rpt):
    n_out = min(n_out, 32)   # the first launch of a layer with more than 32 outputs
    """B operand in row units: input row r of the rpt + 2 rows of a tile (or, with one
    8-channel group, the pair of rows 2j, 2j + 1) holds the weights of the output rows it
    feeds, o in [r - 2, r] within the tile; 3 column taps x channel groups x 8 channels
    of BF16 per output channel slot."""
    npad = 16 if n_out <= 16 else 32
    nr = rpt + 2
    cg = cpin // 8
    if cg == 1:
        units = [(2 * j, min(2 * j + 1, nr - 1)) for j in range((nr + 1) // 2)]
        groups = 6
    else:
        units = [(r, r) for r in range(nr)]
        groups = 3 * (cg + (cg & 1))
    cols = sum(min(r1, rpt - 1) - max(r0 - 2, 0) + 1 for r0, r1 in units)
    return (3 if taps3d else 1) * groups * cols * npad * 16


SHAPES = list(itertools.product((0, 1), (1, 2, 3, 5, 7, 16, 64, 192), (8, 16, 32, 64), (5, 7, 16, 32, 40, 64)))


@pytest.mark.parametrize("taps3d,H,cpin,n_out", SHAPES)
def test_plan_invariants(lib, taps3d, H, cpin, n_out):
    cin = min(cpin, 7 if cpin == 8 else cpin)
    rpt, nbytes, stages, acc = plan(lib, taps3d, H, cpin, cin, n_out)
    npad = 16 if n_out <= 16 else 32     # of the first launch (at most 32 outputs)
    assert 1 <= rpt <= 4
    assert rpt == 1 or rpt <= H
    assert rpt * npad <= 128 or rpt == 1
    # one TMEM accumulator per epilogue warpgroup at least (4 warpgroups)
    assert acc >= 4
    if cpin in (16, 64):
        assert rpt <= 2
    if cpin == 64:
        # every 64-slot shape fits: weights and two input stages, even at one row per tile
        stage = (rpt + 2) * 8 * 2176
        assert stages >= 2 and nbytes + stages * stage < SMEM_LIMIT
    if cpin == 8:
        assert rpt == 1 or rpt % 2 == 0
    assert nbytes == packed_bytes(taps3d, cpin, n_out, rpt)
    if rpt > 1:
        assert stages >= 2
        stage = (rpt + 2) * ((cpin // 8 + 1) & ~1) * 2176
        assert nbytes + stages * stage < SMEM_LIMIT


def test_plan_of_the_learned_blocks(lib):
    """The 128^3 workload's layers: dual (200 images of 192 x 256) and primal (128^3)."""
    assert plan(lib, 0, 192, 8, 7, 32)[0] == 4     # dual layer 1, row pairs
    assert plan(lib, 0, 192, 32, 32, 32)[:3:2] == (4, 3)   # dual layer 2: 4 rows, 3 input stages
    assert plan(lib, 0, 192, 32, 32, 5)[:3:2] == (4, 3)    # dual layer 3 (residual, 16 slots)
    assert plan(lib, 1, 128, 8, 6, 32)[0] == 4     # primal layer 1
    assert plan(lib, 1, 128, 32, 32, 32)[0] == 2   # primal layer 2 (27-tap weights)
    assert plan(lib, 1, 128, 32, 32, 5)[0] == 4    # primal layer 3
    # the paper's dual block (3x3x3 over (angle, v, u), 64 channels): one row per tile
    assert plan(lib, 1, 192, 64, 64, 64)[:3:2] == (1, 2)
    assert plan(lib, 1, 192, 64, 64, 4)[:3:2] == (1, 3)


def test_plan_rejects_bad_shapes(lib):
    z = ctypes.c_int()
    assert lib.cbct_conv_plan(0, 16, 24, 8, 32, 0, ctypes.byref(z), None, None, None) == -1   # cpin
    assert lib.cbct_conv_plan(0, 16, 8, 16, 32, 0, ctypes.byref(z), None, None, None) == -1   # cin > cpin
    assert lib.cbct_conv_plan(0, 16, 32, 32, 65, 0, ctypes.byref(z), None, None, None) == -1  # > 64 outputs
    assert lib.cbct_conv_plan(0, 16, 64, 65, 32, 0, ctypes.byref(z), None, None, None) == -1  # cin > cpin
    assert lib.cbct_conv_plan(0, 0, 32, 32, 32, 0, ctypes.byref(z), None, None, None) == -1   # H = 0

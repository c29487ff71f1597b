"""The largest grid extents, and states of more than 2^31 elements.

The ABI accepts 1 .. 65536 nodes along each axis.  These tests step periodic grids at that limit
whose initial fields repeat one 64 x 64 tile (a drop with random velocity and pressure noise,
gravity along y, density ratio 100, uniform sigma).  Nothing in the step depends on the node's
position when sigma is uniform, so the step commutes with translations by whole tiles: after K
steps every 64 x 64 block of the state must equal the state of a 64 x 64 periodic context
started from the tile.  A block is 64 columns wide, the width of one warp's strip, and the tile
repeats in y as well, so each copy goes through exactly the operations of the small grid's
strip, whatever segment of rows and march direction it falls in: the comparison is byte for
byte, on the device, over the whole state.  It reaches every address of a state with more than
2^31 elements (the widest grid, 65536 x 1856) and of a grid 65536 rows tall.  The small context
itself is checked element by element against the FP64 oracle (FP64 and FP32; the 16-bit storage
modes' accuracy is checked elsewhere).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TILE = 64
STEPS = 8
WIDE = (65536, 1856)     # 1856 rows x 2048 tiles x 576 elements = 2.19e9 > 2^31 (FP32, FP64)
TALL = (64, 65536)
ORACLE_TOL = {"fp64": 1e-12, "fp32": 2e-5}


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def tile():
    return W.random_drop(TILE, TILE, seed=21, rho_ratio=100.0, gravity=1e-6, amp=1e-3)


def state_words(torch, buf, ctx, ny):
    """The current state buffer of a context created on `buf`, as int32 words [ny][words/row]."""
    ptr, nstrips, elems = lbm.lbm_state_device(ctx)
    half = buf.numel() // 2
    off = ptr - buf.data_ptr()
    assert off in (0, half)
    return buf[off:off + half].view(torch.int32).view(ny, -1)


def run_on_device(torch, case, precision, fields):
    """Create a context on a torch buffer, initialise it from device fields, step it; returns
    (buffer, context)."""
    p = lbm.make_params(case, precision, stream=torch.cuda.current_stream().cuda_stream)
    nbytes = lbm.lbm_state_bytes(p)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ctx = lbm.lbm_create_with_buffer(p, buf.data_ptr(), nbytes)
    lbm.lbm_init_fields_device(ctx, *(fields[k].data_ptr() for k in ("phi", "p", "ux", "uy")))
    lbm.lbm_step(ctx, STEPS)
    lbm.lbm_check(ctx)
    return buf, ctx


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", [WIDE, TALL], ids=["65536x1856", "64x65536"])
def test_every_tile_copy_equals_the_tile_run(tile, shape, precision):
    torch = pytest.importorskip("torch")
    nx, ny = shape
    assert nx % TILE == 0 and ny % TILE == 0
    tf = {k: torch.tensor(tile["fields"][k], dtype=torch.float64, device="cuda")
          for k in ("phi", "p", "ux", "uy")}
    small_buf, small_ctx = run_on_device(torch, tile, precision, tf)
    big = W.Case(tile)
    big["nx"], big["ny"] = nx, ny
    big_fields = {k: v.repeat(ny // TILE, nx // TILE).contiguous() for k, v in tf.items()}
    big_buf = big_ctx = None
    try:
        big_buf, big_ctx = run_on_device(torch, big, precision, big_fields)
        del big_fields
        if shape == WIDE:
            ptr, nstrips, elems = lbm.lbm_state_device(big_ctx)
            assert elems > 2 ** 31
        small = state_words(torch, small_buf, small_ctx, TILE)        # [64][2 tiles]
        words = small.shape[1]
        bigw = state_words(torch, big_buf, big_ctx, ny).view(ny // TILE, TILE, nx // TILE, words)
        ref = small.view(TILE, 1, words)
        bad = [by for by in range(ny // TILE)
               if not torch.equal(bigw[by], ref.expand(TILE, nx // TILE, words))]
        assert not bad, f"{len(bad)} block rows differ from the tile run, first {bad[0]}"
        # one step more: the two buffers alternate, so the other buffer is covered as well
        lbm.lbm_step(big_ctx, 1)
        lbm.lbm_step(small_ctx, 1)
        lbm.lbm_check(big_ctx)
        small = state_words(torch, small_buf, small_ctx, TILE)
        bigw = state_words(torch, big_buf, big_ctx, ny).view(ny // TILE, TILE, nx // TILE, words)
        ref = small.view(TILE, 1, words)
        assert all(torch.equal(bigw[by], ref.expand(TILE, nx // TILE, words))
                   for by in range(ny // TILE))
    finally:
        if big_ctx is not None:
            lbm.lbm_destroy(big_ctx)
        del big_buf
        torch.cuda.empty_cache()
    try:
        if precision in ORACLE_TOL:
            g = np.empty((9, TILE, TILE))
            f = np.empty((9, TILE, TILE))
            lbm.lbm_get_populations(small_ctx, g, f)
            oc = O.OracleCase.from_dict(tile.params)
            fl = tile["fields"]
            g0, f0 = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
            g_ref, f_ref = O.run(oc, g0, f0, STEPS + 1)
            assert rel_l2(g, g_ref) <= ORACLE_TOL[precision]
            assert rel_l2(f, f_ref) <= ORACLE_TOL[precision]
    finally:
        lbm.lbm_destroy(small_ctx)

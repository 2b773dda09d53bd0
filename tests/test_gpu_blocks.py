"""GPU parity for block sizes 1, 2 and 16 and for frames whose height is not
a multiple of the block size (a bottom block row cut by the frame edge).

Block 1 is the paper's own per-pixel model; a cut block takes its mean,
extremes and variance sample over its pixels inside the frame.  Every frame
is teacher-forced against the oracle.  The multi-frame entry point falls back
to per-frame launches for these sizes, and the batched entry point refuses
them.
"""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream
from parity_util import StepReport, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


def _teacher_forced(lib, frames, Hs, block, precision="fp32", tile_rows=0, use_pdl=True):
    T, H, W = frames.shape
    m = lib.Dmsgm(W, H, block, precision=precision, tile_rows=tile_rows, use_pdl=use_pdl)
    fn = frames.cpu().numpy()
    rep = StepReport()
    rel = 1e-5 if precision == "fp32" else 6e-4
    mw = lib.mask_words(W)
    # one canary row below the frame's last mask row: nothing may be written there
    buf = torch.full((H + 1, mw), -1, dtype=torch.int32, device="cuda")
    mask = buf[:H]
    for t in range(T):
        prev = m.get_state() if t > 0 else None
        m.process(frames[t], Hs[t], mask)
        got = m.get_state()
        rep.add(compare_step(prev, got, lib.unpack_mask(mask, W), fn[t], Hs[t], block=block,
                             rel=rel))
    torch.cuda.synchronize()
    assert m.status() == 0
    assert bool((buf[H] == -1).all()), "a mask row below the frame was written"
    m.close()
    return rep


@pytest.mark.parametrize("W,H,T,block,precision,tile_rows", [
    (320, 240, 30, 1, "fp32", 0),
    (320, 240, 30, 2, "fp32", 0),
    (320, 240, 30, 16, "fp32", 0),
    (320, 240, 20, 1, "fp16", 0),
    (320, 240, 20, 2, "fp16", 0),
    (320, 240, 20, 16, "fp16", 0),
    (320, 250, 30, 4, "fp32", 0),       # 62 whole block rows + a 2-row cut
    (320, 237, 30, 8, "fp32", 0),       # 29 + a 5-row cut
    (640, 360, 20, 16, "fp32", 0),      # 22 + an 8-row cut
    (272, 33, 20, 2, "fp32", 0),        # ragged right tile, 1-row cut
    (320, 243, 20, 4, "fp16", 0),       # 3-row cut, FP16 state
])
def test_block_sizes_and_cut_rows_teacher_forced(lib, W, H, T, block, precision, tile_rows):
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=block * 7 + H), device="cuda")
    rep = _teacher_forced(lib, frames, Hs, block, precision, tile_rows)
    rep.assert_ok()
    assert rep.exempt <= 2e-3 * rep.blocks, rep


@pytest.mark.parametrize("block,tile_rows", [(1, 4), (1, 8), (1, 16), (2, 8), (2, 16), (2, 32),
                                             (16, 64), (16, 128), (16, 256)])
def test_every_tile_shape(lib, block, tile_rows):
    """Every tile height of the new block sizes (including the 4 x 2 and
    8 x 2 warp shapes), on a frame with a ragged tile in x and y."""
    W, H = 336, 200
    frames, Hs = make_stream(StreamSpec(W, H, 8, seed=5), device="cuda")
    rep = _teacher_forced(lib, frames, Hs, block, tile_rows=tile_rows)
    rep.assert_ok()


def test_hd_block16_cut_row(lib):
    """1920 x 1080 with 16 x 16 blocks: 67 whole block rows and an 8-row cut."""
    frames, Hs = make_stream(StreamSpec(1920, 1080, 6, seed=11, n_objects=12, jitter=2.0),
                             device="cuda")
    rep = _teacher_forced(lib, frames, Hs, 16)
    rep.assert_ok()


def test_seq_falls_back_and_batch_refuses(lib):
    """process_seq runs these sizes as per-frame launches (identical
    results); process_batch refuses them."""
    W, H, T = 320, 250, 6
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=3), device="cuda")
    for block in (2, 4, 16):
        a = lib.Dmsgm(W, H, block)
        ref = lib.new_mask(H, W, n=T)
        for t in range(T):
            a.process(frames[t], Hs[t], ref[t])
        b = lib.Dmsgm(W, H, block)
        out = b.process_seq(frames, Hs)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        sa, sb = a.get_state(), b.get_state()
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), (block, k)
    m = lib.Dmsgm(W, 240, 2)
    with pytest.raises(Exception, match="error -6"):
        lib.process_batch([m], [frames[0, :240].contiguous()], Hs[:1], [lib.new_mask(240, W)])

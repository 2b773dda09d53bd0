"""GPU: the pipelined frame step (kernel="pipe": resident CTAs stream the
tiles, staging pixels and the previous-state box in shared memory) gives
exactly the results of the per-tile kernel, and matches the oracle.

Cases cover frames where every resident CTA runs several tiles, both block
sizes and state precisions, the 16- and 32-row tiles, the first frame (no
state box), a shear whose state box does not fit a tile (global-memory
gathers inside the pipelined kernel) and the general projective form (which
the pipelined kernel hands to the per-tile kernel)."""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream, spec_for
from parity_util import StepReport, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


def _run(lib, kernel, frames, Hs, block, precision, tile_rows, pdl=True):
    T, H, W = frames.shape
    m = lib.Dmsgm(W, H, block, precision=precision, tile_rows=tile_rows, use_pdl=pdl,
                  kernel=kernel)
    masks = lib.new_mask(H, W, n=T)
    used = set()
    for t in range(T):
        m.process(frames[t], Hs[t], masks[t])
        used.add(m.info().last_kernel)
    torch.cuda.synchronize()
    assert m.status() == 0
    st = m.get_state()
    m.close()
    return masks, st, used


def _same(a, b):
    ma, sa, _ = a
    mb, sb, _ = b
    assert torch.equal(ma, mb)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("W,H,T,block,precision,tile_rows", [
    (256, 16384, 6, 4, "fp32", 16),     # 1024 tiles in one column: several per CTA
    (3840, 2160, 6, 4, "fp32", 32),
    (3840, 2160, 6, 4, "fp16", 16),
    (3840, 2160, 6, 8, "fp32", 32),
    (3840, 2160, 5, 8, "fp16", 64),
    (1920, 1080, 8, 4, "fp32", 16),     # fewer tiles than resident CTAs
    (288, 40, 8, 4, "fp32", 16),        # ragged right tile, partial tile rows
])
def test_pipe_equals_tile(lib, W, H, T, block, precision, tile_rows):
    frames, Hs = make_stream(spec_for(W, H, T, seed=31), device="cuda")
    a = _run(lib, "pipe", frames, Hs, block, precision, tile_rows)
    b = _run(lib, "tile", frames, Hs, block, precision, tile_rows)
    assert a[2] == {lib.DMSGM_KERNEL_PIPE}
    assert b[2] == {lib.DMSGM_KERNEL_TILE}
    _same(a, b)


def test_pipe_shear_box_overflow_and_projective_fallback(lib):
    """A strong shear (the affine form with d ex / d by = 1.2, so a 32-row
    tile's source columns span more than the box) gathers from global
    memory; a perspective term sends frames to the per-tile kernel.  Both
    must still equal the per-tile kernel."""
    W, H, T = 1024, 2048, 6
    frames, _ = make_stream(StreamSpec(W, H, T, seed=4), device="cuda")
    shear = np.array([[1.0, 1.2, -300.0], [0.0, 1.0, 2.0], [0.0, 0.0, 1.0]])
    persp = np.array([[1.0, 0.01, 3.0], [-0.01, 1.0, -2.0], [2e-6, -1e-6, 1.0]])
    Hs = np.stack([shear, shear, persp, shear, persp, shear])
    a = _run(lib, "pipe", frames, Hs, 4, "fp32", 32)
    b = _run(lib, "tile", frames, Hs, 4, "fp32", 32)
    assert a[2] == {lib.DMSGM_KERNEL_PIPE, lib.DMSGM_KERNEL_TILE}
    _same(a, b)


def test_pipe_unsupported_size_uses_the_per_tile_kernel(lib):
    """272 px wide: the grid is 68 blocks wide and its age rows are not a
    multiple of 16 bytes, so the state cannot be staged by TMA."""
    W, H, T = 272, 40, 6
    frames, Hs = make_stream(spec_for(W, H, T, seed=2), device="cuda")
    a = _run(lib, "pipe", frames, Hs, 4, "fp32", 16)
    b = _run(lib, "tile", frames, Hs, 4, "fp32", 16)
    assert a[2] == {lib.DMSGM_KERNEL_TILE}
    _same(a, b)


def test_pipe_without_pdl_and_after_reset(lib):
    W, H, T = 3840, 2160, 4
    frames, Hs = make_stream(spec_for(W, H, T, seed=8), device="cuda")
    a = _run(lib, "pipe", frames, Hs, 4, "fp32", 16, pdl=False)
    b = _run(lib, "tile", frames, Hs, 4, "fp32", 16, pdl=False)
    _same(a, b)
    m = lib.Dmsgm(W, H, 4, tile_rows=16, kernel="pipe")
    out = lib.new_mask(H, W, n=T)
    for t in range(T):
        m.process(frames[t], Hs[t], out[t])
    m.reset()
    for t in range(T):
        m.process(frames[t], Hs[t], out[t])
    torch.cuda.synchronize()
    assert torch.equal(out, a[0])


def test_pipe_teacher_forced_vs_oracle(lib):
    """Frame 4 of a 1024-tile stream through the pipelined kernel, from the
    GPU's frame-3 state, checked against the oracle."""
    W, H, T = 256, 4096, 5
    frames, Hs = make_stream(spec_for(W, H, T, seed=12), device="cuda")
    m = lib.Dmsgm(W, H, 4, tile_rows=16, kernel="pipe")
    masks = lib.new_mask(H, W, n=T)
    for t in range(T - 1):
        m.process(frames[t], Hs[t], masks[t])
    prev = m.get_state()
    m.process(frames[T - 1], Hs[T - 1], masks[T - 1])
    torch.cuda.synchronize()
    assert m.info().last_kernel == lib.DMSGM_KERNEL_PIPE
    rep = StepReport()
    rep.add(compare_step(prev, m.get_state(), lib.unpack_mask(masks[T - 1], W),
                         frames[T - 1].cpu().numpy(), Hs[T - 1], block=4))
    rep.assert_ok()

"""GPU: the checked build of the frame step (dmsgm_opts.checked) gives
exactly the results of the plain kernel and finds no index out of range --
every block size, FP16 state, cut rows, ragged tiles, and projective motion
that sends blocks off the grid."""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


def _run(lib, frames, Hs, block, precision, checked, tile_rows=0):
    T, H, W = frames.shape
    m = lib.Dmsgm(W, H, block, precision=precision, checked=checked, tile_rows=tile_rows,
                  use_pdl=True)
    assert m.info().checked == (1 if checked else 0)
    masks = lib.new_mask(H, W, n=T)
    for t in range(T):
        m.process(frames[t], Hs[t], masks[t])
    torch.cuda.synchronize()
    assert m.status() == 0
    st = m.get_state()
    m.close()
    return masks, st


@pytest.mark.parametrize("W,H,block,precision,tile_rows", [
    (320, 240, 4, "fp32", 0), (320, 240, 8, "fp16", 0), (336, 250, 4, "fp32", 16),
    (272, 37, 8, "fp32", 0), (320, 240, 1, "fp32", 0), (320, 242, 2, "fp16", 0),
    (640, 360, 16, "fp32", 0), (1920, 1080, 4, "fp32", 0), (3840, 2160, 4, "fp32", 0),
])
def test_checked_equals_plain(lib, W, H, block, precision, tile_rows):
    frames, Hs = make_stream(StreamSpec(W, H, 5, seed=W + block), device="cuda")
    a = _run(lib, frames, Hs, block, precision, True, tile_rows)
    b = _run(lib, frames, Hs, block, precision, False, tile_rows)
    assert torch.equal(a[0], b[0])
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k


def test_checked_strong_projective_motion(lib):
    W, H, T = 640, 480, 6
    frames, _ = make_stream(StreamSpec(W, H, T, seed=4), device="cuda")
    Hs = [np.eye(3),
          np.array([[1.0, 0.01, 90.0], [-0.01, 1.0, -70.0], [2e-5, -1e-5, 1.0]]),
          np.array([[0.8, 0.3, -200.0], [-0.2, 1.1, 150.0], [1e-4, 2e-4, 1.0]]),
          np.array([[1.0, 0.0, 5000.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]),   # all off the grid
          np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-3e-3, 0.0, 1.0]]),     # w <= 0 right of x = 333
          np.eye(3)]
    a = _run(lib, frames, Hs, 4, "fp32", True)
    b = _run(lib, frames, Hs, 4, "fp32", False)
    assert torch.equal(a[0], b[0])
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k


def test_checked_refusals(lib):
    with pytest.raises(Exception):
        lib.Dmsgm(320, 240, 4, checked=True, mix_spread=True)
    with pytest.raises(Exception):
        lib.Dmsgm(320, 240, 4, checked=True, prefilter=(5, 1.0, True))
    m = lib.Dmsgm(320, 240, 4, checked=True)
    frames, Hs = make_stream(StreamSpec(320, 240, 1, seed=1), device="cuda")
    with pytest.raises(Exception, match="error -6"):
        lib.process_batch([m], [frames[0]], Hs[:1], [lib.new_mask(240, 320)])
    out = m.process_seq(frames, Hs)                 # per-frame launches
    torch.cuda.synchronize()
    assert m.status() == 0 and out.shape[0] == 1

"""GPU: consecutive frame steps of one handle that wait only for the
neighbour tiles their motion compensation reaches (the step counters,
dmsgm_opts.step_wait = 0 with programmatic dependent launch) give bit for bit
the results of steps that wait for the whole previous grid, and of plain
stream order: masks and final state, over streams with strong and
projective motion, CUDA-graph replays, handles interleaved on one stream and
steps mixed with the other entry points."""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream, spec_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


def _run(lib, frames, Hs, block, precision="fp32", **kw):
    T, H, W = frames.shape
    m = lib.Dmsgm(W, H, block, precision=precision, **kw)
    masks = lib.new_mask(H, W, n=T)
    waits = []
    for t in range(T):
        m.process(frames[t], Hs[t], masks[t])
        waits.append(m.info().last_step_wait)
    torch.cuda.synchronize()
    assert m.status() == 0
    st = m.get_state()
    m.close()
    return masks, st, waits


def _same(a, b):
    assert torch.equal(a[0], b[0])
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k


def _strong(T, W, H, seed, projective=False, deg=3.0, shift=12.0):
    rng = np.random.default_rng(seed)
    Hs = [np.eye(3)]
    for _ in range(1, T):
        th = np.radians(rng.uniform(-deg, deg))
        s = 1 + rng.uniform(-0.03, 0.03)
        c, si = np.cos(th) * s, np.sin(th) * s
        tx, ty = rng.uniform(-shift, shift, 2)
        cx, cy = W / 2, H / 2
        M = np.array([[c, -si, cx - c * cx + si * cy + tx], [si, c, cy - si * cx - c * cy + ty],
                      [0, 0, 1.0]])
        if projective:
            M[2, :2] = rng.uniform(-2e-5, 2e-5, 2)
        Hs.append(M)
    return np.array(Hs)


@pytest.mark.parametrize("W,H,T,block,precision,tile_rows", [
    (320, 240, 40, 4, "fp32", 0), (1920, 1080, 30, 4, "fp32", 0), (1920, 1080, 20, 8, "fp16", 0),
    (3840, 2160, 12, 4, "fp32", 0), (3840, 2160, 10, 8, "fp32", 0), (272, 40, 30, 4, "fp16", 16),
    (640, 480, 16, 1, "fp32", 0), (640, 480, 16, 2, "fp32", 0), (640, 488, 16, 16, "fp32", 0),
    (1920, 1080, 16, 4, "fp32", 64)])
def test_tile_wait_equals_grid_wait(lib, W, H, T, block, precision, tile_rows):
    frames, Hs = make_stream(spec_for(W, H, T, seed=31), device="cuda")
    kw = dict(tile_rows=tile_rows)
    tiles = _run(lib, frames, Hs, block, precision, use_pdl=True, **kw)
    grid = _run(lib, frames, Hs, block, precision, use_pdl=True, step_wait="grid", **kw)
    plain = _run(lib, frames, Hs, block, precision, use_pdl=False, **kw)
    _same(tiles, grid)
    _same(tiles, plain)
    assert tiles[2][0] == 0 and all(tiles[2][1:])   # the first step waits for the grid
    assert not any(grid[2]) and not any(plain[2])


@pytest.mark.parametrize("projective", [False, True])
@pytest.mark.parametrize("deg,shift", [(3.0, 12.0), (20.0, 60.0)])
def test_strong_and_projective_motion(lib, projective, deg, shift):
    """Reaches of several tiles, blocks leaving the grid; the largest motion
    exceeds the neighbourhood the counters cover and falls back to the grid."""
    W, H, T = 1280, 720, 14
    frames, _ = make_stream(StreamSpec(W, H, T, seed=3), device="cuda")
    Hs = _strong(T, W, H, 7, projective, deg, shift)
    tiles = _run(lib, frames, Hs, 4, use_pdl=True)
    plain = _run(lib, frames, Hs, 4, use_pdl=False)
    _same(tiles, plain)
    if deg <= 3.0:
        assert sum(tiles[2]) >= T // 2


def test_graph_replays_and_interleaved_handles(lib):
    """Two handles alternate on one stream inside a captured pass; the pass is
    replayed three times; results equal an eager run of the same sequence in
    plain stream order."""
    W, H, T = 960, 544, 10
    fa, Ha = make_stream(spec_for(W, H, T, seed=41), device="cuda")
    fb, Hb = make_stream(spec_for(W, H, T, seed=42), device="cuda")
    s = torch.cuda.Stream()

    def handles(pdl):
        return lib.Dmsgm(W, H, 4, use_pdl=pdl), lib.Dmsgm(W, H, 8, use_pdl=pdl)

    ma, mb = lib.new_mask(H, W, n=T), lib.new_mask(H, W, n=T)

    def one_pass(a, b):
        for t in range(T):
            a.process(fa[t], Ha[t], ma[t], stream=s)
            b.process(fb[t], Hb[t], mb[t], stream=s)

    a, b = handles(True)
    with torch.cuda.stream(s):
        one_pass(a, b)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        one_pass(a, b)
    for _ in range(3):
        g.replay()
    s.synchronize()
    ra, rb = ma.clone(), mb.clone()
    sa, sb = a.get_state(), b.get_state()
    assert a.status() == 0 and b.status() == 0
    # the capture enqueued no work: one eager pass and three replays
    a3, b3 = handles(False)
    for _ in range(4):
        with torch.cuda.stream(s):
            one_pass(a3, b3)
    s.synchronize()
    assert torch.equal(ma, ra) and torch.equal(mb, rb)
    for k in sa:
        assert np.array_equal(sa[k], a3.get_state()[k]), k
        assert np.array_equal(sb[k], b3.get_state()[k]), k
    for m in (a, b, a3, b3):
        m.close()


def test_mixed_with_other_entry_points(lib):
    """Frame steps interleaved with the multi-frame entry point, the batched
    one, set_state and reset, on one stream with programmatic launch."""
    W, H, T = 640, 480, 24
    frames, Hs = make_stream(spec_for(W, H, T, seed=51), device="cuda")

    def run(pdl):
        m = lib.Dmsgm(W, H, 4, use_pdl=pdl)
        masks = lib.new_mask(H, W, n=T)
        for t in range(0, 6):
            m.process(frames[t], Hs[t], masks[t])
        m.process_seq(frames[6:10], Hs[6:10], masks[6:10])
        for t in range(10, 14):
            m.process(frames[t], Hs[t], masks[t])
        for t in range(14, 16):
            lib.process_batch([m], [frames[t]], [Hs[t]], [masks[t]], use_pdl=pdl)
        for t in range(16, 19):
            m.process(frames[t], Hs[t], masks[t])
        m.set_state(m.get_state())
        m.process(frames[19], Hs[19], masks[19])
        m.reset()
        for t in range(20, 24):
            m.process(frames[t], Hs[t], masks[t])
        torch.cuda.synchronize()
        assert m.status() == 0
        st = m.get_state()
        m.close()
        return masks, st

    _same(run(True), run(False))


def test_invalid_step_wait(lib):
    with pytest.raises(Exception):
        o = lib._lib.dmsgm_opts()
        o.step_wait = 2
        lib._lib.dmsgm_create(64, 64, 4, 2.0, 4.0, 30, o)

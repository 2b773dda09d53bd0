"""GPU: the preprocessing of the paper's Sec. 2.1 (Gaussian blur then 3 x 3
median, clamp-to-border, exact fixed-point blur) equals the oracle's filters
bit for bit; a handle that preprocesses its frames -- in the step kernel's own
tile (fused) or as a separate pass -- equals a plain handle fed the filtered
frames, and matches the oracle step on them."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_05156_gb300.synth import StreamSpec, make_stream
from parity_util import StepReport, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


@pytest.mark.parametrize("W,H", [(320, 240), (272, 33), (16, 1), (16, 2), (1920, 1080), (256, 300)])
@pytest.mark.parametrize("n,sigma,median", [(3, 0.8, True), (5, 1.0, True), (7, 1.5, False),
                                            (15, 3.0, True), (0, 1.0, True), (9, 2.0, False)])
def test_prefilter_equals_oracle(lib, W, H, n, sigma, median):
    rng = np.random.default_rng(W + H + n)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    img[: H // 2, : W // 3] = 90                   # flat areas, an edge and impulses
    img[rng.integers(0, H, 20), rng.integers(0, W, 20)] = 255
    got = lib.prefilter(torch.from_numpy(img).cuda(), gauss_size=n, sigma=sigma, median=median)
    want = oracle.prefilter(img, gauss_size=n, sigma=sigma, median=median)
    assert np.array_equal(got.cpu().numpy(), want)


def test_prefilter_rejects_bad_arguments(lib):
    f = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    for args in [dict(gauss_size=4), dict(gauss_size=17), dict(gauss_size=5, sigma=0.0),
                 dict(gauss_size=0, median=False)]:
        with pytest.raises(Exception):
            lib.prefilter(f, **args)
    with pytest.raises(Exception):
        lib.prefilter(f, out=f)                   # in place is not allowed


@pytest.mark.parametrize("block,pre,fused", [(4, (5, 1.0, True), 1), (8, (3, 0.8, False), 1),
                                             (4, (0, 1.0, True), 1), (2, (7, 1.5, True), 0),
                                             (4, (7, 1.5, True), 1), (8, (5, 1.0, True), 1),
                                             (4, (9, 2.0, True), 0), (8, (0, 1.0, True), 1)])
def test_preprocessing_handle_equals_filtered_frames(lib, block, pre, fused):
    W, H, T = 320, 240, 12
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=block), device="cuda")
    a = lib.Dmsgm(W, H, block, prefilter=pre, use_pdl=True)
    assert a.info().pre_fused == fused
    b = lib.Dmsgm(W, H, block, use_pdl=True)
    ma, mb = lib.new_mask(H, W, n=T), lib.new_mask(H, W, n=T)
    for t in range(T):
        a.process(frames[t], Hs[t], ma[t])
        b.process(lib.prefilter(frames[t], *pre[:2], median=pre[2]), Hs[t], mb[t])
    torch.cuda.synchronize()
    assert torch.equal(ma, mb)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_preprocessing_teacher_forced_vs_oracle(lib):
    W, H, T, B = 320, 240, 20, 4
    pre = (5, 1.0, True)
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=13), device="cuda")
    m = lib.Dmsgm(W, H, B, prefilter=pre)
    fn = frames.cpu().numpy()
    rep = StepReport()
    mask = lib.new_mask(H, W)
    for t in range(T):
        prev = m.get_state() if t > 0 else None
        m.process(frames[t], Hs[t], mask)
        filt = oracle.prefilter(fn[t], gauss_size=pre[0], sigma=pre[1], median=pre[2])
        rep.add(compare_step(prev, m.get_state(), lib.unpack_mask(mask, W), filt, Hs[t], block=B))
    rep.assert_ok()


def test_preprocessing_seq_runs_per_frame_and_batch_refuses(lib):
    W, H, T = 320, 240, 6
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=3), device="cuda")
    a = lib.Dmsgm(W, H, 4, prefilter=(5, 1.0, True))
    ref = lib.new_mask(H, W, n=T)
    for t in range(T):
        a.process(frames[t], Hs[t], ref[t])
    b = lib.Dmsgm(W, H, 4, prefilter=(5, 1.0, True))
    out = b.process_seq(frames, Hs)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    with pytest.raises(Exception, match="error -6"):
        lib.process_batch([b], [frames[0]], Hs[:1], [lib.new_mask(H, W)])


@pytest.mark.parametrize("W,H,block,precision,pre,pdl", [
    (1920, 1080, 4, "fp32", (5, 1.0, True), True),     # ragged right tile, 34 tile rows
    (1920, 1080, 8, "fp16", (7, 1.5, True), True),
    (336, 250, 4, "fp32", (3, 0.8, True), False),      # ragged tile, a cut block row
    (272, 37, 8, "fp32", (5, 1.0, False), True),       # 4 block rows + a 5-row cut
    (3840, 2160, 4, "fp32", (5, 1.0, True), True),
    (16, 8, 4, "fp32", (5, 1.0, True), True),          # one tile smaller than the halo
])
def test_fused_preprocessing_equals_separate_pass(lib, W, H, block, precision, pre, pdl):
    """The step kernel that filters its own tile gives exactly the masks and
    states of the separate filter pass followed by the plain step."""
    T = 6
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=W + H), device="cuda")
    out = []
    for separate in (False, True):
        m = lib.Dmsgm(W, H, block, precision=precision, prefilter=pre, prefilter_separate=separate,
                      use_pdl=pdl)
        assert m.info().pre_fused == (0 if separate else 1)
        masks = lib.new_mask(H, W, n=T)
        for t in range(T):
            m.process(frames[t], Hs[t], masks[t])
        torch.cuda.synchronize()
        assert m.status() == 0
        out.append((masks, m.get_state()))
        m.close()
    (ma, sa), (mb, sb) = out
    assert torch.equal(ma, mb)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_fused_preprocessing_teacher_forced_hd_vs_oracle(lib):
    """1920 x 1080, 8x8 blocks, the fused filter: every frame against the
    oracle's filter and step from the GPU's previous state."""
    W, H, T, B = 1920, 1080, 4, 8
    pre = (5, 1.0, True)
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=21, n_objects=12, jitter=2.0), device="cuda")
    m = lib.Dmsgm(W, H, B, prefilter=pre, use_pdl=True)
    assert m.info().pre_fused == 1
    fn = frames.cpu().numpy()
    rep = StepReport()
    mask = lib.new_mask(H, W)
    for t in range(T):
        prev = m.get_state() if t > 0 else None
        m.process(frames[t], Hs[t], mask)
        filt = oracle.prefilter(fn[t], gauss_size=pre[0], sigma=pre[1], median=pre[2])
        rep.add(compare_step(prev, m.get_state(), lib.unpack_mask(mask, W), filt, Hs[t], block=B))
    rep.assert_ok()

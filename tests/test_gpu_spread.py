"""GPU parity of the mixture-variance option (dmsgm_opts.mix_spread: the
compensated variance also carries the spread of the mixed means, Yi et
al.'s form) against the oracle run with the same option; the batched
kernel honours each stream's own flag; the multi-frame call runs such a
stream per frame."""
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


@pytest.mark.parametrize("W,H,T,block,precision", [
    (320, 240, 40, 4, "fp32"), (320, 240, 40, 8, "fp32"), (320, 240, 30, 4, "fp16"),
    (320, 250, 20, 4, "fp32"), (320, 240, 20, 2, "fp32"), (320, 240, 20, 16, "fp32"),
])
def test_spread_teacher_forced(lib, W, H, T, block, precision):
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=21), device="cuda")
    m = lib.Dmsgm(W, H, block, precision=precision, mix_spread=True)
    assert m.info().mix_spread == 1
    fn = frames.cpu().numpy()
    rep = StepReport()
    mask = lib.new_mask(H, W)
    for t in range(T):
        prev = m.get_state() if t > 0 else None
        m.process(frames[t], Hs[t], mask)
        rep.add(compare_step(prev, m.get_state(), lib.unpack_mask(mask, W), fn[t], Hs[t],
                             block=block, rel=1e-5 if precision == "fp32" else 6e-4,
                             mix_spread=True))
    rep.assert_ok()


def test_spread_changes_the_state(lib):
    W, H, T = 320, 240, 10
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=2), device="cuda")
    out = []
    for spread in (False, True):
        m = lib.Dmsgm(W, H, 4, mix_spread=spread)
        for t in range(T):
            m.process(frames[t], Hs[t])
        out.append(m.get_state())
    assert not np.array_equal(out[0]["varA"], out[1]["varA"])


def test_batch_mixes_spread_and_plain_streams(lib):
    """One batched launch over streams with and without the option equals
    each stream run alone."""
    specs = [(320, 240, 4, True), (640, 480, 8, False), (320, 240, 4, False), (1280, 720, 4, True)]
    T = 6
    data = [make_stream(spec_for(W, H, T, seed=40 + i), device="cuda")
            for i, (W, H, _, _) in enumerate(specs)]
    alone, batched = [], []
    for (W, H, B, sp), (fr, Hs) in zip(specs, data):
        m = lib.Dmsgm(W, H, B, mix_spread=sp)
        mk = lib.new_mask(H, W, n=T)
        for t in range(T):
            m.process(fr[t], Hs[t], mk[t])
        alone.append((mk, m.get_state()))
        batched.append(lib.Dmsgm(W, H, B, mix_spread=sp))
    masks = [lib.new_mask(H, W, n=T) for (W, H, _, _) in specs]
    for t in range(T):
        lib.process_batch(batched, [d[0][t] for d in data], np.stack([d[1][t] for d in data]),
                          [mk[t] for mk in masks])
    torch.cuda.synchronize()
    for i, m in enumerate(batched):
        assert torch.equal(masks[i], alone[i][0]), i
        st = m.get_state()
        for k in st:
            assert np.array_equal(st[k], alone[i][1][k]), (i, k)


def test_seq_with_spread_runs_per_frame(lib):
    W, H, T = 320, 240, 8
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=6), device="cuda")
    a = lib.Dmsgm(W, H, 4, mix_spread=True)
    ref = lib.new_mask(H, W, n=T)
    for t in range(T):
        a.process(frames[t], Hs[t], ref[t])
    b = lib.Dmsgm(W, H, 4, mix_spread=True)
    out = b.process_seq(frames, Hs)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    sa, sb = a.get_state(), b.get_state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every test here is marked gpu.  Inputs come from the seeded generator only;
expected values come from the oracle only.
"""
import numpy as np
import pytest
import torch

from oracle import oracle_run, oracle_step, state_from_arrays
from paper_1702_05156_gb300.synth import StreamSpec, make_stream, random_state, spec_for, translation
from parity_util import StepReport, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


def _run_teacher_forced(lib, frames, Hs, *, block, precision="fp32", every=1, rel=None,
                        tile_rows=0, use_pdl=False):
    """Run the stream on the GPU; on every `every`-th frame read the state
    before and after it and compare the step with the oracle."""
    T, H, W = frames.shape
    m = lib.Dmsgm(W, H, block, precision=precision, tile_rows=tile_rows, use_pdl=use_pdl)
    fn = frames.cpu().numpy()
    rep = StepReport()
    rel = rel if rel is not None else (1e-5 if precision == "fp32" else 6e-4)
    mask = lib.new_mask(H, W)
    for t in range(T):
        check = (t % every == 0) or t == T - 1
        prev = m.get_state() if (check and t > 0) else None
        m.process(frames[t], Hs[t], mask)
        if check:
            got = m.get_state()
            bits = lib.unpack_mask(mask, W)
            rep.add(compare_step(prev, got, bits, fn[t], Hs[t], block=block, rel=rel))
    m.close()
    return rep


@pytest.mark.parametrize("block", [4, 8])
def test_plain_320x240_all_frames_teacher_forced(lib, block):
    """320x240, 100 frames of the seeded stream, every frame teacher-forced."""
    frames, Hs = make_stream(StreamSpec(320, 240, 100, seed=0), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=block)
    rep.assert_ok()
    assert rep.exempt <= 1e-3 * rep.blocks, rep


@pytest.mark.parametrize("block,tile_rows", [(4, 16), (4, 32), (4, 64), (8, 32), (8, 64),
                                             (8, 128)])
def test_tile_shapes_agree(lib, block, tile_rows):
    """Every tile height passes (a ragged tail in y for 240 rows)."""
    frames, Hs = make_stream(StreamSpec(320, 240, 12, seed=3), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=block, tile_rows=tile_rows)
    rep.assert_ok()


def test_pdl_launch_matches(lib):
    """Programmatic dependent launch gives the same results."""
    frames, Hs = make_stream(StreamSpec(320, 240, 20, seed=4), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=4, use_pdl=True)
    rep.assert_ok()


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("block", [4, 8])
def test_hd_sampled_teacher_forced(lib, precision, block):
    """1920x1080 (the measured workload), 40 frames, teacher-forced on every
    8th frame at full size, in the launch configuration the benchmark uses."""
    frames, Hs = make_stream(spec_for(1920, 1080, 40, seed=0), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=block, precision=precision, every=8)
    rep.assert_ok()
    assert rep.exempt <= 1e-3 * rep.blocks, rep


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("block", [4, 8])
def test_4k_sampled_teacher_forced(lib, precision, block):
    """3840x2160, 24 frames in the benchmark's launch configuration
    (programmatic dependent launch, neighbour-tile waits), teacher-forced on
    every 5th frame and the last at full size."""
    frames, Hs = make_stream(spec_for(3840, 2160, 24, seed=0), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=block, precision=precision, every=5,
                              use_pdl=True)
    rep.assert_ok()
    assert rep.exempt <= 1e-3 * rep.blocks, rep


def test_hd_full_length_teacher_forced(lib):
    """The measured workload end to end: 1920x1080, block 4, FP32, all 300
    frames in the benchmark's launch configuration, teacher-forced on every
    10th frame and the last."""
    frames, Hs = make_stream(spec_for(1920, 1080, 300, seed=0), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=4, every=10, use_pdl=True)
    rep.assert_ok()
    assert rep.exempt <= 1e-3 * rep.blocks, rep


@pytest.mark.parametrize("W,H,block", [(16, 8, 4), (16, 8, 8), (48, 20, 4), (272, 36, 4),
                                       (272, 40, 8), (528, 264, 8), (16, 1024, 4)])
def test_edge_sizes(lib, W, H, block):
    """Tiny frames, W not a multiple of 32 (half-filled mask words), tiles
    ragged in x and y, a tall narrow frame."""
    frames, Hs = make_stream(StreamSpec(W, H, 6, n_objects=1, seed=W + H), device="cuda")
    rep = _run_teacher_forced(lib, frames, Hs, block=block)
    rep.assert_ok()


def test_random_state_strong_motion(lib):
    """Teacher-forced from a random state under rotation, scale, perspective
    and large shifts (blocks leave the grid; no-source restarts)."""
    rng = np.random.default_rng(9)
    W, H, B = 640, 480, 4
    m = lib.Dmsgm(W, H, B)
    st = dict(zip(("muA", "varA", "ageA", "muC", "varC", "ageC"),
                  random_state(H // B, W // B, 30, seed=2)))
    rep = StepReport()
    mask = lib.new_mask(H, W)
    for trial in range(6):
        th = np.radians(rng.uniform(-8, 8))
        s = 1 + rng.uniform(-0.1, 0.1)
        Hm = np.array([[s * np.cos(th), -s * np.sin(th), rng.uniform(-60, 60)],
                       [s * np.sin(th), s * np.cos(th), rng.uniform(-60, 60)],
                       [rng.uniform(-2e-4, 2e-4), rng.uniform(-2e-4, 2e-4), 1.0]])
        gpu_st = {k: (v.astype(np.float32) if k.startswith(("mu", "var")) else v.astype(np.uint8))
                  for k, v in st.items()}
        m.set_state(gpu_st)
        frame = torch.from_numpy(
            np.clip(np.kron(st["muA"], np.ones((B, B))) + rng.normal(0, 8, (H, W)), 0, 255)
            .round().astype(np.uint8)).cuda()
        m.process(frame, Hm, mask)
        got = m.get_state()
        rep.add(compare_step(gpu_st, got, lib.unpack_mask(mask, W), frame.cpu().numpy(), Hm,
                             block=B))
    rep.assert_ok()


def test_whole_block_shift_exact(lib):
    """Integer block shifts move the state exactly on the GPU too."""
    W, H, B = 320, 240, 4
    m = lib.Dmsgm(W, H, B)
    st0 = dict(zip(("muA", "varA", "ageA", "muC", "varC", "ageC"),
                   random_state(H // B, W // B, 30, seed=7)))
    gpu_st = {k: (v.astype(np.float32) if k.startswith(("mu", "var")) else v.astype(np.uint8))
              for k, v in st0.items()}
    rng = np.random.default_rng(0)
    frame = torch.from_numpy(rng.integers(0, 256, (H, W), dtype=np.uint8)).cuda()
    for k, l in ((1, 0), (0, -2), (3, 5)):
        m.set_state(gpu_st)
        mask = m.process(frame, translation(k * B, l * B))
        got = m.get_state()
        rep = compare_step(gpu_st, got, lib.unpack_mask(mask, W), frame.cpu().numpy(),
                           translation(k * B, l * B), block=B)
        rep.assert_ok()


def test_constant_frame_closed_form_gpu(lib):
    """Identity H, constant frame: mu stays exactly c in FP32 (incremental
    update), var_n = 255/n, ages 1..30 then 30, empty mask."""
    W, H = 64, 32
    m = lib.Dmsgm(W, H, 4)
    frame = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
    for n in range(1, 41):
        mask = m.process(frame, np.eye(3))
        st = m.get_state()
        assert (st["muA"] == 77).all()
        exp = 255.0 / n if n <= 30 else (255.0 / 30) * (30.0 / 31.0) ** (n - 30)
        np.testing.assert_allclose(st["varA"], exp, rtol=1e-5)
        assert (st["ageA"] == min(n, 30)).all()
        assert int(mask.abs().sum()) == 0


def test_free_running_short(lib):
    """20 frames free-running on both sides (no teacher forcing)."""
    frames, Hs = make_stream(StreamSpec(320, 240, 20, seed=11), device="cuda")
    m = lib.Dmsgm(320, 240, 4)
    masks = []
    for t in range(20):
        masks.append(m.process(frames[t], Hs[t]).clone())
    st = m.get_state()
    ost, omasks = oracle_run(frames.cpu().numpy(), Hs, block=4)
    agree_age = (st["ageA"] == ost.ageA).mean()
    assert agree_age >= 0.999, agree_age
    bits = np.stack([lib.unpack_mask(k, 320) for k in masks])
    assert (bits != omasks).mean() <= 1e-4


def test_checkpoint_resume_bit_exact(lib):
    """get_state / set_state mid-stream then continue == uninterrupted run."""
    frames, Hs = make_stream(StreamSpec(320, 240, 16, seed=5), device="cuda")
    a = lib.Dmsgm(320, 240, 4)
    ref = [a.process(frames[t], Hs[t]).clone() for t in range(16)]
    st_ref = a.get_state()
    b = lib.Dmsgm(320, 240, 4)
    for t in range(8):
        b.process(frames[t], Hs[t])
    snap = b.get_state()
    b.reset()
    c = lib.Dmsgm(320, 240, 4)
    c.set_state(snap)
    out = [c.process(frames[t], Hs[t]).clone() for t in range(8, 16)]
    for t in range(8, 16):
        assert torch.equal(out[t - 8], ref[t])
    st = c.get_state()
    for k in st:
        assert np.array_equal(st[k], st_ref[k]), k


def test_reset_restarts(lib):
    frames, Hs = make_stream(StreamSpec(64, 32, 4, seed=1), device="cuda")
    m = lib.Dmsgm(64, 32, 4)
    m.process(frames[0], Hs[0])
    m.process(frames[1], Hs[1])
    m.reset()
    mask = m.process(frames[2], Hs[2])
    st = m.get_state()
    ost, om = oracle_step(frames[2].cpu().numpy(), Hs[2], None, block=4)
    assert (st["ageA"] == 1).all() and (st["varA"] == 255).all()
    np.testing.assert_array_equal(lib.unpack_mask(mask, 64), om)


def test_host_path_equals_device_path(lib):
    """dmsgm_process_host (host buffers, pipelined copies) gives the same
    bits as dmsgm_process on device buffers."""
    frames, Hs = make_stream(StreamSpec(640, 480, 45, seed=2), device="cuda")
    a = lib.Dmsgm(640, 480, 4)
    ref = torch.stack([a.process(frames[t], Hs[t]).clone() for t in range(45)]).cpu()
    b = lib.Dmsgm(640, 480, 4)
    host = frames.cpu().pin_memory()
    masks = b.process_host(host, Hs)
    torch.cuda.synchronize()
    assert torch.equal(masks, ref)
    assert np.array_equal(a.get_state()["muA"], b.get_state()["muA"])


def test_batch_equals_individual(lib):
    """process_batch over streams of mixed size/block/precision equals each
    stream processed alone."""
    cfgs = [(320, 240, 4, "fp32"), (640, 480, 8, "fp32"), (320, 240, 8, "fp16"),
            (1280, 720, 4, "fp16"), (48, 24, 4, "fp32")]
    streams = [make_stream(StreamSpec(w, h, 6, seed=100 + i), device="cuda")
               for i, (w, h, b, p) in enumerate(cfgs)]
    solo = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    bat = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    for t in range(6):
        ref = [m.process(fr[t], Hs[t]).clone() for m, (fr, Hs) in zip(solo, streams)]
        outs = [lib.new_mask(h, w) for (w, h, b, p) in cfgs]
        lib.process_batch(bat, [fr[t] for fr, _ in streams],
                          np.stack([Hs[t] for _, Hs in streams]), outs)
        for r, o in zip(ref, outs):
            assert torch.equal(r, o)
    for a, b in zip(solo, bat):
        sa, sb = a.get_state(), b.get_state()
        for k in sa:
            assert np.array_equal(sa[k], sb[k])


def test_caller_owned_state_memory(lib):
    W, H = 320, 240
    from paper_1702_05156_gb300 import _lib
    nbytes = _lib.dmsgm_state_bytes(W, H, 4, 0)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-buf.data_ptr()) % 256
    view = buf[off:off + nbytes]
    frames, Hs = make_stream(StreamSpec(W, H, 5, seed=8), device="cuda")
    a = lib.Dmsgm(W, H, 4, state_mem=view)
    b = lib.Dmsgm(W, H, 4)
    for t in range(5):
        assert torch.equal(a.process(frames[t], Hs[t]), b.process(frames[t], Hs[t]))
    a.close()


@pytest.mark.parametrize("ctas,pdl,item_warps", [(0, False, 0), (0, True, 0), (1, False, 0),
                                                 (3, True, 0), (7, True, 0), (0, True, 8),
                                                 (5, False, 8), (1 << 30, True, 8),
                                                 (1 << 30, False, 4)])
def test_batch_launch_shapes(lib, ctas, pdl, item_warps):
    """The batched kernels with every launch shape (a single CTA walks the
    whole work list through its two-stage ring; one item per CTA; items of 4
    or 8 warps) match the single-stream kernel bit for bit, over several
    steps."""
    cfgs = [(1920, 1080, 4, "fp32"), (320, 240, 8, "fp32"), (640, 480, 4, "fp16"),
            (272, 40, 8, "fp16")]
    streams = [make_stream(StreamSpec(w, h, 4, seed=200 + i), device="cuda")
               for i, (w, h, b, p) in enumerate(cfgs)]
    solo = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    bat = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    for t in range(4):
        ref = [m.process(fr[t], Hs[t]).clone() for m, (fr, Hs) in zip(solo, streams)]
        outs = [lib.new_mask(h, w) for (w, h, b, p) in cfgs]
        lib.process_batch(bat, [fr[t] for fr, _ in streams],
                          np.stack([Hs[t] for _, Hs in streams]), outs,
                          ctas=ctas, use_pdl=pdl, item_warps=item_warps)
        for r, o in zip(ref, outs):
            assert torch.equal(r, o)
    for a, b in zip(solo, bat):
        sa, sb = a.get_state(), b.get_state()
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
    for m in bat:
        assert m.status() == 0


@pytest.mark.parametrize("item_warps,ctas", [(4, 0), (8, 0), (8, 40)])
def test_batch_beyond_64_streams(lib, item_warps, ctas):
    """More than 64 streams (the kernel stages each tile by 1-D row copies
    instead of tensor maps, with 256 descriptors in its parameters): 70 small
    streams of mixed size, block and precision, one item per CTA and a
    persistent grid, equal each stream alone, bit for bit, over 3 steps."""
    rng = np.random.default_rng(5)
    sizes = [(48, 24), (64, 32), (320, 240), (96, 64)]
    cfgs = [(*sizes[i % 4], 4 if rng.random() < 0.5 else 8, "fp16" if i % 5 == 0 else "fp32")
            for i in range(70)]
    cfgs = [(w, h, b, p) for (w, h, b, p) in cfgs if h % b == 0]
    streams = [make_stream(StreamSpec(w, h, 3, seed=500 + i), device="cuda")
               for i, (w, h, b, p) in enumerate(cfgs)]
    solo = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    bat = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    assert len(cfgs) > 64
    for t in range(3):
        ref = [m.process(fr[t], Hs[t]).clone() for m, (fr, Hs) in zip(solo, streams)]
        outs = [lib.new_mask(h, w) for (w, h, b, p) in cfgs]
        lib.process_batch(bat, [fr[t] for fr, _ in streams],
                          np.stack([Hs[t] for _, Hs in streams]), outs, ctas=ctas,
                          use_pdl=True, item_warps=item_warps)
        for i, (r, o) in enumerate(zip(ref, outs)):
            assert torch.equal(r, o), (i, cfgs[i])
    for a, b in zip(solo, bat):
        sa, sb = a.get_state(), b.get_state()
        for k in sa:
            assert np.array_equal(sa[k], sb[k]), k
        assert b.status() == 0


def test_batch_rejects_bad_item_warps(lib):
    from paper_1702_05156_gb300 import _lib
    m = lib.Dmsgm(64, 32, 4)
    fr = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.DmsgmError, match="item_warps"):
        lib.process_batch([m], [fr], np.eye(3).reshape(1, 9), [lib.new_mask(32, 64)], item_warps=6)


@pytest.mark.parametrize("item_warps", [4, 8])
def test_batch_teacher_forced_vs_oracle(lib, item_warps):
    """A 64-stream-like mix (fewer frames; FP32 and FP16 state, blocks 4 and
    8, up to 1920x1080) through the batched kernel with either item size,
    checked against the oracle, teacher-forced, in the parity bands (FP16
    state: relative 6e-4)."""
    cfgs = [(320, 240, 4, "fp32"), (640, 480, 8, "fp32"), (1280, 720, 4, "fp32"),
            (1920, 1080, 8, "fp16"), (640, 480, 4, "fp16")]
    streams = [make_stream(spec_for(w, h, 3, seed=1000 + i), device="cuda")
               for i, (w, h, b, p) in enumerate(cfgs)]
    ms = [lib.Dmsgm(w, h, b, precision=p) for (w, h, b, p) in cfgs]
    rep = StepReport()
    for t in range(3):
        prev = [m.get_state() for m in ms] if t else [None] * len(ms)
        outs = [lib.new_mask(h, w) for (w, h, b, p) in cfgs]
        lib.process_batch(ms, [fr[t] for fr, _ in streams],
                          np.stack([Hs[t] for _, Hs in streams]), outs, use_pdl=True,
                          item_warps=item_warps)
        for m, (w, h, b, pr), (fr, Hs), o, p in zip(ms, cfgs, streams, outs, prev):
            rep.add(compare_step(p, m.get_state(), lib.unpack_mask(o, w), fr[t].cpu().numpy(),
                                 Hs[t], block=b, rel=6e-4 if pr == "fp16" else 1e-5))
    rep.assert_ok()


@pytest.mark.parametrize("block", [4, 8])
def test_mask_padding_bits_are_zero(lib, block):
    """W % 32 == 16: the last word of each mask row has 16 bits past the
    frame; every kernel writes them as 0 even into a dirty buffer."""
    W, H = 48, 32
    frames, Hs = make_stream(StreamSpec(W, H, 3, seed=12), device="cuda")
    for mode in ("single", "batch", "seq"):
        m = lib.Dmsgm(W, H, block)
        masks = torch.full((3, H, lib.mask_words(W)), -1, dtype=torch.int32, device="cuda")
        if mode == "seq":
            m.process_seq(frames, Hs, masks)
        for t in range(3):
            if mode == "single":
                m.process(frames[t], Hs[t], masks[t])
            elif mode == "batch":
                lib.process_batch([m], [frames[t]], Hs[t][None], [masks[t]])
        w = masks.cpu().numpy().astype(np.uint32)
        assert (w[..., -1] >> 16 == 0).all(), mode
        m.close()


def test_device_wait_timeout_reports_and_context_survives(lib):
    """Failure detection without a fault: a kernel waits on a barrier nothing
    completes, gives up after 2 ms, sets the status word; dmsgm_status
    reports DMSGM_ERR_TIMEOUT once, then the handle works normally."""
    from paper_1702_05156_gb300 import _lib
    m = lib.Dmsgm(64, 32, 4)
    assert m.status() == 0
    _lib.dmsgm_selftest_wait(m.handle, 2_000_000, 0)
    assert m.status() == _lib.DMSGM_ERR_TIMEOUT
    assert "gave up" in _lib.dmsgm_last_error()
    assert m.status() == 0
    frame = torch.full((32, 64), 9, dtype=torch.uint8, device="cuda")
    mask = m.process(frame, np.eye(3))
    torch.cuda.synchronize()
    assert int(mask.abs().sum()) == 0 and m.status() == 0

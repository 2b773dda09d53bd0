"""GPU parity of the motion-estimation front end (include/dmsgm_homog.h)
against the FP64 oracle (homog_oracle.c, readings M1-M8), with the bands of
tests/homog_checks.py, and against an emulator of the kernels' own
arithmetic (tests/homog_checks.py, itself checked against the oracle on the
CPU).

- corners: a selection the method reaches under FP32 rounding of the FP64
  scores (every decision outside the score band as the oracle's; equal to
  the oracle's list when no decision is ambiguous), including frames with
  more candidates than the 8192 considered (the two-level cut) and frames
  whose scores tie; and equal, bit for bit, to the emulated FP32 selection;
- tracking: for points whose iteration converges, the FP32 kernel within
  0.02 px of the FP64 oracle, same status;
- RANSAC: winner, count and inlier set as the oracle's up to pairs within a
  relative 1e-6 of the threshold, the refit homography to rounding when the
  inlier sets agree; and winner, count and inlier set equal to the emulated
  FP64 division-free test (the counts' FP32 pre-test never decides
  otherwise);
- end to end: the GPU estimate close to the oracle's and to the synthetic
  stream's known camera motion; identical and flat frames."""
import numpy as np
import pytest
import torch

import oracle
from homog_checks import check_corners, check_ransac, emu_corners, emu_ransac
from paper_1702_05156_gb300.synth import StreamSpec, make_stream, spec_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import homog
    return homog


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _apply(Hm, p):
    q = np.c_[p, np.ones(len(p))] @ np.asarray(Hm).T
    return q[:, :2] / q[:, 2:]


def _frames(W, H_, T=2, seed=0):
    fr, Hs = make_stream(spec_for(W, H_, T, seed=seed))
    return np.asarray(fr), np.asarray(Hs)


def _cases():
    out = []
    fr, _ = _frames(320, 240, 1, seed=1)
    out.append(("stream320", fr[0], {}))
    fr, _ = _frames(1920, 1080, 1, seed=2)
    out.append(("stream1080", fr[0], {}))
    out.append(("stream1080_b5_md0", fr[0], dict(block_size=5, min_distance=0.0, max_corners=2000)))
    rng = np.random.default_rng(3)
    out.append(("noise_cut", rng.integers(0, 256, (720, 1280), dtype=np.uint8),
                dict(quality=1e-4, max_corners=4000, min_distance=3.0)))
    tile = rng.integers(0, 256, (16, 16), dtype=np.uint8)
    out.append(("periodic_ties", np.tile(tile, (30, 40)), dict(quality=1e-3, max_corners=3000,
                                                             min_distance=2.5)))
    sq = np.full((200, 256), 30, np.uint8)
    sq[40:90, 50:120] = 220
    sq[120:180, 150:230] = 180
    out.append(("squares", sq, dict(quality=0.2, min_distance=5.0, block_size=7)))
    return out


@pytest.mark.parametrize("name,img,kw", _cases(), ids=[c[0] for c in _cases()])
def test_corners_match_oracle_and_emulator(H, name, img, kw):
    h_, w = img.shape
    est = H.HomographyEstimator(w, h_, **kw)
    xy, sc, nc = est.corners(_dev(img))
    p = dict(block_size=3, quality=0.01, min_distance=10.0, max_corners=500)
    p.update({k: v for k, v in kw.items() if k in p})
    st = check_corners(img, xy, sc, nc, **p)
    assert st["common"] >= 0.9 * st["oracle_corners"], st
    exy, esc, enc = emu_corners(img, **p)
    assert nc == enc
    assert np.array_equal(xy, exy), (len(xy), len(exy))
    assert np.array_equal(sc, esc)
    if name == "noise_cut":
        assert nc > 8192          # the two-level cut was exercised
    est.close()


def test_corners_are_repeatable(H):
    fr, _ = _frames(640, 480, 1, seed=4)
    est = H.HomographyEstimator(640, 480)
    a = est.corners(_dev(fr[0]))
    b = est.corners(_dev(fr[0]))
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]


@pytest.mark.parametrize("W,H_,kw,frac", [(320, 240, {}, 0.8), (1920, 1080, {}, 0.6),
                                          (640, 480, dict(levels=2, win_half=7, eps=0.001), 0.9),
                                          (1280, 720, dict(levels=0, win_half=4), 0.25)])
def test_tracking_matches_oracle(H, W, H_, kw, frac):
    """Points whose tracking converges -- the oracle lands within 1 px of the
    stream's true camera motion -- agree to 0.02 px and in status.  A point
    whose iteration does not settle (too much motion for the window and the
    pyramid) follows a different path in FP32 and FP64; no parity is claimed
    for it."""
    fr, Hs = _frames(W, H_, 2, seed=W)
    xy, _, _ = oracle.corners(fr[0])
    pts = xy.astype(np.float64)
    p = dict(levels=5, win_half=10, max_iters=30, eps=0.01, min_eig=1e-3)
    p.update(kw)
    want, wst = oracle.track(fr[0], fr[1], pts, **p)
    est = H.HomographyEstimator(W, H_, **kw)
    got, gst = est.track(_dev(fr[0]), _dev(fr[1]), pts.astype(np.float32))
    truth = _apply(np.linalg.inv(Hs[1]), pts + 0.5) - 0.5
    conv = (wst == 1) & (np.linalg.norm(want - truth, axis=1) < 1.0)
    assert conv.sum() >= frac * len(pts)
    assert np.array_equal(gst[conv], wst[conv])
    assert np.abs(got[conv] - want[conv]).max() < 0.02


def _pattern(h, w, dx=0.0, dy=0.0):
    y, x = np.mgrid[0:h, 0:w].astype(float)
    x, y = x - dx, y - dy
    v = (128 + 50 * np.sin(x / 7.0) * np.cos(y / 9.0) + 40 * np.sin((x + 2 * y) / 13.0)
         + 25 * np.cos((3 * x - y) / 17.0))
    return np.clip(np.round(v), 0, 255).astype(np.uint8)


def test_tracking_translation_and_flat(H):
    prev, cur = _pattern(160, 208), _pattern(160, 208, -7.3, 5.6)
    pts = np.array([[60, 60], [100, 80], [140, 100], [80, 110]], np.float32)
    est = H.HomographyEstimator(208, 160)
    got, st = est.track(_dev(prev), _dev(cur), pts)
    assert np.all(st == 1)
    assert np.abs(got - pts - [-7.3, 5.6]).max() < 0.1
    same, st = est.track(_dev(prev), _dev(prev), pts)
    assert np.all(st == 1) and np.array_equal(same, pts)
    flat = np.full((160, 208), 90, np.uint8)
    _, st = est.track(_dev(flat), _dev(flat), pts)
    assert np.all(st == 0)


@pytest.mark.parametrize("iters,thr,seed", [(2000, 3.0, 0), (500, 1.0, 17), (64, 2.0, 5)])
def test_ransac_matches_oracle_and_emulator(H, iters, thr, seed):
    fr, _ = _frames(640, 480, 2, seed=6)
    xy, _, _ = oracle.corners(fr[0])
    out, st = oracle.track(fr[0], fr[1], xy.astype(np.float64))
    src = out[st == 1] + 0.5
    dst = xy[st == 1] + 0.5
    est = H.HomographyEstimator(640, 480, ransac_iters=iters, thresh=thr, seed=seed)
    Hg, inlg, res = est.ransac(src, dst)
    check_ransac(src, dst, 640, 480, iters, thr, seed, Hg, inlg, res.best, res.inliers)
    eb, ec, einl, _ = emu_ransac(src, dst, 640, 480, iters, thr, seed)
    assert res.best == eb and res.inliers == ec
    assert np.array_equal(inlg, einl)


def test_ransac_counts_at_the_threshold(H):
    """Pairs whose residual under the true motion is the threshold to within a
    few parts in 1e9: for hypotheses drawn from the exact inliers the inlier
    test sits on its threshold, where the counts' FP32 pre-test must leave the
    decision to FP64.  Winner, count and inlier set equal the emulated FP64
    test; against the oracle they differ only by pairs on the threshold."""
    rng = np.random.default_rng(11)
    Ht = np.array([[0.995, 0.012, -6.25], [-0.01, 1.004, 3.5], [1.5e-5, -2e-5, 1.0]])
    n = 1200
    src = rng.uniform(0, 1, (n, 2)) * [640, 480]
    src[: n // 4] = np.round(src[: n // 4]) + 0.5          # pixel centres
    dst = _apply(Ht, src)
    edge = rng.random(n) < 0.45
    ang = rng.uniform(0, 2 * np.pi, n)
    for thr in (1.0, 2.5):
        r = thr * (1.0 + rng.integers(-3, 4, n) * 1e-9)
        r[rng.random(n) < 0.2] = thr                        # exactly on the threshold
        d = dst + edge[:, None] * (r[:, None] * np.c_[np.cos(ang), np.sin(ang)])
        est = H.HomographyEstimator(640, 480, ransac_iters=500, thresh=thr, seed=9)
        Hg, inlg, res = est.ransac(src, d)
        eb, ec, einl, _ = emu_ransac(src, d, 640, 480, 500, thr, 9)
        assert res.best == eb and res.inliers == ec
        assert np.array_equal(inlg, einl)
        # half the pairs sit on the threshold: which of them count moves the
        # refit by up to the threshold itself, so the estimates are compared
        # there only within thr (the refit of the GPU's own inliers is
        # compared to rounding)
        st = check_ransac(src, d, 640, 480, 500, thr, 9, Hg, inlg, res.best, res.inliers,
                          corner_tol=thr)
        assert st["near_pairs"] > 0
        est.close()


def test_ransac_planted_outliers_and_degenerate(H):
    rng = np.random.default_rng(1)
    Ht = np.array([[1.01, -0.02, 4.5], [0.015, 0.99, -3.2], [2e-5, -1e-5, 1.0]])
    src = rng.uniform(0, 640, (1000, 2)) * [1, 0.75]
    dst = _apply(Ht, src)
    out = rng.random(1000) < 0.4
    # every outlier at least 5 px off in each coordinate
    dst[out] += rng.uniform(5, 40, (out.sum(), 2)) * rng.choice([-1.0, 1.0], (out.sum(), 2))
    est = H.HomographyEstimator(640, 480, ransac_iters=300, thresh=1.0, seed=3)
    Hg, inl, res = est.ransac(src, dst)
    st = check_ransac(src, dst, 640, 480, 300, 1.0, 3, Hg, inl, res.best, res.inliers)
    assert st["best"] == st["oracle_best"] and st["inlier_diffs"] == 0
    assert np.array_equal(inl, ~out)
    assert np.abs(Hg - Ht).max() < 1e-8
    line = np.c_[np.arange(20) * 10.0, np.arange(20) * 5.0]
    Hd, _, res = est.ransac(line, line + 1)
    assert res.inliers == -1 and np.array_equal(Hd, np.eye(3))
    H3, _, res = est.ransac(src[:3], dst[:3])
    assert res.inliers == -1


@pytest.mark.parametrize("W,H_", [(320, 240), (1920, 1080)])
def test_estimate_end_to_end(H, W, H_):
    """The GPU estimate against the oracle's (both run the whole front end on
    the same frames) and against the stream's true camera motion.  Corner
    lists may differ in the order of candidates whose scores tie within the
    FP32 band, which changes the pairs RANSAC draws, so the two estimates are
    compared at the frame corners within 0.1 px, not to rounding."""
    # the stand-in stream's high-contrast moving rectangles hold the strongest
    # corners: a 0.1 % quality cut keeps the background texture's as well
    fr, Hs = _frames(W, H_, 3, seed=11)
    est = H.HomographyEstimator(W, H_, thresh=1.0, quality=0.001)
    c = np.array([[0, 0], [W, 0], [0, H_], [W, H_], [W / 2, H_ / 2]], float)
    for t in (1, 2):
        Hg, res = est.estimate(_dev(fr[t - 1]), _dev(fr[t]))
        Hw, cw, ncw, ntw = oracle.estimate_homography(fr[t - 1], fr[t], thresh=1.0, quality=0.001)
        assert abs(res.corners - ncw) <= 2 and res.inliers > 0
        assert abs(res.tracked - ntw) <= 4
        assert np.abs(_apply(Hg, c) - _apply(Hw, c)).max() < 0.1
        assert np.abs(_apply(Hg, c) - _apply(Hs[t], c)).max() < 1.0


def test_estimate_identical_and_flat_frames(H):
    fr, _ = _frames(640, 480, 1, seed=12)
    est = H.HomographyEstimator(640, 480)
    Hg, res = est.estimate(_dev(fr[0]), _dev(fr[0]))
    assert res.inliers == res.tracked > 100
    assert np.abs(Hg - np.eye(3)).max() < 1e-9
    flat = np.full((480, 640), 100, np.uint8)
    Hf, res = est.estimate(_dev(flat), _dev(flat))
    assert res.corners == 0 and res.inliers == -1 and np.array_equal(Hf, np.eye(3))


def test_invalid_parameters(H):
    for kw in [dict(block_size=4), dict(max_corners=0), dict(max_corners=5000), dict(levels=9),
               dict(win_half=0), dict(quality=0.0), dict(ransac_iters=0), dict(thresh=0.0)]:
        with pytest.raises(Exception):
            H.HomographyEstimator(320, 240, **kw)
    with pytest.raises(Exception):
        H.HomographyEstimator(100, 240)          # W % 16 != 0


def test_estimated_motion_drives_the_mask(H):
    """The DMSGM step fed the estimated homographies gives nearly the mask it
    gives with the stream's true camera motion."""
    from paper_1702_05156_gb300 import dmsgm
    W, H_, T = 640, 480, 8
    frames, Hs = make_stream(StreamSpec(W, H_, T, seed=21), device="cuda")
    est = H.HomographyEstimator(W, H_, thresh=1.0, quality=0.001)
    a, b = dmsgm.Dmsgm(W, H_, 4), dmsgm.Dmsgm(W, H_, 4)
    agree = []
    for t in range(T):
        He = np.eye(3) if t == 0 else est.estimate(frames[t - 1], frames[t])[0]
        ma = dmsgm.unpack_mask(a.process(frames[t], He), W)
        mb = dmsgm.unpack_mask(b.process(frames[t], Hs[t]), W)
        agree.append(float(np.mean(np.asarray(ma) == np.asarray(mb))))
    assert min(agree) > 0.97, agree

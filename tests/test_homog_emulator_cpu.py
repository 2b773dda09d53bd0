"""CPU checks of the test emulator of the motion-estimation kernels
(tests/homog_checks.py) against the FP64 oracle, and of the banded
comparison itself: the emulator's FP32 scores stay inside the derived band
of the oracle's FP64 scores, its selection is one the banded check accepts,
its division-free inlier counts differ from the oracle's only by pairs on
the threshold, and planted mistakes in a corner list are rejected."""
import numpy as np
import pytest

import oracle
from homog_checks import (U32, check_corners, check_ransac, emu_corners, emu_ransac, emu_scores)
from paper_1702_05156_gb300.synth import make_stream, spec_for


def _frame(W, H, seed):
    fr, Hs = make_stream(spec_for(W, H, 2, seed=seed))
    return np.asarray(fr), np.asarray(Hs)


@pytest.mark.parametrize("bs", [1, 3, 5, 7])
def test_fp32_scores_inside_the_derived_band(bs):
    """|s32 - s64| <= 5.5 u (A + C), the bound derived in homog_checks (the
    checks use 8 u (A + C)); noise frames drive A, B, C to their extremes."""
    rng = np.random.default_rng(bs)
    worst = 0.0
    for img in (rng.integers(0, 256, (64, 80)).astype(np.uint8), _frame(320, 240, bs)[0][0],
                (rng.random((64, 80)) > 0.5).astype(np.uint8) * 255):
        A, B, C = oracle.tensor_map(img, bs)
        s = oracle.score_map(img, bs)
        e = np.abs(emu_scores(A, B, C).astype(np.float64) - s) / (U32 * (A + C) + 1e-300)
        worst = max(worst, float(e.max()))
    assert worst <= 5.5, worst


CASES = [
    ("stream320", lambda: _frame(320, 240, 1)[0][0], {}),
    ("stream640_md0", lambda: _frame(640, 480, 2)[0][0], dict(min_distance=0.0, max_corners=2000)),
    ("noise", lambda: np.random.default_rng(3).integers(0, 256, (240, 320), dtype=np.uint8),
     dict(quality=1e-4, max_corners=3000, min_distance=3.0)),
    ("periodic", lambda: np.tile(np.random.default_rng(3).integers(0, 256, (16, 16), dtype=np.uint8),
                                 (12, 16)), dict(quality=1e-3, max_corners=1000, min_distance=2.5)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_emulated_selection_passes_the_banded_check(name, make, kw):
    img = make()
    xy, sc, nc = emu_corners(img, **kw)
    st = check_corners(img, xy, sc, nc, **kw)
    assert st["common"] >= 0.9 * st["oracle_corners"], st


def test_banded_check_rejects_planted_mistakes():
    """A dropped strongest corner (nothing blocks it), a corner moved onto a
    non-maximum, a wrong candidate count and a swapped order all fail."""
    img = _frame(320, 240, 1)[0][0]
    xy, sc, nc = oracle.corners(img)
    check_corners(img, xy, sc, nc)
    with pytest.raises(AssertionError):
        check_corners(img, xy[1:], sc[1:], nc)
    bad = xy.copy()
    bad[3] += [0, 1]
    with pytest.raises(AssertionError):
        check_corners(img, bad, sc, nc)
    with pytest.raises(AssertionError):
        check_corners(img, xy, sc, nc + 50)
    sw = xy.copy()
    sw[[0, 5]] = sw[[5, 0]]
    ss = sc.copy()
    ss[[0, 5]] = ss[[5, 0]]
    with pytest.raises(AssertionError):
        check_corners(img, sw, ss, nc)


def _pairs(W, H, seed):
    fr, _ = _frame(W, H, seed)
    xy, _, _ = oracle.corners(fr[0])
    out, st = oracle.track(fr[0], fr[1], xy.astype(np.float64))
    return out[st == 1] + 0.5, xy[st == 1] + 0.5


def test_emulated_counts_differ_only_on_the_threshold():
    src, dst = _pairs(640, 480, 6)
    for thr in (1.0, 3.0):
        counts, near = oracle.ransac_counts(src, dst, 640, 480, 300, thr, 4)
        _, _, _, ec = emu_ransac(src, dst, 640, 480, 300, thr, 4)
        assert np.array_equal(ec < 0, counts < 0)
        assert np.all(np.abs(ec - counts) <= near)


def test_pairs_on_the_threshold_pass_the_banded_check():
    """Pairs planted at the threshold (exactly, or within parts in 1e9): the
    emulated kernel decisions differ from the oracle's only there, and the
    banded check accepts the emulated winner."""
    rng = np.random.default_rng(11)
    Ht = np.array([[0.995, 0.012, -6.25], [-0.01, 1.004, 3.5], [1.5e-5, -2e-5, 1.0]])
    n = 600
    src = rng.uniform(0, 1, (n, 2)) * [640, 480]
    q = np.c_[src, np.ones(n)] @ Ht.T
    dst = q[:, :2] / q[:, 2:]
    edge = rng.random(n) < 0.45
    ang = rng.uniform(0, 2 * np.pi, n)
    r = 1.0 * (1.0 + rng.integers(-3, 4, n) * 1e-9)
    r[rng.random(n) < 0.2] = 1.0
    d = dst + edge[:, None] * (r[:, None] * np.c_[np.cos(ang), np.sin(ang)])
    best, cnt, inl, _ = emu_ransac(src, d, 640, 480, 200, 1.0, 9)
    Hm = oracle.refit(src, d, inl, 640, 480)
    st = check_ransac(src, d, 640, 480, 200, 1.0, 9, Hm, inl, best, cnt, corner_tol=1.0)
    assert st["near_pairs"] > 0

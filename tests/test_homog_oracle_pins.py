"""CPU pins of the motion-estimation oracle (homog_oracle.c, readings M1-M8):
closed forms, invariants and special cases of Shi-Tomasi corners, the
binomial pyramid, pyramidal Lucas-Kanade and the RANSAC homography, each
chosen so that a plausible mistake in the oracle (a wrong Sobel sign or
tap, a transposed tensor entry, a wrong eigenvalue branch, a lost pyramid
level, a sign error in the Lucas-Kanade update, a wrong DLT row) fails."""
import numpy as np
import pytest

import oracle
from paper_1702_05156_gb300.synth import StreamSpec, make_stream


# ---------------------------------------------------------------- M1 score
def test_score_of_an_isolated_pixel_is_twelve_v_squared():
    """A single pixel of value v on a flat field: the 3 x 3 Sobel responses
    around it give A = C = 12 v^2 and B = 0 over the 3 x 3 window centred on
    it, so the smaller eigenvalue is 12 v^2."""
    img = np.full((21, 23), 50, np.uint8)
    img[10, 11] = 60
    s = oracle.score_map(img)
    assert s[10, 11] == 12 * 10 ** 2
    assert s[10, 11] == s.max()


def test_score_of_a_straight_edge_is_zero():
    """A vertical step has no y gradient: C = B = 0, so min(A, C) = 0."""
    img = np.zeros((16, 16), np.uint8)
    img[:, 8:] = 200
    assert np.all(oracle.score_map(img) == 0)
    assert np.all(oracle.score_map(img.T) == 0)


def test_score_is_transpose_and_offset_invariant():
    rng = np.random.default_rng(3)
    img = rng.integers(20, 200, (37, 41)).astype(np.uint8)
    s = oracle.score_map(img)
    assert np.array_equal(oracle.score_map(np.ascontiguousarray(img.T)), s.T)
    assert np.array_equal(oracle.score_map(img + 30), s)
    assert np.all(oracle.score_map(np.full((9, 9), 77, np.uint8)) == 0)


def test_score_of_a_corner_exceeds_its_edges():
    """At the corner of a bright quadrant both gradients are present, along
    its edges only one: the corner is the unique maximum."""
    img = np.zeros((30, 30), np.uint8)
    img[15:, 15:] = 255
    s = oracle.score_map(img)
    y, x = np.unravel_index(np.argmax(s), s.shape)
    assert abs(y - 15) <= 1 and abs(x - 15) <= 1
    assert s[25, 15] == 0 and s[15, 25] == 0


def _sobel_tensor_bruteforce(img, bs):
    """Structure tensor by explicit edge-padded Sobel filtering and window
    sums (numpy, independent of the oracle's loops)."""
    p = np.pad(img.astype(np.int64), 1, mode="edge")
    h, w = img.shape
    sh = lambda dy, dx: p[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]  # noqa: E731
    gx = (sh(-1, 1) + 2 * sh(0, 1) + sh(1, 1)) - (sh(-1, -1) + 2 * sh(0, -1) + sh(1, -1))
    gy = (sh(1, -1) + 2 * sh(1, 0) + sh(1, 1)) - (sh(-1, -1) + 2 * sh(-1, 0) + sh(-1, 1))
    r = bs // 2
    out = []
    for q in (gx * gx, gx * gy, gy * gy):
        qp = np.pad(q, r, mode="edge")
        acc = np.zeros_like(q)
        for j in range(bs):
            for i in range(bs):
                acc += qp[j:j + h, i:i + w]
        out.append(acc.astype(np.float64))
    return out


@pytest.mark.parametrize("bs", [1, 3, 5, 7])
def test_tensor_and_score_are_the_smaller_eigenvalue(bs):
    """M1: A, B, C equal an independent edge-padded Sobel filtering and window
    sum, and the score is the smaller eigenvalue of [A B; B C] as LAPACK's
    symmetric eigen-solver gives it (clamped at 0)."""
    rng = np.random.default_rng(bs)
    img = rng.integers(0, 256, (23, 31)).astype(np.uint8)
    A, B, C = oracle.tensor_map(img, bs)
    bA, bB, bC = _sobel_tensor_bruteforce(img, bs)
    assert np.array_equal(A, bA) and np.array_equal(B, bB) and np.array_equal(C, bC)
    ev = np.linalg.eigvalsh(np.stack([np.stack([A, B], -1), np.stack([B, C], -1)], -2))[..., 0]
    s = oracle.score_map(img, bs)
    assert np.all(s >= 0)
    assert np.allclose(s, np.maximum(ev, 0), rtol=0, atol=1e-9 * (A + C).max())


# ------------------------------------------------------------- M2-M4 corners
def _squares(h, w, boxes):
    img = np.full((h, w), 30, np.uint8)
    for (y0, x0, s) in boxes:
        img[y0:y0 + s, x0:x0 + s] = 220
    return img


def test_corners_of_squares():
    boxes = [(20, 20, 30), (20, 90, 25), (80, 40, 40)]
    img = _squares(140, 140, boxes)
    xy, sc, nc = oracle.corners(img, quality=0.2, min_distance=5, max_corners=100)
    true = []
    for (y0, x0, s) in boxes:
        true += [(x0, y0), (x0 + s - 1, y0), (x0, y0 + s - 1), (x0 + s - 1, y0 + s - 1)]
    true = np.array(true, float)
    d = np.linalg.norm(xy[:, None, :] - true[None], axis=2)
    assert len(xy) == len(true)
    assert d.min(axis=1).max() <= 1.5          # each found corner is a square's corner
    assert d.min(axis=0).max() <= 1.5          # each square's corner is found


def test_corner_spacing_order_and_cap():
    fr, _ = make_stream(StreamSpec(320, 240, 1, seed=5))
    img = np.asarray(fr[0])
    xy, sc, nc = oracle.corners(img, quality=0.01, min_distance=12.0, max_corners=150)
    assert 0 < len(xy) <= 150 and nc >= len(xy)
    assert np.all(np.diff(sc) <= 0)
    d2 = ((xy[:, None, :] - xy[None]) ** 2).sum(-1)
    np.fill_diagonal(d2, 10 ** 9)
    assert d2.min() >= 144
    assert np.all((xy[:, 0] >= 1) & (xy[:, 0] <= 318) & (xy[:, 1] >= 1) & (xy[:, 1] <= 238))
    # the first corner is the strongest interior local maximum
    s = oracle.score_map(img)
    assert sc[0] == s[1:-1, 1:-1].max()
    few, _, _ = oracle.corners(img, quality=0.01, min_distance=12.0, max_corners=10)
    assert np.array_equal(few, xy[:10])        # greedy: a prefix of the longer run


# ---------------------------------------------------------------- M5 pyramid
def test_pyramid_keeps_constants_and_halves_ramps():
    c = oracle.pyr_down(np.full((33, 20), 91, np.uint8))
    assert c.shape == (17, 10) and np.all(c == 91)
    ramp = np.tile((2 * np.arange(64)).astype(np.uint8), (16, 1))
    d = oracle.pyr_down(ramp)
    # a symmetric binomial keeps linear functions: level 1 at x' is 2 * (2 x')
    assert np.array_equal(d[:, 1:-1], np.tile(4 * np.arange(1, 31), (8, 1)).astype(np.uint8))


# ---------------------------------------------------------------- M6 tracking
def _pattern(h, w, dx=0.0, dy=0.0):
    """A smooth analytic texture, shifted by (dx, dy) (content moves +dx)."""
    y, x = np.mgrid[0:h, 0:w].astype(float)
    x, y = x - dx, y - dy
    v = (128 + 50 * np.sin(x / 7.0) * np.cos(y / 9.0) + 40 * np.sin((x + 2 * y) / 13.0)
         + 25 * np.cos((3 * x - y) / 17.0))
    return np.clip(np.round(v), 0, 255).astype(np.uint8)


def test_tracking_without_motion_is_exactly_zero():
    img = _pattern(120, 160)
    pts = np.array([[40, 40], [80, 60], [120, 90], [60, 100]], float)
    out, st = oracle.track(img, img, pts)
    assert np.all(st == 1)
    assert np.array_equal(out, pts)


@pytest.mark.parametrize("dx,dy,tol", [(3.0, -2.0, 0.05), (0.4, 0.7, 0.1), (-7.3, 5.6, 0.1)])
def test_tracking_recovers_a_translation(dx, dy, tol):
    prev, cur = _pattern(160, 200), _pattern(160, 200, dx, dy)
    pts = np.array([[60, 60], [100, 80], [140, 100], [80, 110]], float)
    out, st = oracle.track(prev, cur, pts)
    assert np.all(st == 1)
    assert np.abs(out - pts - [dx, dy]).max() < tol


def test_tracking_fails_on_a_flat_image():
    flat = np.full((80, 80), 100, np.uint8)
    out, st = oracle.track(flat, flat, np.array([[40.0, 40.0]]))
    assert st[0] == 0


# ---------------------------------------------------------------- M7-M8 RANSAC
def test_splitmix64_reference_outputs():
    """SplitMix64 from state 0: its first two outputs (the counters gamma and
    2 gamma) are 0xe220a8397b1dcdaf and 0x6e789e6aa1b965f4."""
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(g) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(2 * g % 2 ** 64) == 0x6E789E6AA1B965F4


def test_samples_are_distinct_and_in_range():
    for m in range(200):
        idx = oracle.sample4(123, m, 9)
        assert idx is not None and len(set(idx.tolist())) == 4 and idx.min() >= 0 and idx.max() < 9
    assert sorted(oracle.sample4(7, 3, 4).tolist()) == [0, 1, 2, 3]


def _apply(H, p):
    q = np.c_[p, np.ones(len(p))] @ H.T
    return q[:, :2] / q[:, 2:]


def test_ransac_recovers_an_exact_homography_among_outliers():
    rng = np.random.default_rng(1)
    H = np.array([[1.01, -0.02, 4.5], [0.015, 0.99, -3.2], [2e-5, -1e-5, 1.0]])
    src = rng.uniform(0, 640, (300, 2)) * [1, 0.75]
    dst = _apply(H, src)
    out = rng.random(300) < 0.3
    dst[out] += rng.uniform(-40, 40, (out.sum(), 2))
    dst[out] += np.sign(dst[out] - _apply(H, src[out])) * 5   # at least 5 px off
    Hm, inl, cnt, best = oracle.ransac(src, dst, 640, 480, iters=500, thresh=1.0, seed=9)
    assert cnt == (~out).sum()
    assert np.array_equal(inl, ~out)
    assert np.abs(Hm - H).max() < 1e-9 * np.abs(H).max()


def test_inlier_test_is_the_reprojection_distance():
    """M7: pairs placed at known reprojection distances r from the exact
    model: inliers are exactly those with r < thr; a model that sends a
    point behind the camera (w <= 0) never counts it; the band marks the
    pairs whose r^2 is within band * thr^2 of thr^2."""
    rng = np.random.default_rng(4)
    H = np.array([[1.02, 0.01, -3.0], [-0.015, 0.98, 2.5], [1e-5, 2e-5, 1.0]])
    src = rng.uniform(0, 1, (400, 2)) * [640, 480]
    r = rng.choice([0.0, 0.5, 0.99, 1.01, 2.0, 5.0], 400)
    ang = rng.uniform(0, 2 * np.pi, 400)
    dst = _apply(H, src) + r[:, None] * np.c_[np.cos(ang), np.sin(ang)]
    inl, near = oracle.inliers(H, src, dst, 1.0, band=0.05)
    assert np.array_equal(inl, r < 1.0)
    assert np.array_equal(near, np.abs(r * r - 1.0) <= 0.05 + 1e-12)
    behind = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, -1.0]])
    inl, _ = oracle.inliers(behind, src, -src, 1.0)
    assert not inl.any()
    counts, nearc = oracle.ransac_counts(src, dst, 640, 480, iters=50, thresh=1.0, seed=2)
    Hm = oracle.hypothesis(src, dst, 640, 480, 2, int(np.argmax(counts)))
    assert counts.max() == oracle.inliers(Hm, src, dst, 1.0)[0].sum()


def test_hypothesis_of_exact_pairs_is_the_model():
    """M7: any 4 distinct pairs of an exact homography in general position
    give back that homography (h33 = 1)."""
    rng = np.random.default_rng(8)
    H = np.array([[0.99, -0.03, 7.0], [0.02, 1.01, -4.0], [-2e-5, 1e-5, 1.0]])
    src = rng.uniform(0, 1, (30, 2)) * [320, 240]
    dst = _apply(H, src)
    for m in range(10):
        Hm = oracle.hypothesis(src, dst, 320, 240, 5, m)
        assert Hm is not None and np.abs(Hm - H).max() < 1e-9


def test_refit_is_the_least_squares_of_the_marked_pairs():
    """M8: exact pairs give back the homography; the RANSAC result is the
    refit of its own inlier set; noisy pairs give the model whose normal
    equations' residual vanishes (checked by an independent numpy lstsq of
    the same normalised DLT rows)."""
    rng = np.random.default_rng(13)
    H = np.array([[1.01, 0.02, -5.0], [-0.01, 0.99, 3.0], [1e-5, -2e-5, 1.0]])
    src = rng.uniform(0, 1, (200, 2)) * [640, 480]
    dst = _apply(H, src)
    assert np.abs(oracle.refit(src, dst, np.ones(200, bool), 640, 480) - H).max() < 1e-9
    noisy = dst + rng.normal(0, 0.3, dst.shape)
    Hr, inl, _, _ = oracle.ransac(src, noisy, 640, 480, iters=100, thresh=1.0, seed=1)
    assert np.array_equal(Hr, oracle.refit(src, noisy, inl, 640, 480))
    s, ox, oy = 2.0 / 640, 320.0, 240.0
    x, y = (src[inl, 0] - ox) * s, (src[inl, 1] - oy) * s
    X, Y = (noisy[inl, 0] - ox) * s, (noisy[inl, 1] - oy) * s
    z, o = np.zeros_like(x), np.ones_like(x)
    A = np.r_[np.c_[x, y, o, z, z, z, -x * X, -y * X], np.c_[z, z, z, x, y, o, -x * Y, -y * Y]]
    h = np.linalg.lstsq(A, np.r_[X, Y], rcond=None)[0]
    T = np.array([[s, 0, -s * ox], [0, s, -s * oy], [0, 0, 1.0]])
    Hl = np.linalg.inv(T) @ np.r_[h, 1.0].reshape(3, 3) @ T
    Hl /= Hl[2, 2]
    assert np.abs(Hr - Hl).max() < 1e-9 * np.abs(Hl).max()
    assert oracle.refit(src[:3], dst[:3], np.ones(3, bool), 640, 480) is None


def test_ransac_four_points_and_degenerate_data():
    src = np.array([[10, 10], [300, 20], [290, 230], [15, 220]], float)
    dst = np.array([[12, 9], [305, 25], [280, 240], [20, 215]], float)
    Hm, inl, cnt, best = oracle.ransac(src, dst, 320, 240, iters=20)
    assert cnt == 4 and np.abs(_apply(Hm, src) - dst).max() < 1e-9
    line = np.c_[np.arange(20) * 10.0, np.arange(20) * 5.0]
    Hn, _, cnt, best = oracle.ransac(line, line + 1, 320, 240, iters=50)
    assert Hn is None and cnt == 0


# ---------------------------------------------------------------- end to end
def test_front_end_recovers_the_synthetic_camera_motion():
    """Frames of the synthetic stream with their known homographies: the
    estimate maps the frame's corners within 1 px of the truth."""
    fr, Hs = make_stream(StreamSpec(320, 240, 4, seed=2))
    fr, Hs = np.asarray(fr), np.asarray(Hs)
    c = np.array([[0, 0], [320, 0], [0, 240], [320, 240], [160, 120]], float)
    for t in range(1, 4):
        Hm, cnt, nc, nt = oracle.estimate_homography(fr[t - 1], fr[t], thresh=1.0)
        assert Hm is not None and cnt >= 50
        assert np.abs(_apply(Hm, c) - _apply(Hs[t], c)).max() < 1.0
    Hm, cnt, nc, nt = oracle.estimate_homography(fr[0], fr[0])
    assert np.abs(Hm - np.eye(3)).max() < 1e-9

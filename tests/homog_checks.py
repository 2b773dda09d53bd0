"""Checks of the GPU motion-estimation front end against the FP64 oracle
(oracle/homog_oracle.c), with the bands that FP32 and FP64 rounding leave,
and an emulator of the kernels' own arithmetic.

Two different claims are checked.

1. Parity with the oracle (the method's plain FP64 definition).  The GPU
   scores corners in FP32, so decisions whose FP64 margin is inside the FP32
   error band can go either way; every other decision must match.
   - Score band.  The kernel takes A, B, C (exact integers) to FP32 and
     evaluates s = (t - sqrt(d^2 + 4 B^2)) / 2 with t = A + C, d = A - C,
     every operation rounded to nearest (u = 2^-24).  Rounding A, B, C moves
     t, d and B by at most u (A + C) each (|B| <= (A + C) / 2);
     sqrt(d^2 + 4 B^2) is the length of (d, 2 B), so it moves by at most
     |dd| + 2 |dB| <= 2 u (A + C), and its own four roundings add about
     3 u (A + C); the last subtraction and halving add u s.  In total
     |s32 - s| <= 5.5 u (A + C).  The band is 8 u (A + C).
   - Candidates, order, spacing: a pixel whose score sits within the band
     of the quality cut or of a neighbour's score, or two candidates whose
     bands overlap, are decisions either side may take; the GPU's corners
     must be a result the greedy selection can reach with SOME resolution
     of those decisions (validity, spacing, order, maximality), and must
     equal the oracle's exactly when no decision is ambiguous.
   - RANSAC: a pair whose squared reprojection error lies within a relative
     1e-6 of thr^2 is a decision either side may take (the GPU tests the
     same inequality without a division and rounds its models differently
     in principle); counts, the winner and inlier sets must agree up to
     those pairs.

2. Agreement with the kernels' own arithmetic (an emulator, NOT the oracle):
   numpy float32 evaluates the kernel's score in its operation order, and
   numpy float64 evaluates the kernel's division-free inlier test
   |(X, Y) - Z dst|^2 < thr^2 Z^2 on the oracle's hypothesis models (the
   kernel solves the same elimination without contraction).  The GPU must
   equal the emulator exactly; the emulator is itself checked against the
   oracle within the bands above (CPU tests)."""
from __future__ import annotations

import numpy as np

import oracle

U32 = 2.0 ** -24
SCORE_BAND = 8.0          # x u (A + C)
RANSAC_BAND = 1e-6        # relative, on the squared reprojection error
KMAX = 8192               # candidates the selection considers


# ----------------------------------------------------------------- scores
def score_band(A: np.ndarray, C: np.ndarray) -> np.ndarray:
    return SCORE_BAND * U32 * (A + C) + 1e-300


def emu_scores(A: np.ndarray, B: np.ndarray, C: np.ndarray) -> np.ndarray:
    """The kernel's FP32 score, operation by operation (round to nearest)."""
    f32 = np.float32
    fa, fb, fc = A.astype(f32), B.astype(f32), C.astype(f32)
    t = fa + fc
    d = fa - fc
    e = d * d
    f = fb * fb
    g = f32(4.0) * f
    rr = np.sqrt(e + g)
    v = f32(0.5) * (t - rr)
    return np.where(v > 0, v, f32(0.0)).astype(f32)


def _neighbour_views(a: np.ndarray):
    """For the interior (1..H-2, 1..W-2): the 8 shifted views of a."""
    h, w = a.shape[:2]
    return [a[1 + j:h - 1 + j, 1 + i:w - 1 + i] for j in (-1, 0, 1) for i in (-1, 0, 1)
            if (i, j) != (0, 0)]


def greedy(order_xy: np.ndarray, min_distance: float, max_corners: int) -> np.ndarray:
    """Greedy spacing (M4) over candidates already in selection order."""
    md2 = float(min_distance) ** 2
    kept = np.zeros((0, 2), np.int64)
    out = []
    for x, y in order_xy:
        if len(kept):
            d2 = (kept[:, 0] - x) ** 2 + (kept[:, 1] - y) ** 2
            if np.any(d2 < md2):
                continue
        kept = np.vstack([kept, [[x, y]]])
        out.append((x, y))
        if len(out) == max_corners:
            break
    return np.array(out, np.int64).reshape(-1, 2)


def emu_corners(img: np.ndarray, block_size=3, quality=0.01, min_distance=10.0, max_corners=500):
    """The kernels' selection on their FP32 scores: candidates above the FP32
    cut quality * max, local maxima, the 8192 strongest (score descending,
    index ascending), greedy spacing.  Returns (xy, scores, n_candidates)."""
    A, B, C = oracle.tensor_map(img, block_size)
    s = emu_scores(A, B, C)
    h, w = s.shape
    cut = np.float32(np.float32(quality) * s.max())
    c = s[1:-1, 1:-1]
    lm = np.ones_like(c, bool)
    for v in _neighbour_views(s):
        lm &= ~(v > c)
    cand = lm & (c > cut) & (c > 0)
    ys, xs = np.nonzero(cand)
    ys, xs = ys + 1, xs + 1
    sc = s[ys, xs]
    idx = ys.astype(np.int64) * w + xs
    order = np.lexsort((idx, -sc.astype(np.float64)))[:KMAX]
    xy = np.c_[xs[order], ys[order]]
    kept = greedy(xy, min_distance, max_corners)
    pos = {tuple(p): k for k, p in enumerate(xy.tolist())}
    ksc = np.array([sc[order][pos[tuple(p)]] for p in kept.tolist()], np.float32)
    return kept, ksc, int(len(xs))


# ------------------------------------------------------- corners vs oracle
def check_corners(img, gxy, gsc, gnc, block_size=3, quality=0.01, min_distance=10.0,
                  max_corners=500):
    """Assert that the GPU's corners (gxy, gsc) and candidate count gnc are
    a selection the method reaches under FP32 rounding of its FP64 scores
    (see the module docstring); returns statistics of the ambiguity."""
    A, B, C = oracle.tensor_map(img, block_size)
    s = oracle.score_map(img, block_size)
    D = score_band(A, C)
    h, w = s.shape
    oxy, osc, onc = oracle.corners(img, block_size, quality, min_distance, max_corners)
    mx = float(s.max())
    near_max = s >= mx - 2.0 * float(D.max())
    dmx = float(D[near_max].max())
    cut = quality * mx
    dcut = quality * dmx + 4.0 * U32 * quality * mx + 1e-300
    tens = np.stack([A, B, C], -1)
    ci, di = s[1:-1, 1:-1], D[1:-1, 1:-1]
    ti = tens[1:-1, 1:-1]
    sure_lm = np.ones_like(ci, bool)
    maybe_lm = np.ones_like(ci, bool)
    for v, dv, tv in zip(_neighbour_views(s), _neighbour_views(D), _neighbour_views(tens)):
        same = np.all(tv == ti, -1)
        sure_lm &= same | (ci - di >= v + dv)
        maybe_lm &= same | (v - dv <= ci + di)
    definite = sure_lm & (ci - di > cut + dcut)
    possible = maybe_lm & (ci + di > cut - dcut) & (ci + di > 0)
    n_def, n_pos = int(definite.sum()), int(possible.sum())
    assert n_def <= onc <= n_pos, (n_def, onc, n_pos)          # the oracle is one resolution
    assert n_def <= gnc <= n_pos, (n_def, gnc, n_pos)
    gxy = np.asarray(gxy, np.int64).reshape(-1, 2)
    gsc = np.asarray(gsc, np.float64)
    m = len(gxy)
    assert 0 < m <= max_corners or onc == 0
    gx, gy = gxy[:, 0], gxy[:, 1]
    # (a) every corner is a possible candidate, (c) its score is within the band
    assert np.all(possible[gy - 1, gx - 1]), "a corner that cannot be a candidate"
    assert np.all(np.abs(gsc - s[gy, gx]) <= D[gy, gx]), np.abs(gsc - s[gy, gx]).max()
    # (b) spacing
    md2 = float(min_distance) ** 2
    if m > 1:
        d2 = (gx[:, None] - gx[None]) ** 2 + (gy[:, None] - gy[None]) ** 2
        np.fill_diagonal(d2, 1 << 40)
        assert d2.min() >= md2
    # (d) strongest first, ties by index
    gidx = gy * w + gx
    assert np.all((np.diff(gsc) < 0) | ((np.diff(gsc) == 0) & (np.diff(gidx) > 0)))
    # (f) maximality: a definite candidate that is certainly considered (fewer
    # than KMAX possible candidates can rank above it) and certainly ranks
    # above the last accepted corner (when the list is full) is accepted or
    # blocked by a corner within min_distance that may rank above it
    py, px = np.nonzero(possible)
    up = (ci + di)[py, px]
    up_sorted = np.sort(up)
    dy, dx = np.nonzero(definite)
    lo = (ci - di)[dy, dx]
    ahead = len(up_sorted) - np.searchsorted(up_sorted, lo, side="left") - 1
    cons = ahead < KMAX
    if m == max_corners:
        last = s[gy[-1], gx[-1]] + D[gy[-1], gx[-1]]
        cons &= lo > last
    cx, cy = dx[cons] + 1, dy[cons] + 1
    clo = lo[cons]
    inG = np.zeros((h, w), bool)
    inG[gy, gx] = True
    free = ~inG[cy, cx]
    cx, cy, clo = cx[free], cy[free], clo[free]
    gup = s[gy, gx] + D[gy, gx]
    for k0 in range(0, len(cx), 1024):
        sx, sy, sl = cx[k0:k0 + 1024], cy[k0:k0 + 1024], clo[k0:k0 + 1024]
        d2 = (sx[:, None] - gx[None]) ** 2 + (sy[:, None] - gy[None]) ** 2
        blocked = np.any((d2 < md2) & (gup[None] >= sl[:, None]), axis=1)
        assert np.all(blocked), f"{int((~blocked).sum())} definite candidates neither kept nor blocked"
    # ambiguity of the whole selection: candidacy, and overlapping bands among
    # the possible candidates (identical tensors give identical scores on both sides)
    amb_cand = n_pos - n_def
    order = np.argsort(up)
    lo_p = (ci - di)[py, px][order]
    up_p = up[order]
    tp = ti[py, px][order]
    overl = (lo_p[1:] <= up_p[:-1]) & ~np.all(tp[1:] == tp[:-1], -1)
    amb_order = int(overl.sum())
    if amb_cand == 0 and amb_order == 0:
        assert gnc == onc
        assert np.array_equal(gxy, oxy)
    common = len(set(map(tuple, gxy.tolist())) & set(map(tuple, np.asarray(oxy).tolist())))
    return dict(corners=m, oracle_corners=len(oxy), common=common, candidates=gnc,
                oracle_candidates=onc, ambiguous_candidates=amb_cand, ambiguous_order=amb_order)


# --------------------------------------------------------------- RANSAC
def emu_inliers(Hm, src, dst, thr):
    """The kernel's FP64 division-free inlier test, as written."""
    Hm = np.asarray(Hm, np.float64).reshape(9)
    x, y = src[:, 0], src[:, 1]
    X = Hm[0] * x + Hm[1] * y + Hm[2]
    Y = Hm[3] * x + Hm[4] * y + Hm[5]
    Z = Hm[6] * x + Hm[7] * y + Hm[8]
    t2 = thr * thr
    ex = X - dst[:, 0] * Z
    ey = Y - dst[:, 1] * Z
    return (Z > 0.0) & (ex * ex + ey * ey < t2 * Z * Z)


def emu_ransac(src, dst, W, H, iters, thr, seed):
    """Per-hypothesis counts of the kernel's test on the oracle's models; the
    winner (most inliers, lowest index), its count and inlier mask."""
    counts = np.full(iters, -1, np.int64)
    best, bc, binl = -1, -1, None
    for m in range(iters):
        Hm = oracle.hypothesis(src, dst, W, H, seed, m)
        if Hm is None:
            continue
        inl = emu_inliers(Hm, src, dst, thr)
        counts[m] = int(inl.sum())
        if counts[m] > bc:
            best, bc, binl = m, int(counts[m]), inl
    return best, bc, binl, counts


def check_ransac(src, dst, W, H, iters, thr, seed, gH, ginl, gbest, gcount, corner_tol=0.05):
    """Assert that the GPU's RANSAC result is one the FP64 oracle's method
    reaches up to pairs within the band of the threshold; returns statistics."""
    counts, near = oracle.ransac_counts(src, dst, W, H, iters, thr, seed, RANSAC_BAND)
    oH, oinl, ocnt, obest = oracle.ransac(src, dst, W, H, iters=iters, thresh=thr, seed=seed)
    valid = counts >= 0
    if not valid.any():
        assert gcount == -1
        return dict(best=-1)
    assert gbest >= 0 and counts[gbest] >= 0
    lo, hi = counts - near, counts + near
    assert hi[gbest] >= lo[valid].max(), "a winner no rounding of the counts makes"
    assert lo[gbest] <= gcount <= hi[gbest]
    others = np.where(valid & (np.arange(iters) != obest))[0]
    if len(others) == 0 or lo[obest] > hi[others].max():
        assert gbest == obest                       # the oracle's winner is unambiguous
    Hb = oracle.hypothesis(src, dst, W, H, seed, gbest)
    binl, bnear = oracle.inliers(Hb, src, dst, thr, RANSAC_BAND)
    diff = np.asarray(ginl, bool) != binl
    assert not np.any(diff & ~bnear), "inlier decisions outside the band differ"
    corners = np.array([[0, 0], [W, 0], [0, H], [W, H]], float)
    q = lambda M, p: (np.c_[p, np.ones(len(p))] @ np.asarray(M).T)  # noqa: E731
    at = lambda M: (lambda v: v[:, :2] / v[:, 2:])(q(M, corners))  # noqa: E731
    # the refit (M8) of the GPU's own inlier set, as the oracle computes it
    Hr = oracle.refit(src, dst, np.asarray(ginl, bool), W, H) if gcount >= 4 else None
    if Hr is not None:
        assert float(np.abs(at(gH) - at(Hr)).max()) < 1e-6
    err = float(np.abs(at(gH) - at(oH)).max())
    if gbest == obest and not diff.any():
        assert err < 1e-6, err                      # same inliers: the same least squares
    else:
        assert err < corner_tol, err
    return dict(best=int(gbest), oracle_best=int(obest), count=int(gcount), oracle_count=int(ocnt),
                near_pairs=int(near[gbest]), inlier_diffs=int(diff.sum()), corner_err_px=err)

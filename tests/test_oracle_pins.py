"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test fixes one part of arXiv:1702.05156 Sec. 2.2-2.4 by a closed form,
an exact symmetry, a hand-computed fixture or brute-force counting, so that a
dropped term, a wrong sign, a swapped index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import DIAG, oracle_step, state_from_arrays
from paper_1702_05156_gb300.synth import random_state, translation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _q(s):
    """'a' or 'a/b' with decimal a and b, evaluated exactly."""
    if not isinstance(s, str):
        return float(s)
    num, _, den = s.partition("/")
    return float(Fraction(num) / Fraction(den or "1"))


# ---------------------------------------------------------------- hand fixture
def test_hand_computed_8x8_sequence():
    """Three frames computed by hand (tests/golden/hand_8x8.json): pins the
    mean/variance/age equations (Sec. 2.2), V with the UPDATED mean, the
    match -> candidate -> reset -> swap order (Sec. 2.3) and the mask taken
    after the swap."""
    with open(os.path.join(GOLDEN, "hand_8x8.json")) as f:
        g = json.load(f)
    st = None
    for fr in g["frames"]:
        img = np.array(fr["pixels"], dtype=np.uint8)
        st, mask = oracle_step(img, np.eye(3), st, block=g["block"], theta_s=g["theta_s"],
                               theta_d=g["theta_d"], age_max=g["age_max"])
        e = fr["expect"]
        for name in ("muA", "varA", "muC", "varC"):
            exp = np.array([_q(v) for v in e[name]]).reshape(2, 2)
            np.testing.assert_allclose(getattr(st, name), exp, rtol=1e-13, atol=0, err_msg=name)
        for name in ("ageA", "ageC"):
            np.testing.assert_array_equal(getattr(st, name), np.array(e[name]).reshape(2, 2), name)
        np.testing.assert_array_equal(mask, np.array(e["mask"], dtype=np.uint8))


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("block", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("c", [0, 37, 255])
def test_constant_frame_identity_closed_form(block, c):
    """Identity H and a constant frame c: mu == c, var_n = 255/n while the
    age n <= 30, then var_n = (255/30) * (30/31)^(n-30) at the cap; ages
    1, 2, ..., 30, 30, ...; the candidate stays (c, 255, 1); the mask is
    empty on every frame (Sec. 2.2 equations with V = 0)."""
    W, H = 16, 8
    img = np.full((H, W), c, dtype=np.uint8)
    st = None
    for n in range(1, 46):
        st, mask = oracle_step(img, np.eye(3), st, block=block)
        np.testing.assert_allclose(st.muA, c, rtol=0, atol=1e-12)
        exp_var = 255.0 / n if n <= 30 else (255.0 / 30) * (30.0 / 31.0) ** (n - 30)
        np.testing.assert_allclose(st.varA, exp_var, rtol=1e-12)
        assert (st.ageA == min(n, 30)).all()
        assert (st.muC == c).all() and (st.varC == 255).all() and (st.ageC == 1).all()
        assert mask.sum() == 0


def test_swap_script_and_age_cap_quirk():
    """Background 50 for 10 frames, then 200: the candidate is reset at frame
    11, grows one year per frame and wins at frame 21 when its age 11 exceeds
    the apparent age 10 (Sec. 2.3, strict '>').  Before the swap every pixel
    is foreground against A = 50, right after it none is.  If the apparent
    model has reached the cap (age 30), a candidate capped at 30 can never
    exceed it and no swap ever happens."""
    W = H = 8
    bg = np.full((H, W), 50, np.uint8)
    fg = np.full((H, W), 200, np.uint8)
    st = None
    for t in range(1, 11):
        st, _ = oracle_step(bg, np.eye(3), st, block=4)
    assert (st.ageA == 10).all()
    for t in range(11, 22):
        st, mask, dg = oracle_step(fg, np.eye(3), st, block=4, diag=True)
        k = t - 10  # frames of the new background so far
        if t < 21:
            assert (st.muA == 50).all() and (st.ageA == 10).all()
            assert (st.ageC == k).all()
            np.testing.assert_allclose(st.muC, 200, rtol=1e-14)
            np.testing.assert_allclose(st.varC, 255.0 / k, rtol=1e-12)
            assert mask.all()
            assert (dg[..., DIAG["BRANCH"]] == (2 if t == 11 else 1)).all()
        else:
            assert (dg[..., DIAG["SWAP"]] == 1).all()
            np.testing.assert_allclose(st.muA, 200, rtol=1e-14)
            assert (st.ageA == 11).all()
            np.testing.assert_allclose(st.varA, 255.0 / 11, rtol=1e-12)
            assert (st.muC == 200).all() and (st.varC == 255).all() and (st.ageC == 1).all()
            assert mask.sum() == 0

    st = None
    for t in range(40):
        st, _ = oracle_step(bg, np.eye(3), st, block=4)
    for t in range(60):
        st, mask = oracle_step(fg, np.eye(3), st, block=4)
    np.testing.assert_allclose(st.muA, 50, rtol=1e-14)
    np.testing.assert_allclose(st.muC, 200, rtol=1e-14)
    assert (st.ageA == 30).all() and (st.ageC == 30).all()
    assert mask.all()


# ---------------------------------------------------------------- compensation
def _shift_blocks(a, k, l, fill):
    out = np.full_like(a, fill)
    gy, gx = a.shape
    ys = slice(max(l, 0), gy + min(l, 0))
    xs = slice(max(k, 0), gx + min(k, 0))
    ys0 = slice(max(-l, 0), gy + min(-l, 0))
    xs0 = slice(max(-k, 0), gx + min(-k, 0))
    out[ys, xs] = a[ys0, xs0]
    return out


@pytest.mark.parametrize("block", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("k,l", [(1, 0), (0, 1), (-2, 3), (3, -1), (0, 0)])
def test_whole_block_translation_is_an_exact_shift(block, k, l):
    """Content moving by (k*B, l*B) px: the compensated state of block
    (bx, by) is EXACTLY the previous state of block (bx-k, by-l) (all weight
    on one block); blocks whose source is off the grid have no source and
    restart both models at (M, 255, 1)."""
    gx, gy = 11, 7
    W, H = gx * block, gy * block
    prev = state_from_arrays(*random_state(gy, gx, 30, seed=5))
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    Hm = translation(k * block, l * block)
    st, mask, dg = oracle_step(img, Hm, prev, block=block, diag=True)
    nos = _shift_blocks(np.zeros((gy, gx)), k, l, 1.0) > 0
    assert (dg[..., DIAG["NOSRC"]].astype(bool) == nos).all()
    for name, col in (("muA", "MU_A"), ("varA", "VAR_A"), ("muC", "MU_C"), ("varC", "VAR_C"),
                      ("ageA", "XAGE_A"), ("ageC", "XAGE_C")):
        exp = _shift_blocks(getattr(prev, name).astype(np.float64), k, l, np.nan)
        got = dg[..., DIAG[col]]
        assert np.array_equal(got[~nos], exp[~nos]), name
    # the whole step equals an identity step on the shifted state
    shifted = state_from_arrays(*[_shift_blocks(getattr(prev, n), k, l, 1)
                                  for n in ("muA", "varA", "ageA", "muC", "varC", "ageC")])
    st2, mask2 = oracle_step(img, np.eye(3), shifted, block=block)
    M = img.reshape(gy, block, gx, block).mean(axis=(1, 3))
    for n in ("muA", "varA", "ageA", "muC", "varC", "ageC"):
        a, b = getattr(st, n), getattr(st2, n)
        assert np.array_equal(a[~nos], b[~nos]), n
    assert np.array_equal(st.muA[nos], M[nos]) and (st.varA[nos] == 255).all()
    assert (st.ageA[nos] == 1).all() and (st.ageC[nos] == 1).all()
    pix_nos = np.kron(nos, np.ones((block, block), bool))
    assert np.array_equal(mask[~pix_nos], mask2[~pix_nos])


def test_fractional_shifts_hand_weights():
    """Sub-block shifts with hand-derived weights (B = 4, block centres at
    4*b + 2).  Content moving right by 2 px: the back-projected square starts
    at u = bx - 1/2, so blocks bx-1 and bx get 1/2 each; at the left edge only
    block 0 is in the grid and renormalisation gives it all the weight.  An
    age mix of 1 and 2 gives 1.5, rounded half up to 2.  Moving right 1 px:
    weights 1/4 (bx-1) and 3/4 (bx).  Moving (1, 3) px: rows by-1 / by get
    3/4 / 1/4, columns 1/4 / 3/4."""
    gx, gy = 4, 3
    muA = np.arange(gx * gy, dtype=np.float64).reshape(gy, gx) * 10 + 5
    varA = np.arange(gx * gy, dtype=np.float64).reshape(gy, gx) + 1
    ageA = (np.arange(gx * gy).reshape(gy, gx) % 7 + 1).astype(np.int32)
    prev = state_from_arrays(muA, varA, ageA, muA + 1, varA + 2, ageA)
    img = np.zeros((gy * 4, gx * 4), np.uint8)

    _, _, dg = oracle_step(img, translation(2, 0), prev, block=4, diag=True)
    for by in range(gy):
        for bx in range(gx):
            if bx == 0:
                e_mu, e_age = muA[by, 0], float(ageA[by, 0])
                e_w = 0.5
            else:
                e_mu = 0.5 * muA[by, bx - 1] + 0.5 * muA[by, bx]
                e_age = 0.5 * ageA[by, bx - 1] + 0.5 * ageA[by, bx]
                e_w = 1.0
            assert dg[by, bx, DIAG["WSUM"]] == e_w
            assert dg[by, bx, DIAG["MU_A"]] == e_mu
            assert dg[by, bx, DIAG["XAGE_A"]] == e_age
    # rounding half up: ages 1 and 2 -> 1.5 -> 2
    prev2 = state_from_arrays(muA, varA, np.array([[1, 2, 1, 2]] * gy, np.int32),
                              muA, varA, np.array([[2, 3, 2, 3]] * gy, np.int32))
    _, _, dg = oracle_step(img, translation(2, 0), prev2, block=4, diag=True)
    assert dg[0, 1, DIAG["XAGE_A"]] == 1.5 and dg[0, 1, DIAG["XAGE_C"]] == 2.5

    _, _, dg = oracle_step(img, translation(1, 0), prev, block=4, diag=True)
    for bx in range(1, gx):
        assert dg[1, bx, DIAG["MU_A"]] == 0.25 * muA[1, bx - 1] + 0.75 * muA[1, bx]

    _, _, dg = oracle_step(img, translation(1, 3), prev, block=4, diag=True)
    for by in range(1, gy):
        for bx in range(1, gx):
            e = (0.25 * 0.75 * muA[by - 1, bx - 1] + 0.75 * 0.75 * muA[by - 1, bx]
                 + 0.25 * 0.25 * muA[by, bx - 1] + 0.75 * 0.25 * muA[by, bx])
            assert abs(dg[by, bx, DIAG["MU_A"]] - e) < 1e-12


def test_half_up_age_rounding_enters_the_update():
    """A mixed age of 1.5 rounds to 2, so a matching block's stored age is 3
    and its learning rate is 1/3 (Sec. 2.2 with the rounded age~)."""
    gx, gy = 3, 1
    mu = np.full((gy, gx), 100.0)
    prev = state_from_arrays(mu, np.full((gy, gx), 50.0), np.array([[1, 2, 1]], np.int32),
                             mu, np.full((gy, gx), 50.0), np.array([[1, 1, 1]], np.int32))
    img = np.full((4, 12), 103, np.uint8)
    st, _, dg = oracle_step(img, translation(2, 0), prev, block=4, diag=True)
    assert dg[0, 1, DIAG["XAGE_A"]] == 1.5 and dg[0, 1, DIAG["BRANCH"]] == 0
    assert st.ageA[0, 1] == 3
    assert abs(st.muA[0, 1] - (2 / 3 * 100 + 1 / 3 * 103)) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_mixing_weights_equal_brute_force_overlap_area(seed):
    """R6: the mixing weight of a previous block is the area that the
    back-projected BxB square shares with it.  Shifts are multiples of B/16
    px, so counting the 16x16 sub-cells of the square that fall in each
    block is exact; the oracle's compensated mean must equal the area-
    weighted mean of the in-grid blocks, renormalised."""
    rng = np.random.default_rng(seed)
    B, S = 4, 16
    gx, gy = 6, 5
    prev = state_from_arrays(*random_state(gy, gx, 30, seed=seed + 10))
    dx = rng.integers(-3 * S, 3 * S) * B / S
    dy = rng.integers(-3 * S, 3 * S) * B / S
    img = np.zeros((gy * B, gx * B), np.uint8)
    _, _, dg = oracle_step(img, translation(dx, dy), prev, block=B, diag=True)
    for by in range(gy):
        for bx in range(gx):
            # square top-left in pixels (in the previous frame)
            qx = bx * B - dx
            qy = by * B - dy
            area = {}
            for sy in range(S):
                for sx in range(S):
                    px = qx + (sx + 0.5) * B / S
                    py = qy + (sy + 0.5) * B / S
                    cell = (int(np.floor(py / B)), int(np.floor(px / B)))
                    area[cell] = area.get(cell, 0) + 1
            inn = {c: a for c, a in area.items() if 0 <= c[0] < gy and 0 <= c[1] < gx}
            tot = sum(inn.values())
            assert dg[by, bx, DIAG["WSUM"]] == pytest.approx(tot / S ** 2, abs=1e-12)
            if tot / S ** 2 < 1e-3:
                assert dg[by, bx, DIAG["NOSRC"]] == 1
                continue
            e_mu = sum(a * prev.muA[c] for c, a in inn.items()) / tot
            e_var = sum(a * prev.varC[c] for c, a in inn.items()) / tot
            e_age = sum(a * prev.ageA[c] for c, a in inn.items()) / tot
            assert dg[by, bx, DIAG["MU_A"]] == pytest.approx(e_mu, rel=1e-12)
            assert dg[by, bx, DIAG["VAR_C"]] == pytest.approx(e_var, rel=1e-12)
            assert dg[by, bx, DIAG["XAGE_A"]] == pytest.approx(e_age, rel=1e-12)


def test_no_source_cases():
    """R10: a homography that sends every block off the grid, one with
    Z <= 0, and the first frame all restart both models at (M, 255, 1)."""
    gx, gy = 4, 4
    prev = state_from_arrays(*random_state(gy, gx, 30, seed=3))
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (16, 16), dtype=np.uint8)
    M = img.reshape(4, 4, 4, 4).mean(axis=(1, 3))
    flip = np.diag([1.0, 1.0, -1.0])  # Z = -1 everywhere
    for Hm in (translation(1000, 0), flip):
        st, _, dg = oracle_step(img, Hm, prev, block=4, diag=True)
        assert (dg[..., DIAG["NOSRC"]] == 1).all()
        assert np.array_equal(st.muA, M) and np.array_equal(st.muC, M)
        assert (st.varA == 255).all() and (st.ageA == 1).all() and (st.ageC == 1).all()


# ---------------------------------------------------------------- symmetries
def _random_case(seed, gx=9, gy=6, B=4):
    rng = np.random.default_rng(seed)
    prev = state_from_arrays(*random_state(gy, gx, 30, seed=seed))
    # frames close to the state so that all three branches occur
    base = np.kron(prev.muA, np.ones((B, B)))
    img = np.clip(base + rng.normal(0, 6, base.shape) + (rng.random(base.shape) < 0.2) * 90,
                  0, 255).round().astype(np.uint8)
    th = np.radians(rng.uniform(-2, 2))
    s = 1 + rng.uniform(-0.02, 0.02)
    Hm = np.array([[s * np.cos(th), -s * np.sin(th), rng.uniform(-5, 5)],
                   [s * np.sin(th), s * np.cos(th), rng.uniform(-5, 5)],
                   [rng.uniform(-1e-4, 1e-4), rng.uniform(-1e-4, 1e-4), 1.0]])
    return prev, img, Hm


@pytest.mark.parametrize("seed", range(4))
def test_mirror_symmetry(seed):
    """Mirroring the frame left-right, the state and the homography
    (conjugated by x -> W - x) mirrors every output.  Catches swapped
    neighbour weights and x/y index slips in the compensation."""
    prev, img, Hm = _random_case(seed)
    gy, gx = prev.muA.shape
    W = gx * 4
    Fm = np.array([[-1.0, 0, W], [0, 1, 0], [0, 0, 1]])
    st, mask, dg = oracle_step(img, Hm, prev, block=4, diag=True)
    fprev = state_from_arrays(*[getattr(prev, n)[:, ::-1] for n in
                                ("muA", "varA", "ageA", "muC", "varC", "ageC")])
    st2, mask2, dg2 = oracle_step(img[:, ::-1], Fm @ Hm @ Fm, fprev, block=4, diag=True)
    assert len(set(dg[..., DIAG["BRANCH"]].ravel())) >= 3
    for n in ("muA", "varA", "muC", "varC"):
        np.testing.assert_allclose(getattr(st2, n)[:, ::-1], getattr(st, n), rtol=1e-10)
    for n in ("ageA", "ageC"):
        np.testing.assert_array_equal(getattr(st2, n)[:, ::-1], getattr(st, n))
    np.testing.assert_array_equal(mask2[:, ::-1], mask)


@pytest.mark.parametrize("seed", range(4))
def test_transpose_symmetry(seed):
    """Swapping x and y in the frame, state and homography transposes every
    output (square grid)."""
    prev, img, Hm = _random_case(seed, gx=7, gy=7)
    P = np.array([[0.0, 1, 0], [1, 0, 0], [0, 0, 1]])
    st, mask = oracle_step(img, Hm, prev, block=4)
    tprev = state_from_arrays(*[getattr(prev, n).T for n in
                                ("muA", "varA", "ageA", "muC", "varC", "ageC")])
    st2, mask2 = oracle_step(img.T, P @ Hm @ P, tprev, block=4)
    for n in ("muA", "varA", "muC", "varC"):
        np.testing.assert_allclose(getattr(st2, n).T, getattr(st, n), rtol=1e-10)
    for n in ("ageA", "ageC"):
        np.testing.assert_array_equal(getattr(st2, n).T, getattr(st, n))
    np.testing.assert_array_equal(mask2.T, mask)


@pytest.mark.parametrize("seed", range(4))
def test_negation_symmetry(seed):
    """I -> 255 - I with mu -> 255 - mu and the same variances and ages gives
    mu -> 255 - mu, var -> var, ages and mask unchanged: the equations only
    use differences and squares.  Catches a sign slip in V or the tests."""
    prev, img, Hm = _random_case(seed)
    st, mask = oracle_step(img, Hm, prev, block=4)
    nprev = state_from_arrays(255 - prev.muA, prev.varA, prev.ageA,
                              255 - prev.muC, prev.varC, prev.ageC)
    st2, mask2 = oracle_step(255 - img, Hm, nprev, block=4)
    np.testing.assert_allclose(255 - st2.muA, st.muA, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(255 - st2.muC, st.muC, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(st2.varA, st.varA, rtol=1e-10)
    np.testing.assert_allclose(st2.varC, st.varC, rtol=1e-10)
    np.testing.assert_array_equal(st2.ageA, st.ageA)
    np.testing.assert_array_equal(st2.ageC, st.ageC)
    np.testing.assert_array_equal(mask2, mask)


def test_interior_weights_sum_to_one():
    """Away from the border all four overlapped blocks are in the grid and
    the area weights sum to one for any homography."""
    prev, img, Hm = _random_case(7, gx=12, gy=12)
    _, _, dg = oracle_step(img, Hm, prev, block=4, diag=True)
    np.testing.assert_allclose(dg[3:-3, 3:-3, DIAG["WSUM"]], 1.0, rtol=0, atol=1e-12)


def test_variance_sample_min_max_identity():
    """max_j (mu - I_j)^2 over a block equals max((mu - min)^2, (max - mu)^2)
    (the shortcut the GPU uses), checked by brute force against the oracle's
    own output: V recovered from the variance update equals the min/max
    form built from the block's extreme pixels."""
    prev, img, Hm = _random_case(11)
    st, _, dg = oracle_step(img, Hm, prev, block=4, diag=True)
    upd = dg[..., DIAG["BRANCH"]] == 0
    a = np.floor(dg[..., DIAG["XAGE_A"]] + 0.5)
    V = (st.varA - a / (a + 1) * dg[..., DIAG["VAR_A"]]) * (a + 1)
    mn, mx = dg[..., DIAG["MIN"]], dg[..., DIAG["MAX"]]
    Vmm = np.maximum((st.muA - mn) ** 2, (mx - st.muA) ** 2)
    no_swap = dg[..., DIAG["SWAP"]] == 0
    sel = upd & no_swap
    assert sel.sum() > 5
    np.testing.assert_allclose(V[sel], Vmm[sel], rtol=1e-8, atol=1e-8)


def test_invalid_sizes_rejected():
    with pytest.raises(ValueError):
        oracle_step(np.zeros((6, 8), np.uint8), np.eye(3), None, block=0)


# ---------------------------------------------------------------- per-pixel model
def test_hand_computed_per_pixel_sequence():
    """Block 1 is the paper's own per-pixel model (M_i = I, V_i = (mu - I)^2).
    Five hand-computed frames (tests/golden/hand_b1.json) take one pixel
    through an apparent match, a candidate reset, a candidate match, a
    refused swap at equal ages (strict '>') and a swap; the other pixel is a
    constant control."""
    with open(os.path.join(GOLDEN, "hand_b1.json")) as f:
        g = json.load(f)
    st = None
    for fr in g["frames"]:
        img = np.array(fr["pixels"], dtype=np.uint8)
        st, mask = oracle_step(img, np.eye(3), st, block=1, theta_s=g["theta_s"],
                               theta_d=g["theta_d"], age_max=g["age_max"])
        e = fr["expect"]
        for name in ("muA", "varA", "muC", "varC"):
            exp = np.array([_q(v) for v in e[name]]).reshape(img.shape)
            np.testing.assert_allclose(getattr(st, name), exp, rtol=1e-13, atol=0, err_msg=name)
        for name in ("ageA", "ageC"):
            np.testing.assert_array_equal(getattr(st, name), np.array(e[name]).reshape(img.shape))
        np.testing.assert_array_equal(mask, np.array(e["mask"], dtype=np.uint8).reshape(img.shape))


# ---------------------------------------------------------------- clipped edge blocks (R11)
@pytest.mark.parametrize("W,H,block", [(10, 7, 4), (13, 10, 4), (16, 20, 16), (9, 5, 2), (17, 9, 8)])
def test_clipped_blocks_first_frame_brute_force(W, H, block):
    """Sides that are not multiples of B: the grid is ceil(W/B) x ceil(H/B);
    each block's M, min and max are those of its pixels inside the frame
    (brute force over the clipped slice), and on the first frame the mask is
    the per-pixel test against the reset model (M, 255)."""
    rng = np.random.default_rng(W * 31 + H)
    img = rng.integers(0, 256, (H, W), dtype=np.uint8)
    st, mask, dg = oracle_step(img, np.eye(3), None, block=block, diag=True)
    gy, gx = -(-H // block), -(-W // block)
    assert st.muA.shape == (gy, gx)
    Mpix = np.zeros((H, W))
    for by in range(gy):
        for bx in range(gx):
            sl = img[by * block:(by + 1) * block, bx * block:(bx + 1) * block].astype(np.float64)
            assert dg[by, bx, DIAG["M"]] == sl.mean()
            assert dg[by, bx, DIAG["MIN"]] == sl.min() and dg[by, bx, DIAG["MAX"]] == sl.max()
            assert st.muA[by, bx] == sl.mean() and st.varA[by, bx] == 255
            Mpix[by * block:(by + 1) * block, bx * block:(bx + 1) * block] = sl.mean()
    np.testing.assert_array_equal(mask, ((img - Mpix) ** 2 > 4.0 * 255).astype(np.uint8))


@pytest.mark.parametrize("W,H,block", [(10, 7, 4), (18, 21, 8), (16, 9, 16)])
@pytest.mark.parametrize("c", [3, 200])
def test_clipped_blocks_constant_closed_form(W, H, block, c):
    """A constant frame follows the full-block closed form in every block,
    clipped ones included: their mean over the pixels inside the frame is
    exactly c and their V is 0."""
    img = np.full((H, W), c, dtype=np.uint8)
    st = None
    for n in range(1, 35):
        st, mask = oracle_step(img, np.eye(3), st, block=block)
        np.testing.assert_allclose(st.muA, c, rtol=0, atol=1e-12)
        exp_var = 255.0 / n if n <= 30 else (255.0 / 30) * (30.0 / 31.0) ** (n - 30)
        np.testing.assert_allclose(st.varA, exp_var, rtol=1e-12)
        assert (st.ageA == min(n, 30)).all() and mask.sum() == 0


@pytest.mark.parametrize("W,H,block", [(13, 10, 4), (21, 19, 8), (9, 7, 2)])
def test_identity_motion_crop_invariance(W, H, block):
    """With the identity homography no block mixes with another, so the
    whole blocks of a clipped frame evolve exactly as the same pixels cropped
    to a multiple of the block size."""
    rng = np.random.default_rng(block + W)
    frames = np.clip(rng.normal(120, 25, (6, H, W)), 0, 255).astype(np.uint8)
    frames[3:, : H // 2] = 30
    gx, gy = W // block, H // block
    st = sc = None
    for t in range(6):
        st, m = oracle_step(frames[t], np.eye(3), st, block=block)
        sc, mc = oracle_step(frames[t, : gy * block, : gx * block], np.eye(3), sc, block=block)
        for n in ("muA", "varA", "ageA", "muC", "varC", "ageC"):
            assert np.array_equal(getattr(st, n)[:gy, :gx], getattr(sc, n)), n
        assert np.array_equal(m[: gy * block, : gx * block], mc)


def test_run_equals_repeated_steps():
    rng = np.random.default_rng(2)
    frames = rng.integers(0, 256, (5, 8, 16), dtype=np.uint8)
    Hs = np.stack([np.eye(3), translation(1, 0), translation(0, 2), translation(-3, 1),
                   np.eye(3)])
    st_run, masks = oracle.oracle_run(frames, Hs, block=4)
    st = None
    for t in range(5):
        st, m = oracle_step(frames[t], Hs[t], st, block=4)
        np.testing.assert_array_equal(m, masks[t])
    for n in ("muA", "varA", "ageA", "muC", "varC", "ageC"):
        np.testing.assert_array_equal(getattr(st, n), getattr(st_run, n))


def test_clipped_block_variance_sees_only_its_pixels():
    """Right-edge blocks of a 10-px-wide frame (B = 4) hold 2 columns. Those
    columns are constant while the rest of the frame is random, so their V
    is 0 and their variance follows the closed form; a V loop over all B
    columns would wrap into the next row's random pixels."""
    W, H, B = 10, 8, 4
    rng = np.random.default_rng(4)
    st = None
    for n in range(1, 8):
        img = rng.integers(0, 256, (H, W), dtype=np.uint8)
        img[:, 8:] = 77
        st, mask = oracle_step(img, np.eye(3), st, block=B)
        np.testing.assert_allclose(st.muA[:, 2], 77, rtol=0, atol=1e-12)
        np.testing.assert_allclose(st.varA[:, 2], 255.0 / n, rtol=1e-12)
        assert (st.ageA[:, 2] == n).all() and mask[:, 8:].sum() == 0


# ---------------------------------------------------------------- mixture spread (R12)
def test_spread_half_half_hand_value():
    """A half-block shift mixes two blocks with weights 1/2: the compensated
    variance is the mean of their variances plus the spread of their means,
    (v1 + v2)/2 + ((m1 - m2)/2)^2 (the variance of an equal two-component
    mixture), and the mean is unchanged by the option."""
    B, gx, gy = 4, 3, 1
    prev = state_from_arrays(np.array([[10.0, 50.0, 90.0]]), np.array([[4.0, 9.0, 16.0]]),
                             np.full((1, 3), 5), np.array([[20.0, 30.0, 40.0]]),
                             np.array([[1.0, 1.0, 1.0]]), np.full((1, 3), 2))
    img = np.full((gy * B, gx * B), 60, np.uint8)
    Hm = translation(B / 2, 0)   # block 1 draws half from block 0, half from block 1
    _, _, d0 = oracle_step(img, Hm, prev, block=B, diag=True)
    _, _, d1 = oracle_step(img, Hm, prev, block=B, diag=True, mix_spread=True)
    assert d0[0, 1, DIAG["MU_A"]] == d1[0, 1, DIAG["MU_A"]] == 30.0
    assert d0[0, 1, DIAG["VAR_A"]] == (4.0 + 9.0) / 2
    assert d1[0, 1, DIAG["VAR_A"]] == (4.0 + 9.0) / 2 + 20.0 ** 2
    assert d1[0, 1, DIAG["VAR_C"]] == 1.0 + 5.0 ** 2


@pytest.mark.parametrize("k,l", [(1, 0), (-2, 1), (0, 0)])
def test_spread_vanishes_on_whole_block_shifts(k, l):
    """All weight on one block: no spread, so the option changes nothing."""
    gx, gy, B = 9, 6, 4
    prev = state_from_arrays(*random_state(gy, gx, 30, seed=3))
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, (gy * B, gx * B), dtype=np.uint8)
    a = oracle_step(img, translation(k * B, l * B), prev, block=B)
    b = oracle_step(img, translation(k * B, l * B), prev, block=B, mix_spread=True)
    for n in ("muA", "varA", "ageA", "muC", "varC", "ageC"):
        assert np.array_equal(getattr(a[0], n), getattr(b[0], n)), n
    assert np.array_equal(a[1], b[1])


def test_spread_is_the_mixture_variance_by_sampling_weights():
    """For a fractional shift the spread term equals the weighted variance
    of the four source means about their weighted mean, computed here by
    brute force over a 1000x1000 sub-cell count of the overlap (the same
    counting as the weight pin), so no formula of the oracle is retyped."""
    B = 4
    prev = state_from_arrays(np.array([[10.0, 70.0], [40.0, 100.0]]), np.zeros((2, 2)),
                             np.full((2, 2), 3), np.zeros((2, 2)), np.zeros((2, 2)),
                             np.full((2, 2), 1))
    img = np.zeros((8, 8), np.uint8)
    dx, dy = 0.3, 0.8                       # block units
    Hm = translation(-dx * B, -dy * B)      # block (0, 0) back-projects to [dx, dx+1) x [dy, dy+1)
    _, _, d = oracle_step(img, Hm, prev, block=B, diag=True, mix_spread=True)
    # brute force: the back-projected square of block (0, 0) covers [dx, dx+1) x [dy, dy+1)
    n = 1000
    c = (np.arange(n) + 0.5) / n
    xs, ys = dx + c, dy + c
    ix, iy = np.floor(xs).astype(int), np.floor(ys).astype(int)
    vals = prev.muA[np.clip(iy, 0, 1)[:, None], np.clip(ix, 0, 1)[None, :]]
    inside = ((iy < 2)[:, None] & (ix < 2)[None, :])
    v = vals[inside]
    np.testing.assert_allclose(d[0, 0, DIAG["VAR_A"]], v.var(), rtol=1e-3)


# ---------------------------------------------------------------- preprocessing (P1-P4)
def _brute_blur(img, q):
    h = len(q) // 2
    p = np.pad(img.astype(np.int64), h, mode="edge")
    k = np.outer(q, q).astype(np.int64)
    H, W = img.shape
    out = np.zeros((H, W), np.int64)
    for i in range(len(q)):
        for j in range(len(q)):
            out += k[i, j] * p[i:i + H, j:j + W]
    return (out >> 16).astype(np.uint8)


def _brute_median(img):
    p = np.pad(img, 1, mode="edge")
    H, W = img.shape
    win = np.stack([p[i:i + H, j:j + W] for i in range(3) for j in range(3)])
    return np.sort(win, axis=0)[4]


@pytest.mark.parametrize("n,sigma", [(3, 0.8), (5, 1.0), (5, 2.5), (7, 1.5), (9, 3.0)])
def test_gauss_weights_quantise_the_normalised_gaussian(n, sigma):
    """Weights sum to exactly 256, are symmetric and unimodal; each off-centre
    weight is the normalised Gaussian rounded to the nearest 1/256, and the
    centre weight takes up their rounding (at most (N-1)/2 steps of 1/256)."""
    q = oracle.gauss_weights(n, sigma)
    assert q.sum() == 256 and np.array_equal(q, q[::-1])
    assert np.all(np.diff(q[: n // 2 + 1]) >= 0)
    x = np.arange(n) - n // 2
    g = np.exp(-x.astype(np.float64) ** 2 / (2 * sigma ** 2))
    err = np.abs(q / 256.0 - g / g.sum())
    off = np.arange(n) != n // 2
    assert np.all(err[off] <= 0.5 / 256)
    assert err[n // 2] <= (n - 1) * 0.5 / 256


@pytest.mark.parametrize("shape", [(7, 9), (16, 16), (1, 5), (12, 3)])
@pytest.mark.parametrize("n,sigma", [(3, 0.8), (5, 1.0), (7, 1.5)])
def test_blur_equals_brute_force_clamped_convolution(shape, n, sigma):
    rng = np.random.default_rng(sum(shape) + n)
    img = rng.integers(0, 256, shape, dtype=np.uint8)
    got = oracle.prefilter(img, gauss_size=n, sigma=sigma, median=False)
    assert np.array_equal(got, _brute_blur(img, oracle.gauss_weights(n, sigma)))


@pytest.mark.parametrize("shape", [(7, 9), (16, 16), (1, 5), (2, 2), (12, 3)])
def test_median_equals_brute_force_clamped_window(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    img = rng.integers(0, 256, shape, dtype=np.uint8)
    got = oracle.prefilter(img, gauss_size=0, median=True)
    assert np.array_equal(got, _brute_median(img))
    both = oracle.prefilter(img, gauss_size=5, sigma=1.0, median=True)
    assert np.array_equal(both, _brute_median(_brute_blur(img, oracle.gauss_weights(5, 1.0))))


def test_filters_keep_constants_remove_impulses_keep_ramps():
    c = np.full((10, 12), 77, np.uint8)
    assert np.array_equal(oracle.prefilter(c, gauss_size=7, sigma=2.0), c)
    spike = c.copy()
    spike[4, 5] = 250
    assert np.array_equal(oracle.prefilter(spike, gauss_size=0, median=True), c)
    ramp = np.tile(np.arange(0, 240, 20, dtype=np.uint8), (10, 1))
    assert np.array_equal(oracle.prefilter(ramp, gauss_size=0, median=True), ramp)

"""CPU check of the error bound behind the RANSAC counts' FP32 pre-test
(csrc/dmsgm_homog_ransac.cu, ho_inlier_f32): its FP32 arithmetic, evaluated
here with numpy float32 (IEEE single, round to nearest, no contraction, as the
unit is built), must never decide a pair differently from the FP64 test of
Sec. 2.4's RANSAC (the oracle's |(X, Y) - Z dst|^2 < t^2 Z^2).  Pairs are
placed on the threshold to within a few ulps, where the pre-test has to leave
the decision to FP64, and spread uniformly, where it should decide almost all.
The kernel's constants are restated here: a change to them must change this
test too."""
import numpy as np

f32 = np.float32
U = f32(2.0 ** -24)


def _in_range(v64):
    v = v64.astype(np.float32)
    a = np.abs(v)
    return (v64 == 0) | ((a >= f32(1e-15)) & (a <= f32(1e15))), v


def _pretest(h, t2, x, y, dx, dy):
    """1 inlier, 0 not, 2 undecided: the kernel's operations in its order."""
    with np.errstate(all="ignore"):
        a0, a1 = h[0] * x, h[1] * y
        b0, b1 = h[3] * x, h[4] * y
        c0, c1 = h[6] * x, h[7] * y
        X, Y, Z = (a0 + a1) + h[2], (b0 + b1) + h[5], (c0 + c1) + h[8]
        MX = (np.abs(a0) + np.abs(a1)) + np.abs(h[2])
        MY = (np.abs(b0) + np.abs(b1)) + np.abs(h[5])
        MZ = (np.abs(c0) + np.abs(c1)) + np.abs(h[8])
        eZ = (f32(16) * U) * MZ + f32(1e-30)
        front = Z > eZ
        behind = (Z < -eZ) & (eZ < f32(3e38))
        ex, ey = X - dx * Z, Y - dy * Z
        ax = (f32(20) * U) * (MX + np.abs(dx) * MZ) + f32(1e-30)
        ay = (f32(20) * U) * (MY + np.abs(dy) * MZ) + f32(1e-30)
        lhs = ex * ex + ey * ey
        rhs = (t2 * Z) * Z
        el = ((f32(2) * np.abs(ex) * ax + ax * ax) + (f32(2) * np.abs(ey) * ay + ay * ay)) + \
             ((f32(8) * U) * lhs + f32(1e-36))
        er = t2 * (f32(2) * Z * eZ + eZ * eZ) + ((f32(16) * U) * rhs + f32(1e-36))
        fin = (np.abs(lhs) < f32(3e38)) & (rhs < f32(3e38)) & (el < f32(3e38)) & \
              (er < f32(3e38)) & (rhs >= f32(1e-30))
        d = np.full(x.shape, 2, dtype=np.int8)
        d[front & fin & ((lhs + el) + er < rhs)] = 1
        d[front & fin & (lhs > rhs + (el + er))] = 0
        d[~front] = 2
        d[behind] = 0
    return d


def _fp64(Hp, t2, x, y, dx, dy):
    X = Hp[0] * x + Hp[1] * y + Hp[2]
    Y = Hp[3] * x + Hp[4] * y + Hp[5]
    Z = Hp[6] * x + Hp[7] * y + Hp[8]
    ex, ey = X - dx * Z, Y - dy * Z
    return (Z > 0) & (ex * ex + ey * ey < t2 * Z * Z)


def test_pretest_never_contradicts_fp64():
    rng = np.random.default_rng(2024)
    undecided = {0: [0, 0], 1: [0, 0]}
    for trial in range(300):
        W = int(rng.choice([320, 1920, 3840, 16384]))
        Hh = W * 9 // 16
        A = np.eye(3) + rng.normal(0, [[0.05, 0.05, 20], [0.05, 0.05, 20], [1e-5, 1e-5, 0.05]])
        if trial % 7 == 0:
            A[2, :2] = rng.normal(0, 1e-3, 2)
        A /= A[2, 2]
        Hp = A.ravel()
        thr = float(rng.choice([0.5, 1.0, 3.0, rng.uniform(0.01, 20)]))
        t2 = thr * thr
        n = 512
        x = rng.uniform(0, W, n) + 0.5
        y = rng.uniform(0, Hh, n) + 0.5
        p = np.c_[x, y, np.ones(n)] @ A.T
        ang = rng.uniform(0, 2 * np.pi, n)
        near = np.arange(n) % 2 == 0
        r = np.where(near, thr * (1 + rng.integers(-4, 5, n) * 2.0 ** -52 * rng.integers(0, 2, n)),
                     rng.uniform(0, 3 * thr, n))
        r[np.arange(n) % 8 == 0] = thr
        with np.errstate(all="ignore"):
            dx = p[:, 0] / p[:, 2] + r * np.cos(ang)
            dy = p[:, 1] / p[:, 2] + r * np.sin(ang)
        back = p[:, 2] <= 0
        dx[back], dy[back] = rng.uniform(0, W, back.sum()), rng.uniform(0, Hh, back.sum())
        rd = np.arange(n) % 16 == 3
        dx[rd], dy[rd] = np.round(dx[rd]), np.round(dy[rd])
        want = _fp64(Hp, t2, x, y, dx, dy)
        okh = True
        h = []
        for v in Hp:
            o, fv = _in_range(np.array([v]))
            okh &= bool(o[0])
            h.append(fv[0])
        ot, t2f = _in_range(np.array([t2]))
        if not (okh and ot[0] and t2f[0] > 0):
            continue
        okp = np.ones(n, bool)
        vals = []
        for v in (x, y, dx, dy):
            o, fv = _in_range(v)
            okp &= o
            vals.append(fv)
        got = _pretest(h, t2f[0], *vals)
        got[~okp] = 2
        decided = got != 2
        assert np.array_equal(got[decided].astype(bool), want[decided]), trial
        for k, m in ((0, ~near), (1, near)):
            undecided[k][0] += int(m.sum())
            undecided[k][1] += int((got[m] == 2).sum())
    # uniformly spread residuals: almost all decided in FP32
    assert undecided[0][1] < 0.02 * undecided[0][0], undecided
    # residuals on the threshold: mostly left to FP64
    assert undecided[1][1] > 0.5 * undecided[1][0], undecided

"""ctypes shim around ``dmsgm_oracle.c`` -- the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library and never imports the product package.

Everything the method computes lives in ``dmsgm_oracle.c`` (one plain loop
nest per equation of arXiv:1702.05156 Sec. 2.2-2.4); this file only moves
NumPy arrays in and out.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmsgm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "homog_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Column indices of the per-block diagnostics (mirrors the enum in the C file).
DIAG = dict(M=0, NOSRC=1, WSUM=2, MU_A=3, VAR_A=4, XAGE_A=5, MU_C=6, VAR_C=7,
            XAGE_C=8, BRANCH=9, SWAP=10, MIN=11, MAX=12)


def build_oracle(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no -ffast-math, no FP contraction)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(p) for p in _SRCS))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
        # OpenMP over the step's block rows when the compiler has it
        r = subprocess.run(base + ["-fopenmp", "-o", tmp, *_SRCS, "-lm"], capture_output=True)
        if r.returncode != 0:
            subprocess.run(base + ["-o", tmp, *_SRCS, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_step.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                ctypes.c_int, ctypes.c_int] + [P] * 16
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_run.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                ctypes.c_int, ctypes.c_int] + [P] * 15
            lib.oracle_step_ex.restype = ctypes.c_int
            lib.oracle_step_ex.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                ctypes.c_int] * 3 + [P] * 16
            lib.oracle_run_ex.restype = ctypes.c_int
            lib.oracle_run_ex.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [
                ctypes.c_int] * 3 + [P] * 15
            lib.oracle_gauss_weights.restype = ctypes.c_int
            lib.oracle_gauss_weights.argtypes = [ctypes.c_int, ctypes.c_double, P]
            lib.oracle_prefilter.restype = ctypes.c_int
            lib.oracle_prefilter.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_int]
            lib.oracle_median3.restype = ctypes.c_int
            lib.oracle_median3.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
            lib.oracle_diag_stride.restype = ctypes.c_int
            assert lib.oracle_diag_stride() == len(DIAG)
            _lib = lib
    return _lib


@dataclass
class OracleState:
    """Block-grid state in FP64 / int32, each array of shape (Gy, Gx)."""
    muA: np.ndarray
    varA: np.ndarray
    ageA: np.ndarray
    muC: np.ndarray
    varC: np.ndarray
    ageC: np.ndarray

    @staticmethod
    def empty(gy: int, gx: int) -> "OracleState":
        z = lambda dt: np.zeros((gy, gx), dtype=dt)  # noqa: E731
        return OracleState(z(np.float64), z(np.float64), z(np.int32),
                           z(np.float64), z(np.float64), z(np.int32))


def state_from_arrays(muA, varA, ageA, muC, varC, ageC) -> OracleState:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    i = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
    return OracleState(f(muA), f(varA), i(ageA), f(muC), f(varC), i(ageC))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def oracle_step(frame: np.ndarray, H: np.ndarray, prev: OracleState | None, *,
                block: int, theta_s: float = 2.0, theta_d: float = 4.0,
                age_max: int = 30, diag: bool = False, mix_spread: bool = False):
    """One frame.  ``prev=None`` means the first frame of a stream.

    Returns ``(state, mask)`` or ``(state, mask, diag)``; ``mask`` is uint8
    (H, W) with 1 = foreground.
    """
    lib = _load()
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = frame.shape
    if block < 1:
        raise ValueError("block size must be >= 1")
    gy, gx = -(-h // block), -(-w // block)   # ceil: edge blocks are clipped (R11)
    Hm = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    first = prev is None
    if first:
        prev = OracleState.empty(gy, gx)
    nxt = OracleState.empty(gy, gx)
    mask = np.zeros((h, w), dtype=np.uint8)
    dg = np.zeros((gy, gx, len(DIAG)), dtype=np.float64) if diag else None
    rc = lib.oracle_step_ex(
        w, h, block, float(theta_s), float(theta_d), int(age_max), int(bool(mix_spread)),
        int(first),
        _ptr(frame), _ptr(Hm),
        _ptr(prev.muA), _ptr(prev.varA), _ptr(prev.ageA),
        _ptr(prev.muC), _ptr(prev.varC), _ptr(prev.ageC),
        _ptr(nxt.muA), _ptr(nxt.varA), _ptr(nxt.ageA),
        _ptr(nxt.muC), _ptr(nxt.varC), _ptr(nxt.ageC),
        _ptr(mask), _ptr(dg) if diag else None)
    if rc:
        raise ValueError(f"oracle_step failed ({rc})")
    return (nxt, mask, dg) if diag else (nxt, mask)


def oracle_run(frames: np.ndarray, Hs: np.ndarray, *, block: int,
               theta_s: float = 2.0, theta_d: float = 4.0, age_max: int = 30,
               mix_spread: bool = False):
    """T frames free-running from an empty state; returns (state, masks[T,H,W])."""
    lib = _load()
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    T, h, w = frames.shape
    gy, gx = -(-h // block), -(-w // block)
    Hs = np.ascontiguousarray(Hs, dtype=np.float64).reshape(T, 9)
    st = OracleState.empty(gy, gx)
    tmp = OracleState.empty(gy, gx)
    masks = np.zeros((T, h, w), dtype=np.uint8)
    rc = lib.oracle_run_ex(
        w, h, block, float(theta_s), float(theta_d), int(age_max), int(bool(mix_spread)), T,
        _ptr(frames), _ptr(Hs),
        _ptr(st.muA), _ptr(st.varA), _ptr(st.ageA),
        _ptr(st.muC), _ptr(st.varC), _ptr(st.ageC),
        _ptr(tmp.muA), _ptr(tmp.varA), _ptr(tmp.ageA),
        _ptr(tmp.muC), _ptr(tmp.varC), _ptr(tmp.ageC),
        _ptr(masks))
    if rc:
        raise ValueError(f"oracle_run failed ({rc})")
    return st, masks


def set_threads(n: int = 0) -> int:
    """Threads of the step's block-row loop (0: all available); returns the
    count in use (1 without OpenMP).  Results do not depend on it."""
    lib = _load()
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_threads.argtypes = [ctypes.c_int]
    return int(lib.oracle_threads(int(n)))


def gauss_weights(gauss_size: int, sigma: float) -> np.ndarray:
    """The quantised 1-D Gaussian weights (sum 256) of the preprocessing blur."""
    lib = _load()
    q = np.zeros(64, dtype=np.int32)
    if lib.oracle_gauss_weights(int(gauss_size), float(sigma), _ptr(q)):
        raise ValueError("invalid Gaussian size or sigma")
    return q[:gauss_size].copy()


def prefilter(frame: np.ndarray, *, gauss_size: int = 5, sigma: float = 1.0,
              median: bool = True) -> np.ndarray:
    """The preprocessing of the paper's Sec. 2.1: N x N Gaussian blur, then
    the 3 x 3 median, both clamp-to-border (readings P1-P4 in the C file)."""
    lib = _load()
    frame = np.ascontiguousarray(frame, dtype=np.uint8)
    h, w = frame.shape
    blur = np.empty_like(frame)
    if lib.oracle_prefilter(w, h, _ptr(frame), _ptr(blur), int(gauss_size), float(sigma),
                            int(bool(median))) < 0:
        raise ValueError("invalid preprocessing arguments")
    if not median:
        return blur
    out = np.empty_like(frame)
    if lib.oracle_median3(w, h, _ptr(blur), _ptr(out)):
        raise ValueError("invalid size")
    return out


# ----------------------------------------------------------------------------
# Motion-estimation front end (homog_oracle.c, readings M1-M8): corners,
# pyramidal tracking, RANSAC homography.

def _homog_sigs(lib):
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ho_tensor_map.restype = None
    lib.ho_tensor_map.argtypes = [P, I, I, I, P, P, P]
    lib.ho_score_map.restype = None
    lib.ho_score_map.argtypes = [P, I, I, I, P]
    lib.ho_corners.restype = I
    lib.ho_corners.argtypes = [P, I, I, I, D, D, I, P, P, P]
    lib.ho_pyr_down.restype = None
    lib.ho_pyr_down.argtypes = [P, I, I, P]
    lib.ho_track.restype = I
    lib.ho_track.argtypes = [P, P, I, I, I, I, I, D, D, P, I, P, P]
    lib.ho_splitmix64.restype = ctypes.c_uint64
    lib.ho_splitmix64.argtypes = [ctypes.c_uint64]
    lib.ho_sample4.restype = I
    lib.ho_sample4.argtypes = [ctypes.c_uint64, I, I, P]
    lib.ho_ransac.restype = I
    lib.ho_ransac.argtypes = [P, P, I, I, I, I, D, ctypes.c_uint64, P, P, P]
    lib.ho_hypothesis.restype = I
    lib.ho_hypothesis.argtypes = [P, P, I, I, I, ctypes.c_uint64, I, P]
    lib.ho_refit.restype = I
    lib.ho_refit.argtypes = [P, P, P, I, I, I, P]
    lib.ho_inliers.restype = I
    lib.ho_inliers.argtypes = [P, P, P, I, D, D, P, P]
    lib.ho_ransac_counts.restype = I
    lib.ho_ransac_counts.argtypes = [P, P, I, I, I, I, D, ctypes.c_uint64, D, P, P]
    lib.ho_estimate.restype = I
    lib.ho_estimate.argtypes = [P, P, I, I, I, D, D, I, I, I, I, D, D, I, D, ctypes.c_uint64,
                                P, P, P]
    return lib


_homog_ready = False


def _hlib():
    global _homog_ready
    lib = _load()
    if not _homog_ready:
        _homog_sigs(lib)
        _homog_ready = True
    return lib


# defaults: the paper's window (20 x 20, read as half-width 10) and 5 levels;
# the others are the usual defaults of the methods
HOMOG_DEFAULTS = dict(block_size=3, quality=0.01, min_distance=10.0, max_corners=500, levels=5,
                      win_half=10, max_iters=30, eps=0.01, min_eig=1e-3, ransac_iters=2000,
                      thresh=3.0, seed=0)


def tensor_map(img: np.ndarray, block_size: int = 3):
    """M1: the structure tensor (A, B, C) of every pixel, exact integers as
    float64 arrays."""
    lib = _hlib()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    A, B, C = (np.empty((h, w), dtype=np.float64) for _ in range(3))
    lib.ho_tensor_map(_ptr(img), w, h, int(block_size), _ptr(A), _ptr(B), _ptr(C))
    return A, B, C


def score_map(img: np.ndarray, block_size: int = 3) -> np.ndarray:
    """M1: the FP64 Shi-Tomasi score (smaller tensor eigenvalue) of every pixel."""
    lib = _hlib()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.empty((h, w), dtype=np.float64)
    lib.ho_score_map(_ptr(img), w, h, int(block_size), _ptr(out))
    return out


def corners(img: np.ndarray, block_size: int = 3, quality: float = 0.01,
            min_distance: float = 10.0, max_corners: int = 500):
    """M2-M4: corner pixel indices (m x 2, x then y), strongest first, their
    scores and the number of candidates before the cap."""
    lib = _hlib()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    xy = np.zeros((max_corners, 2), dtype=np.int32)
    sc = np.zeros(max_corners, dtype=np.float64)
    nc = ctypes.c_int(0)
    m = lib.ho_corners(_ptr(img), w, h, int(block_size), float(quality), float(min_distance),
                       int(max_corners), _ptr(xy), _ptr(sc), ctypes.byref(nc))
    if m < 0:
        raise ValueError("invalid corner arguments")
    return xy[:m].copy(), sc[:m].copy(), nc.value


def pyr_down(img: np.ndarray) -> np.ndarray:
    """M5: one pyramid step."""
    lib = _hlib()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2), dtype=np.uint8)
    lib.ho_pyr_down(_ptr(img), w, h, _ptr(out))
    return out


def track(prev: np.ndarray, cur: np.ndarray, pts: np.ndarray, levels: int = 5,
          win_half: int = 10, max_iters: int = 30, eps: float = 0.01, min_eig: float = 1e-3):
    """M6: pyramidal Lucas-Kanade of points (n x 2 pixel indices) from prev
    to cur: tracked positions (n x 2) and status (n, 1 = tracked)."""
    lib = _hlib()
    prev = np.ascontiguousarray(prev, dtype=np.uint8)
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    h, w = prev.shape
    out = np.empty_like(pts)
    st = np.zeros(len(pts), dtype=np.uint8)
    if lib.ho_track(_ptr(prev), _ptr(cur), w, h, int(levels), int(win_half), int(max_iters),
                    float(eps), float(min_eig), _ptr(pts), len(pts), _ptr(out), _ptr(st)):
        raise ValueError("invalid tracking arguments")
    return out, st


def splitmix64(z: int) -> int:
    return int(_hlib().ho_splitmix64(ctypes.c_uint64(z & (2 ** 64 - 1))))


def sample4(seed: int, m: int, n: int) -> np.ndarray | None:
    idx = np.zeros(4, dtype=np.int32)
    rc = _hlib().ho_sample4(ctypes.c_uint64(seed), int(m), int(n), _ptr(idx))
    return None if rc else idx


def ransac(src: np.ndarray, dst: np.ndarray, width: int, height: int, iters: int = 2000,
           thresh: float = 3.0, seed: int = 0):
    """M7-M8: the homography src -> dst (pixel coordinates): (H 3x3, inlier
    mask, inlier count, best hypothesis); H is None when no model exists."""
    lib = _hlib()
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    dst = np.ascontiguousarray(dst, dtype=np.float64).reshape(-1, 2)
    n = len(src)
    Hm = np.zeros(9)
    inl = np.zeros(max(n, 1), dtype=np.uint8)
    best = ctypes.c_int(-1)
    cnt = lib.ho_ransac(_ptr(src), _ptr(dst), n, int(width), int(height), int(iters),
                        float(thresh), ctypes.c_uint64(seed), _ptr(Hm), _ptr(inl),
                        ctypes.byref(best))
    if cnt < 0:
        return None, inl[:n], 0, -1
    return Hm.reshape(3, 3), inl[:n].astype(bool), cnt, best.value


def hypothesis(src: np.ndarray, dst: np.ndarray, width: int, height: int, seed: int, m: int):
    """M7: the model (3x3) of hypothesis m over the pairs src -> dst, or None."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    dst = np.ascontiguousarray(dst, dtype=np.float64).reshape(-1, 2)
    Hm = np.zeros(9)
    rc = _hlib().ho_hypothesis(_ptr(src), _ptr(dst), len(src), int(width), int(height),
                               ctypes.c_uint64(seed), int(m), _ptr(Hm))
    return None if rc else Hm.reshape(3, 3)


def inliers(Hm: np.ndarray, src: np.ndarray, dst: np.ndarray, thresh: float, band: float = 1e-6):
    """M7: the inlier mask of model Hm over the pairs src -> dst, and the mask
    of pairs whose squared reprojection error lies within band * thresh^2 of
    thresh^2."""
    Hm = np.ascontiguousarray(Hm, dtype=np.float64).reshape(9)
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    dst = np.ascontiguousarray(dst, dtype=np.float64).reshape(-1, 2)
    n = len(src)
    inl = np.zeros(max(n, 1), dtype=np.uint8)
    near = np.zeros(max(n, 1), dtype=np.uint8)
    _hlib().ho_inliers(_ptr(Hm), _ptr(src), _ptr(dst), n, float(thresh), float(band), _ptr(inl),
                       _ptr(near))
    return inl[:n].astype(bool), near[:n].astype(bool)


def refit(src: np.ndarray, dst: np.ndarray, inl: np.ndarray, width: int, height: int):
    """M8: the least-squares homography of the marked pairs, or None."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    dst = np.ascontiguousarray(dst, dtype=np.float64).reshape(-1, 2)
    m = np.ascontiguousarray(inl, dtype=np.uint8).reshape(-1)
    Hm = np.zeros(9)
    rc = _hlib().ho_refit(_ptr(src), _ptr(dst), _ptr(m), len(src), int(width), int(height),
                          _ptr(Hm))
    return None if rc else Hm.reshape(3, 3)


def ransac_counts(src: np.ndarray, dst: np.ndarray, width: int, height: int, iters: int = 2000,
                  thresh: float = 3.0, seed: int = 0, band: float = 1e-6):
    """M7: per hypothesis its inlier count (-1: no model) and the number of
    pairs whose squared reprojection error lies within band * thresh^2 of
    thresh^2."""
    src = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, 2)
    dst = np.ascontiguousarray(dst, dtype=np.float64).reshape(-1, 2)
    counts = np.zeros(iters, dtype=np.int32)
    near = np.zeros(iters, dtype=np.int32)
    if _hlib().ho_ransac_counts(_ptr(src), _ptr(dst), len(src), int(width), int(height),
                                int(iters), float(thresh), ctypes.c_uint64(seed), float(band),
                                _ptr(counts), _ptr(near)):
        raise ValueError("invalid RANSAC arguments")
    return counts, near


def estimate_homography(prev: np.ndarray, cur: np.ndarray, **kw):
    """The front end end to end: (H mapping cur pixel centres to prev ones,
    inlier count, corners, tracked points); H is None on failure."""
    p = dict(HOMOG_DEFAULTS)
    p.update(kw)
    lib = _hlib()
    prev = np.ascontiguousarray(prev, dtype=np.uint8)
    cur = np.ascontiguousarray(cur, dtype=np.uint8)
    h, w = prev.shape
    Hm = np.zeros(9)
    nc, nt = ctypes.c_int(0), ctypes.c_int(0)
    cnt = lib.ho_estimate(_ptr(prev), _ptr(cur), w, h, p["block_size"], p["quality"],
                          p["min_distance"], p["max_corners"], p["levels"], p["win_half"],
                          p["max_iters"], p["eps"], p["min_eig"], p["ransac_iters"], p["thresh"],
                          ctypes.c_uint64(p["seed"]), _ptr(Hm), ctypes.byref(nc), ctypes.byref(nt))
    if cnt < 0:
        return None, 0, nc.value, nt.value
    return Hm.reshape(3, 3), cnt, nc.value, nt.value

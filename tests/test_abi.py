"""CPU checks of the C ABI: the library builds, loads and exports every
symbol include/dmsgm.h declares; argument validation and size arithmetic
need no GPU (they return before any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import _lib
    return _lib


def _declared():
    """Every function any public header under include/ declares."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", h)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(dmsgm_[a-z_0-9]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(L):
    lib = L.load_library()
    declared = _declared()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(L.EXPORTS), declared ^ set(L.EXPORTS)


def test_version_and_sizes(L):
    assert "sm_103a" in L.dmsgm_version()
    # 1920x1080, B=4: 480x270 blocks; a buffer = mu and var arrays of N
    # (A, C) pairs and an age array of N byte pairs, each rounded up to 256
    # bytes; two buffers plus a 256-byte control block
    # plus one progress counter per 256 x 32 tile (8 x 34 tiles)
    N = 480 * 270
    r = lambda x: (x + 255) // 256 * 256  # noqa: E731
    flags = r(4 * 8 * 34)
    assert L.dmsgm_state_bytes(1920, 1080, 4, 0) == 256 + flags + 2 * (2 * r(8 * N) + r(2 * N))
    assert L.dmsgm_state_bytes(1920, 1080, 4, 1) == 256 + flags + 2 * (2 * r(4 * N) + r(2 * N))
    assert L.dmsgm_host_state_bytes(1920, 1080, 4, 0) == N * 18
    assert L.dmsgm_host_state_bytes(3840, 2160, 8, 1) == 480 * 270 * 10
    assert L.dmsgm_state_bytes(100, 100, 4, 0) == 0       # W % 16 != 0
    assert L.dmsgm_state_bytes(320, 240, 5, 0) == 0       # block 5
    assert L.dmsgm_state_bytes(320, 240, 32, 0) == 0      # block 32
    assert L.dmsgm_state_bytes(320, 240, 4, 7) == 0       # precision
    # a bottom block row cut by the frame edge counts as a block row:
    # 320 x 242 at B = 4 is 80 x 61 blocks; block 1 is one block per pixel
    assert L.dmsgm_host_state_bytes(320, 242, 4, 0) == 80 * 61 * 18
    assert L.dmsgm_host_state_bytes(320, 250, 16, 1) == 20 * 16 * 10
    assert L.dmsgm_host_state_bytes(64, 3, 1, 0) == 64 * 3 * 18
    assert L.dmsgm_host_state_bytes(64, 5, 2, 0) == 32 * 3 * 18


@pytest.mark.parametrize("args", [
    (100, 240, 4, 2.0, 4.0, 30),     # W % 16
    (320, 240, 5, 2.0, 4.0, 30),     # block
    (320, 240, 32, 2.0, 4.0, 30),    # block
    (320, 240, 0, 2.0, 4.0, 30),     # block
    (0, 240, 4, 2.0, 4.0, 30),
    (320, 240, 4, 0.0, 4.0, 30),     # theta_s
    (320, 240, 4, 2.0, float("nan"), 30),
    (320, 240, 4, 2.0, 4.0, 0),      # age_max
    (320, 240, 4, 2.0, 4.0, 256),
])
def test_create_rejects_invalid(L, args):
    lib = L.load_library()
    h = ctypes.c_void_p(123)
    rc = lib.dmsgm_create(*args, ctypes.byref(h))
    assert rc == L.DMSGM_ERR_INVALID_ARG
    assert h.value is None
    assert L.dmsgm_last_error()


def test_null_arguments(L):
    lib = L.load_library()
    assert lib.dmsgm_destroy(None) == 0
    assert lib.dmsgm_process(None, None, None, None, None) == L.DMSGM_ERR_INVALID_ARG
    assert lib.dmsgm_reset(None) == L.DMSGM_ERR_INVALID_ARG
    assert lib.dmsgm_process_batch(-1, None, None, None, None, None) == L.DMSGM_ERR_INVALID_ARG
    assert lib.dmsgm_process_batch(0, None, None, None, None, None) == 0
    assert lib.dmsgm_process_batch(L.DMSGM_MAX_BATCH + 1, None, None, None, None, None) == \
        L.DMSGM_ERR_INVALID_ARG


def test_package_import_does_not_need_library():
    import importlib
    import paper_1702_05156_gb300.synth as s  # noqa: F401
    importlib.import_module("paper_1702_05156_gb300")


def test_product_package_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_1702_05156_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), fn
                assert "dmsgm_oracle" not in src, fn


def test_homography_defaults_and_validation(L):
    """include/dmsgm_homog.h: the documented defaults, and every out-of-range
    parameter, frame size or NULL handle refused with DMSGM_ERR_INVALID_ARG
    before any device work (so on a machine without a GPU as well)."""
    p = L.dmsgm_homog_default_params()
    assert (p.block_size, p.max_corners, p.levels, p.win_half, p.max_iters, p.ransac_iters,
            p.seed) == (3, 500, 5, 10, 30, 2000, 0)
    assert (p.quality, p.min_distance, p.eps, p.min_eig, p.thresh) == (0.01, 10.0, 0.01, 1e-3, 3.0)
    bad = [dict(block_size=2), dict(block_size=9), dict(quality=0.0), dict(quality=float("nan")),
           dict(min_distance=-1.0), dict(min_distance=5000.0), dict(max_corners=0),
           dict(max_corners=4097), dict(levels=-1), dict(levels=9), dict(win_half=0),
           dict(win_half=16), dict(max_iters=0), dict(eps=-1.0), dict(min_eig=float("inf")),
           dict(ransac_iters=0), dict(ransac_iters=65537), dict(thresh=0.0)]
    for kw in bad:
        q = L.dmsgm_homog_default_params()
        for k, v in kw.items():
            setattr(q, k, v)
        with pytest.raises(L.DmsgmError) as e:
            L.dmsgm_homog_create(640, 480, q)
        assert e.value.code == L.DMSGM_ERR_INVALID_ARG, kw
    for W, H in ((8, 480), (640, 8), (632, 480), (16400, 480), (640, 16400)):
        with pytest.raises(L.DmsgmError) as e:
            L.dmsgm_homog_create(W, H)
        assert e.value.code == L.DMSGM_ERR_INVALID_ARG, (W, H)
    calls = [lambda: L.dmsgm_homog_estimate(None, 0, 0),
             lambda: L.dmsgm_homog_corners(None, 0, 8),
             lambda: L.dmsgm_homog_track(None, 0, 0, [[1.0, 2.0]]),
             lambda: L.dmsgm_homog_ransac(None, [[0.0, 0.0]], [[0.0, 0.0]])]
    for call in calls:
        with pytest.raises(L.DmsgmError) as e:
            call()
        assert e.value.code == L.DMSGM_ERR_INVALID_ARG
    L.dmsgm_homog_destroy(None)

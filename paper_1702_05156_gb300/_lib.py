"""ctypes binding of ``libdmsgm.so`` (include/dmsgm.h).

Argument marshalling only: every step of the motion-mask path runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If the
library is missing this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdmsgm.so")

DMSGM_OK = 0
DMSGM_ERR_INVALID_ARG = -1
DMSGM_ERR_OOM = -2
DMSGM_ERR_CUDA = -3
DMSGM_ERR_TIMEOUT = -4
DMSGM_ERR_DEVICE_STATUS = -5
DMSGM_ERR_UNSUPPORTED = -6
DMSGM_STATE_FP32 = 0
DMSGM_STATE_FP16 = 1
DMSGM_KERNEL_AUTO = 0
DMSGM_KERNEL_TILE = 1
DMSGM_MAX_BATCH = 256

# every symbol include/dmsgm.h declares
EXPORTS = ("dmsgm_state_bytes", "dmsgm_host_state_bytes", "dmsgm_create", "dmsgm_create_ex",
           "dmsgm_destroy", "dmsgm_process", "dmsgm_process_seq", "dmsgm_process_seq_noalloc",
           "dmsgm_process_host", "dmsgm_process_batch",
           "dmsgm_process_batch_ex", "dmsgm_process_batch_host",
           "dmsgm_get_state", "dmsgm_set_state", "dmsgm_reset", "dmsgm_get_info",
           "dmsgm_status", "dmsgm_selftest_wait", "dmsgm_prefilter", "dmsgm_last_error",
           "dmsgm_version", "dmsgm_fault_inject",
           # include/dmsgm_homog.h
           "dmsgm_homog_default_params", "dmsgm_homog_create", "dmsgm_homog_estimate",
           "dmsgm_homog_corners", "dmsgm_homog_track", "dmsgm_homog_ransac",
           "dmsgm_homog_destroy")


class dmsgm_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("state_mem", ctypes.c_void_p),
                ("state_bytes", ctypes.c_size_t), ("tile_rows", ctypes.c_int),
                ("use_pdl", ctypes.c_int), ("seq_tile_rows", ctypes.c_int),
                ("kernel", ctypes.c_int), ("mix_spread", ctypes.c_int),
                ("pre_gauss", ctypes.c_int), ("pre_sigma", ctypes.c_double),
                ("pre_median", ctypes.c_int), ("pre_separate", ctypes.c_int),
                ("checked", ctypes.c_int)]


class dmsgm_batch_opts(ctypes.Structure):
    _fields_ = [("reserved", ctypes.c_int), ("ctas", ctypes.c_int), ("use_pdl", ctypes.c_int),
                ("item_warps", ctypes.c_int)]


class dmsgm_info(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("block", ctypes.c_int),
                ("grid_w", ctypes.c_int), ("grid_h", ctypes.c_int), ("precision", ctypes.c_int),
                ("age_max", ctypes.c_int), ("theta_s", ctypes.c_float),
                ("theta_d", ctypes.c_float), ("initialized", ctypes.c_int),
                ("parity", ctypes.c_int), ("frames", ctypes.c_ulonglong),
                ("state_bytes", ctypes.c_size_t), ("host_state_bytes", ctypes.c_size_t),
                ("tile_rows", ctypes.c_int), ("device", ctypes.c_int), ("kernel", ctypes.c_int),
                ("last_kernel", ctypes.c_int), ("mix_spread", ctypes.c_int),
                ("pre_fused", ctypes.c_int), ("checked", ctypes.c_int)]


class DmsgmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dmsgm error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libdmsgm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is missing: build it with paper_1702_05156_gb300.build.build()")
        lib = ctypes.CDLL(p)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        F = ctypes.c_float
        sig = {
            "dmsgm_state_bytes": (S, [I, I, I, I]),
            "dmsgm_host_state_bytes": (S, [I, I, I, I]),
            "dmsgm_create": (I, [I, I, I, F, F, I, P]),
            "dmsgm_create_ex": (I, [I, I, I, F, F, I, P, P]),
            "dmsgm_destroy": (I, [P]),
            "dmsgm_process": (I, [P, P, P, P, P]),
            "dmsgm_process_seq": (I, [P, P, I, P, P, P]),
            "dmsgm_process_seq_noalloc": (I, [I, I, I, I, F, F, I, P, S, P, I, P, I, P, P, P]),
            "dmsgm_process_host": (I, [P, P, I, P, P, P]),
            "dmsgm_process_batch": (I, [I, P, P, P, P, P]),
            "dmsgm_process_batch_ex": (I, [I, P, P, P, P, P, P]),
            "dmsgm_process_batch_host": (I, [I, P, P, P, P, P, P, P, P, P, P]),
            "dmsgm_get_state": (I, [P, P, S]),
            "dmsgm_set_state": (I, [P, P, S]),
            "dmsgm_reset": (I, [P]),
            "dmsgm_get_info": (I, [P, P]),
            "dmsgm_status": (I, [P]),
            "dmsgm_selftest_wait": (I, [P, ctypes.c_ulonglong, P]),
            "dmsgm_prefilter": (I, [P, P, I, I, I, ctypes.c_double, I, P]),
            "dmsgm_last_error": (ctypes.c_char_p, []),
            "dmsgm_version": (ctypes.c_char_p, []),
            "dmsgm_fault_inject": (None, [ctypes.c_char_p]),
            "dmsgm_homog_default_params": (None, [P]),
            "dmsgm_homog_create": (I, [I, I, P, P]),
            "dmsgm_homog_estimate": (I, [P, P, P, P, P, P]),
            "dmsgm_homog_corners": (I, [P, P, P, P, P, P, P]),
            "dmsgm_homog_track": (I, [P, P, P, P, I, P, P, P]),
            "dmsgm_homog_ransac": (I, [P, P, P, I, P, P, P, P]),
            "dmsgm_homog_destroy": (I, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != DMSGM_OK:
        msg = load_library().dmsgm_last_error().decode(errors="replace")
        raise DmsgmError(rc, msg)


def _h9(H) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1))
    return a


# ----------------------------------------------------------- same-name functions
def dmsgm_state_bytes(width, height, block, precision=DMSGM_STATE_FP32) -> int:
    return load_library().dmsgm_state_bytes(width, height, block, precision)


def dmsgm_host_state_bytes(width, height, block, precision=DMSGM_STATE_FP32) -> int:
    return load_library().dmsgm_host_state_bytes(width, height, block, precision)


def dmsgm_create(width, height, block, theta_s, theta_d, age_max, opts: dmsgm_opts | None = None):
    lib = load_library()
    h = ctypes.c_void_p()
    if opts is None:
        _check(lib.dmsgm_create(width, height, block, theta_s, theta_d, age_max, ctypes.byref(h)))
    else:
        _check(lib.dmsgm_create_ex(width, height, block, theta_s, theta_d, age_max,
                                   ctypes.byref(opts), ctypes.byref(h)))
    return h


dmsgm_create_ex = dmsgm_create


def dmsgm_destroy(h):
    _check(load_library().dmsgm_destroy(h))


def dmsgm_process(h, frame_ptr: int, H, mask_ptr: int, stream: int = 0):
    Hm = _h9(H)
    _check(load_library().dmsgm_process(h, frame_ptr, Hm.ctypes.data, mask_ptr, stream))


def dmsgm_process_seq(h, frames_ptr: int, n: int, Hs, masks_ptr: int, stream: int = 0):
    Hm = _h9(Hs)
    assert Hm.size == 9 * n
    _check(load_library().dmsgm_process_seq(h, frames_ptr, n, Hm.ctypes.data, masks_ptr, stream))


def dmsgm_process_seq_noalloc(width, height, block, precision, theta_s, theta_d, age_max,
                              state_ptr: int, state_bytes: int, parity: ctypes.c_int, first: int,
                              frames_ptr: int, n: int, Hs, masks_ptr: int, stream: int = 0):
    """No-allocation multi-frame call; `parity` (a ctypes.c_int) is updated."""
    Hm = _h9(Hs)
    assert Hm.size == 9 * n
    _check(load_library().dmsgm_process_seq_noalloc(
        width, height, block, precision, theta_s, theta_d, age_max, state_ptr, state_bytes,
        ctypes.byref(parity), first, frames_ptr, n, Hm.ctypes.data, masks_ptr, stream))


def dmsgm_process_host(h, frames_ptr: int, n: int, Hs, masks_ptr: int, stream: int = 0):
    Hm = _h9(Hs)
    assert Hm.size == 9 * n
    _check(load_library().dmsgm_process_host(h, frames_ptr, n, Hm.ctypes.data, masks_ptr, stream))


def dmsgm_process_batch(handles, frame_ptrs, Hs, mask_ptrs, stream: int = 0,
                        opts: dmsgm_batch_opts | None = None):
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    fr = (ctypes.c_void_p * n)(*frame_ptrs)
    mk = (ctypes.c_void_p * n)(*mask_ptrs)
    Hm = _h9(Hs)
    assert Hm.size == 9 * n
    lib = load_library()
    if opts is None:
        _check(lib.dmsgm_process_batch(n, hs, fr, Hm.ctypes.data, mk, stream))
    else:
        _check(lib.dmsgm_process_batch_ex(n, hs, fr, Hm.ctypes.data, mk, ctypes.byref(opts), stream))


dmsgm_process_batch_ex = dmsgm_process_batch


def dmsgm_get_state(h, buf: np.ndarray):
    _check(load_library().dmsgm_get_state(h, buf.ctypes.data, buf.nbytes))


def dmsgm_set_state(h, buf: np.ndarray):
    _check(load_library().dmsgm_set_state(h, buf.ctypes.data, buf.nbytes))


def dmsgm_reset(h):
    _check(load_library().dmsgm_reset(h))


def dmsgm_get_info(h) -> dmsgm_info:
    info = dmsgm_info()
    _check(load_library().dmsgm_get_info(h, ctypes.byref(info)))
    return info


def dmsgm_status(h) -> int:
    return load_library().dmsgm_status(h)


def dmsgm_selftest_wait(h, timeout_ns: int, stream: int = 0):
    _check(load_library().dmsgm_selftest_wait(h, timeout_ns, stream))


def dmsgm_prefilter(in_dev: int, out_dev: int, width: int, height: int, gauss_size: int,
                    sigma: float, median: int, stream: int = 0):
    _check(load_library().dmsgm_prefilter(in_dev, out_dev, width, height, gauss_size, sigma,
                                          median, stream))


def dmsgm_last_error() -> str:
    return load_library().dmsgm_last_error().decode(errors="replace")


def dmsgm_version() -> str:
    return load_library().dmsgm_version().decode()


def dmsgm_fault_inject(spec: str | None):
    """Failure-handling tests only: "launch:n" / "alloc:n" (see dmsgm.h)."""
    load_library().dmsgm_fault_inject(spec.encode() if spec else None)


# ----------------------------------------------------------- include/dmsgm_homog.h
class dmsgm_homog_params(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int), ("quality", ctypes.c_double),
                ("min_distance", ctypes.c_double), ("max_corners", ctypes.c_int),
                ("levels", ctypes.c_int), ("win_half", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("eps", ctypes.c_double),
                ("min_eig", ctypes.c_double), ("ransac_iters", ctypes.c_int),
                ("thresh", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class dmsgm_homog_result(ctypes.Structure):
    _fields_ = [("corners", ctypes.c_int), ("candidates", ctypes.c_int),
                ("tracked", ctypes.c_int), ("inliers", ctypes.c_int), ("best", ctypes.c_int)]


def dmsgm_homog_default_params() -> dmsgm_homog_params:
    p = dmsgm_homog_params()
    load_library().dmsgm_homog_default_params(ctypes.byref(p))
    return p


def dmsgm_homog_create(width: int, height: int, params: dmsgm_homog_params | None = None):
    h = ctypes.c_void_p()
    _check(load_library().dmsgm_homog_create(width, height,
                                             ctypes.byref(params) if params is not None else None,
                                             ctypes.byref(h)))
    return h


def dmsgm_homog_destroy(h):
    _check(load_library().dmsgm_homog_destroy(h))


def dmsgm_homog_estimate(h, prev_dev: int, cur_dev: int, stream: int = 0):
    Hm = np.zeros(9)
    res = dmsgm_homog_result()
    _check(load_library().dmsgm_homog_estimate(h, prev_dev, cur_dev, Hm.ctypes.data,
                                               ctypes.byref(res), stream))
    return Hm.reshape(3, 3), res


def dmsgm_homog_corners(h, img_dev: int, max_corners: int, stream: int = 0):
    xy = np.zeros((max_corners, 2), dtype=np.int32)
    sc = np.zeros(max_corners, dtype=np.float32)
    n, nc = ctypes.c_int(0), ctypes.c_int(0)
    _check(load_library().dmsgm_homog_corners(h, img_dev, xy.ctypes.data, sc.ctypes.data,
                                              ctypes.byref(n), ctypes.byref(nc), stream))
    return xy[:n.value].copy(), sc[:n.value].copy(), nc.value


def dmsgm_homog_track(h, prev_dev: int, cur_dev: int, pts, stream: int = 0):
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.float32).reshape(-1, 2))
    n = len(pts)
    out = np.zeros((n, 2), dtype=np.float32)
    st = np.zeros(n, dtype=np.uint8)
    _check(load_library().dmsgm_homog_track(h, prev_dev, cur_dev, pts.ctypes.data, n,
                                            out.ctypes.data, st.ctypes.data, stream))
    return out, st


def dmsgm_homog_ransac(h, src, dst, stream: int = 0):
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 2))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.float64).reshape(-1, 2))
    n = len(src)
    Hm = np.zeros(9)
    inl = np.zeros(max(n, 1), dtype=np.uint8)
    res = dmsgm_homog_result()
    _check(load_library().dmsgm_homog_ransac(h, src.ctypes.data, dst.ctypes.data, n,
                                             Hm.ctypes.data, inl.ctypes.data, ctypes.byref(res),
                                             stream))
    return Hm.reshape(3, 3), inl[:n].astype(bool), res

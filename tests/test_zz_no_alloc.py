"""GPU: dmsgm_process_seq_noalloc, the entry point for callers that may not
allocate device memory (their memory belongs to their own allocator or a
fixed budget), gives the same masks and state as dmsgm_process_seq.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  It also passes alone in a fresh
process: it builds what it needs itself.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import spec_for, make_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import _lib, dmsgm
    return _lib, dmsgm


def _aligned(nbytes):
    raw = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    return raw, raw[off:off + nbytes]


def _state(mem, W, H, B, precision, which):
    """(A, C) means, variances and ages of buffer `which` of a state memory
    laid out as a handle's: control block, counter region, two buffers."""
    r = lambda x: (x + 255) // 256 * 256  # noqa: E731
    s = 2 if precision else 4
    N = (W // B) * (H // B)
    tiles = ((W + 255) // 256) * ((H + 8 * B - 1) // (8 * B))
    buf = 2 * r(N * 2 * s) + r(N * 2)
    base = 256 + r(4 * tiles) + which * buf
    host = mem.cpu().numpy()
    fdt = np.float16 if precision else np.float32
    mu = host[base:base + N * 2 * s].view(fdt).reshape(N, 2).astype(np.float64)
    var = host[base + r(N * 2 * s):base + r(N * 2 * s) + N * 2 * s].view(fdt).reshape(N, 2)
    age = host[base + 2 * r(N * 2 * s):base + 2 * r(N * 2 * s) + 2 * N].reshape(N, 2)
    return mu, var.astype(np.float64), age


@pytest.mark.parametrize("W,H,B,precision", [(640, 480, 4, 0), (1920, 1080, 8, 1)])
def test_noalloc_matches_process_seq_on_two_calls(lib, W, H, B, precision):
    _lib, dmsgm = lib
    T1, T2 = 9, 6
    frames, Hs = make_stream(spec_for(W, H, T1 + T2, seed=31), device="cuda")
    nbytes = _lib.dmsgm_state_bytes(W, H, B, precision)
    prec = "fp16" if precision else "fp32"

    # the existing entry point, state in caller memory so its bytes can be read
    _, ref_mem = _aligned(nbytes)
    ref = dmsgm.Dmsgm(W, H, B, precision=prec, state_mem=ref_mem)
    ref_m1 = ref.process_seq(frames[:T1], Hs[:T1])
    ref_m2 = ref.process_seq(frames[T1:], Hs[T1:])
    torch.cuda.synchronize()
    ref_parity = ref.info().parity

    # the no-allocation entry point, two calls in a row on the same state
    _, mem = _aligned(nbytes)
    parity = ctypes.c_int(0)
    m1 = dmsgm.new_mask(H, W, n=T1)
    m2 = dmsgm.new_mask(H, W, n=T2)
    stream = torch.cuda.current_stream().cuda_stream
    _lib.dmsgm_process_seq_noalloc(W, H, B, precision, 2.0, 4.0, 30, mem.data_ptr(), nbytes,
                                   parity, 1, frames[:T1].data_ptr(), T1, Hs[:T1],
                                   m1.data_ptr(), stream)
    _lib.dmsgm_process_seq_noalloc(W, H, B, precision, 2.0, 4.0, 30, mem.data_ptr(), nbytes,
                                   parity, 0, frames[T1:].data_ptr(), T2, Hs[T1:],
                                   m2.data_ptr(), stream)
    torch.cuda.synchronize()
    assert parity.value == ref_parity

    # the same kernel on the same inputs: identical masks and state
    assert torch.equal(m1, ref_m1) and torch.equal(m2, ref_m2)
    mu, var, age = _state(mem, W, H, B, precision, parity.value)
    rmu, rvar, rage = _state(ref_mem, W, H, B, precision, ref_parity)
    for a, b in ((mu, rmu), (var, rvar), (age, rage)):
        np.testing.assert_array_equal(a, b)
    # no device-side wait ran out
    assert int(mem[:4].view(torch.int32).item()) == 0
    ref.close()


def test_noalloc_rejects_bad_arguments(lib):
    _lib, _ = lib
    L = _lib.load_library()
    par = ctypes.c_int(0)
    # state memory too small / misaligned / bad parity: rejected before any device work
    rc = L.dmsgm_process_seq_noalloc(320, 240, 4, 0, 2.0, 4.0, 30, 256, 16, ctypes.byref(par), 1,
                                     None, 0, None, None, None)
    assert rc == _lib.DMSGM_ERR_INVALID_ARG
    par = ctypes.c_int(2)
    rc = L.dmsgm_process_seq_noalloc(320, 240, 4, 0, 2.0, 4.0, 30, 256, 1 << 30,
                                     ctypes.byref(par), 1, None, 0, None, None, None)
    assert rc == _lib.DMSGM_ERR_INVALID_ARG
    # a block other than 4 or 8, and a frame even a 256 x 256 tiling of which
    # needs more counters than the array's 4096: rejected before any CUDA call
    par = ctypes.c_int(0)
    need = _lib.dmsgm_state_bytes(320, 240, 16, 0)
    rc = L.dmsgm_process_seq_noalloc(320, 240, 16, 0, 2.0, 4.0, 30, 256, need,
                                     ctypes.byref(par), 1, None, 0, None, None, None)
    assert rc == _lib.DMSGM_ERR_UNSUPPORTED
    need = _lib.dmsgm_state_bytes(16384, 16640, 4, 0)
    rc = L.dmsgm_process_seq_noalloc(16384, 16640, 4, 0, 2.0, 4.0, 30, 256, need,
                                     ctypes.byref(par), 1, None, 0, None, None, None)
    assert rc == _lib.DMSGM_ERR_INVALID_ARG
    assert "4096" in _lib.dmsgm_last_error()

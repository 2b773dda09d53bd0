"""GPU: failure handling with host-injected faults (dmsgm_fault_inject).

No GPU fault, trap or hang is provoked: the injection makes the library
return DMSGM_ERR_CUDA (a frame launch) or DMSGM_ERR_OOM (a handle allocation)
before anything reaches the GPU.  The tests check that the failed call
leaves the handle's state untouched, that the next call works, and that the
serving loop fails only the requests of the failed step."""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream

pytestmark = pytest.mark.gpu


@pytest.fixture()
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import _lib, dmsgm
    yield dmsgm
    _lib.dmsgm_fault_inject(None)


def test_injected_launch_failure_leaves_the_state(lib):
    from paper_1702_05156_gb300 import _lib
    W, H, T = 320, 240, 6
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=8), device="cuda")
    ref = lib.Dmsgm(W, H, 4)
    for t in (0, 1, 3, 4, 5):                 # the run without frame 2
        ref.process(frames[t], Hs[t])
    m = lib.Dmsgm(W, H, 4)
    _lib.dmsgm_fault_inject("launch:3")       # the third launch from now fails
    for t in range(T):
        if t == 2:
            with pytest.raises(_lib.DmsgmError) as e:
                m.process(frames[t], Hs[t])
            assert e.value.code == _lib.DMSGM_ERR_CUDA and "injected" in str(e.value)
        else:
            m.process(frames[t], Hs[t])
    torch.cuda.synchronize()
    assert m.status() == 0
    a, b = m.get_state(), ref.get_state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_injected_allocation_failure(lib):
    from paper_1702_05156_gb300 import _lib
    _lib.dmsgm_fault_inject("alloc:1")
    with pytest.raises(_lib.DmsgmError) as e:
        lib.Dmsgm(320, 240, 4)
    assert e.value.code == _lib.DMSGM_ERR_OOM
    m = lib.Dmsgm(320, 240, 4)                # the next one is allocated
    assert m.info().state_bytes > 0


def test_serving_fails_only_the_failed_step(lib):
    from paper_1702_05156_gb300 import _lib
    from paper_1702_05156_gb300.serve import GpuEngine, Server
    W, H, T = 320, 240, 12
    frames, Hs = make_stream(StreamSpec(W, H, T, seed=9), device="cuda")
    host = frames.cpu().pin_memory()
    srv = Server(GpuEngine(), hbm_budget=1 << 30)
    srv.open_stream(0, W, H, 4)
    _lib.dmsgm_fault_inject("launch:4")       # the fourth batched step fails
    results, errors = {}, {}
    for t in range(T):
        f = srv.submit(0, host[t], Hs[t])
        e = f.exception(timeout=60)          # one frame per step
        if e is None:
            results[t] = f.result().clone()   # the mask lives in a reused host ring
        else:
            errors[t] = e
    assert list(errors) == [3]
    err = errors[3]
    assert isinstance(err, _lib.DmsgmError) and err.code == _lib.DMSGM_ERR_CUDA
    # the stream's later frames are processed: the step after the failure
    # continues the recurrence from the state before it
    ref = lib.Dmsgm(W, H, 4)
    for t in range(T):
        if t in errors:
            continue
        want = ref.process(frames[t], Hs[t]).cpu()
        assert torch.equal(results[t], want), t
    srv.close_stream(0)
    srv.shutdown()

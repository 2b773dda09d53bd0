"""Host logic of the serving loop, on CPU with a fake engine (no GPU)."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.serve import Server


class FakeEngine:
    """Records launches; 'computes' a step after a short delay."""

    def __init__(self, delay=0.002, per_px=1):
        self.delay = delay
        self.per_px = per_px
        self.open_ids = set()
        self.launches = []
        self.lock = threading.Lock()
        self.max_open_bytes = 0
        self.bytes = {}

    def stream_bytes(self, W, H, block):
        return W * H * self.per_px

    def open(self, sid, W, H, block):
        with self.lock:
            assert sid not in self.open_ids
            self.open_ids.add(sid)
            self.bytes[sid] = W * H * self.per_px
            self.max_open_bytes = max(self.max_open_bytes, sum(self.bytes.values()))

    def close(self, sid):
        with self.lock:
            self.open_ids.remove(sid)
            del self.bytes[sid]

    def launch(self, reqs):
        with self.lock:
            for r in reqs:
                assert r.sid in self.open_ids, "launch on a stream that is not admitted"
            self.launches.append([(r.sid, int(r.frame[0, 0])) for r in reqs])
            for r in reqs:
                r.mask_host = (r.sid, int(r.frame[0, 0]))
        return time.perf_counter() + self.delay

    @staticmethod
    def wait(t):
        d = t - time.perf_counter()
        if d > 0:
            time.sleep(d)


def _frame(k):
    return torch.full((4, 4), k % 256, dtype=torch.uint8)


def test_every_frame_completes_in_order_one_per_stream_per_step():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget=10_000)
    futs = {}
    for sid in range(5):
        srv.open_stream(sid, 16, 16)
    for k in range(20):
        for sid in range(5):
            futs[(sid, k)] = srv.submit(sid, _frame(k), np.eye(3))
    for sid in range(5):
        srv.close_stream(sid)
    for (sid, k), f in futs.items():
        assert f.result(timeout=10) == (sid, k)
    srv.shutdown()
    seen = {}
    for step in eng.launches:
        sids = [s for s, _ in step]
        assert len(sids) == len(set(sids)), "a stream appears twice in one step"
        for sid, k in step:
            assert seen.get(sid, -1) == k - 1, "frames of a stream out of order"
            seen[sid] = k
    assert all(v == 19 for v in seen.values())
    st = srv.stats()
    assert st["frames"] == 100 and st["p99_ms"] >= st["p50_ms"] > 0
    assert eng.open_ids == set()


def test_admission_respects_the_memory_budget():
    """Budget for 2 streams of 256 bytes; 6 streams arrive: at most 2 are
    resident at any time, the rest wait for memory and still finish."""
    eng = FakeEngine(delay=0.003)
    srv = Server(eng, hbm_budget=2 * 256)
    futs = []
    for sid in range(6):
        srv.open_stream(sid, 16, 16)
        for k in range(4):
            futs.append(srv.submit(sid, _frame(k), np.eye(3)))
        srv.close_stream(sid)
    for f in futs:
        f.result(timeout=10)
    srv.shutdown()
    assert eng.max_open_bytes <= 512
    assert len(srv.admit_log) == 6
    assert srv.used == 0


def test_frames_arriving_during_a_step_join_the_next():
    """Continuous batching: a stream opened while others are in flight is
    picked up by a later step without waiting for the others to finish."""
    eng = FakeEngine(delay=0.02)
    srv = Server(eng, hbm_budget=10_000)
    srv.open_stream(0, 8, 8)
    f0 = [srv.submit(0, _frame(k), np.eye(3)) for k in range(10)]
    time.sleep(0.03)
    srv.open_stream(1, 8, 8)
    f1 = srv.submit(1, _frame(0), np.eye(3))
    f1.result(timeout=10)
    assert not f0[-1].done(), "the late stream should not wait behind the whole queue"
    for f in f0:
        f.result(timeout=10)
    srv.close_stream(0)
    srv.close_stream(1)
    srv.shutdown()
    mixed = [s for s in eng.launches if {x for x, _ in s} == {0, 1}]
    assert mixed, "the two streams never shared a step"


def test_rejects_oversized_and_unknown_streams():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget=100)
    with pytest.raises(ValueError):
        srv.open_stream(0, 16, 16)          # 256 bytes > 100
    with pytest.raises(ValueError):
        srv.submit(7, _frame(0), np.eye(3))
    srv.shutdown()


class FailingEngine(FakeEngine):
    """Fails the launch of every step that contains stream 1's third frame."""

    def launch(self, reqs):
        if any(r.sid == 1 and int(r.frame[0, 0]) == 2 for r in reqs):
            raise RuntimeError("injected launch failure")
        return super().launch(reqs)


def test_a_failed_step_fails_its_requests_and_the_loop_goes_on():
    """Failure injected on the host: the step's futures carry the error,
    other steps still complete, and the server shuts down cleanly."""
    eng = FailingEngine()
    srv = Server(eng, hbm_budget=10_000)
    futs = {}
    for sid in (0, 1):
        srv.open_stream(sid, 8, 8)
    for k in range(6):
        for sid in (0, 1):
            futs[(sid, k)] = srv.submit(sid, _frame(k), np.eye(3))
    for sid in (0, 1):
        srv.close_stream(sid)
    failed = []
    for key, f in futs.items():
        try:
            f.result(timeout=10)
        except RuntimeError as e:
            assert "injected" in str(e)
            failed.append(key)
    srv.shutdown()
    assert (1, 2) in failed
    assert len(failed) < len(futs)
    assert srv.stats()["failed"] == len(failed)

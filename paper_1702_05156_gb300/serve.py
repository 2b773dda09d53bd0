"""Continuous-batching server of DMSGM video streams on one GPU.

Requests are frames of independent streams.  A scheduler thread admits
streams while their device memory (model state plus frame / mask slots)
fits a fixed HBM budget, keeps admitted streams' state resident, and at
every step gathers at most one pending frame per stream (frames of one
stream form a recurrence) into ONE batched kernel launch.  Frames that
arrive while a step runs join the next step.  The host->device copies of
step k+1 overlap the kernel of step k (separate copy stream, double-buffered
per-stream slots); a completer thread resolves each request's future when
its mask is back in host memory and records its latency.

The engine (device memory, copies, kernel launches) is behind a small
interface; GpuEngine is the only one in the product.  It reserves the HBM
budget in the caching allocator and loads the batched kernel's variants at
start, and recycles a closed stream's device slot for the next stream of the
same shape, so admitting a stream allocates nothing once warm.

Latency: Python's cyclic garbage collector stops every thread while it scans
the live objects (requests, futures); with ~10^5 of them alive its pauses set
the tail.  A latency-sensitive application calls gc.freeze() after its setup
and keeps the collector off while serving (measured: p99 0.42 ms instead of
11-14 ms for 256 streams at 30 fps).
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from .dmsgm import Dmsgm, mask_words


@dataclass
class Request:
    sid: int
    frame: torch.Tensor            # uint8 (H, W), host (pinned for overlap)
    H: np.ndarray                  # (3, 3) current -> previous
    t_submit: float
    future: Future = field(default_factory=Future)
    t_done: float = 0.0


@dataclass
class StreamInfo:
    sid: int
    W: int
    H: int
    block: int
    nbytes: int
    queue: collections.deque = field(default_factory=collections.deque)
    closing: bool = False
    in_flight: int = 0
    frames_done: int = 0


class GpuEngine:
    """Device side of the server: per-stream handles and double-buffered
    frame / mask slots, one copy stream and one compute stream."""

    POOL = 16   # released device slots kept per (W, H, block) for the next stream

    def __init__(self, precision: str = "fp32", device: int = 0, use_pdl: bool = True):
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.h2d = torch.cuda.Stream(device=self.device)
        self.compute = torch.cuda.Stream(device=self.device)
        self.d2h = torch.cuda.Stream(device=self.device)
        self.slots = {}
        self.free = collections.defaultdict(list)
        self.use_pdl = use_pdl

    def stream_bytes(self, W, H, block) -> int:
        prec = _lib.DMSGM_STATE_FP16 if self.precision == "fp16" else _lib.DMSGM_STATE_FP32
        return (_lib.dmsgm_state_bytes(W, H, block, prec) + 2 * W * H
                + 2 * H * mask_words(W) * 4)

    def warm(self):
        """Run one batched step of 1, 17 and 65 tiny streams, so that the
        batched kernel's variants (descriptor capacities 16, 64, 256) are
        loaded before the first real request rather than during it."""
        with torch.cuda.device(self.device):
            W, H, n = 32, 16, 65
            ms = [Dmsgm(W, H, 4, precision=self.precision) for _ in range(n)]
            fr = torch.zeros((n, H, W), dtype=torch.uint8, pin_memory=True)
            fd = torch.zeros((n, H, W), dtype=torch.uint8, device=self.device)
            md = torch.zeros((n, H, mask_words(W)), dtype=torch.int32, device=self.device)
            mh = torch.zeros((n, H, mask_words(W)), dtype=torch.int32, pin_memory=True)
            for k in (1, 17, 65):
                ptr = lambda t: np.array([t[i].data_ptr() for i in range(k)], np.uint64)  # noqa: E731
                hs = np.array([m.handle.value for m in ms[:k]], np.uint64)
                Hs = np.tile(np.eye(3).reshape(1, 9), (k, 1))
                opts = _lib.dmsgm_batch_opts(0, 0, 1 if self.use_pdl else 0)
                a = [hs, ptr(fr), ptr(fd), Hs, ptr(md), ptr(mh)]
                _lib._check(_lib.load_library().dmsgm_process_batch_host(
                    k, a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data, a[3].ctypes.data,
                    a[4].ctypes.data, a[5].ctypes.data, _lib.ctypes.byref(opts),
                    self.h2d.cuda_stream, self.compute.cuda_stream, self.d2h.cuda_stream))
            torch.cuda.synchronize(self.device)
            for m in ms:
                m.close()

    def reserve(self, nbytes: int):
        """Warm the caching allocator with nbytes of device memory, so that
        admitting streams later carves their memory from it instead of
        calling cudaMalloc (which can stall the device) mid-serving."""
        with torch.cuda.device(self.device):
            blk = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            del blk

    def open(self, sid, W, H, block):
        pool = self.free.get((W, H, block))
        if pool:
            # a released stream's slot: device memory, handle and pinned ring
            # are reused, nothing is allocated
            sl = pool.pop()
            sl["m"].reset()
            sl["n"] = 0
            self.slots[sid] = sl
            return
        # state memory from the caching allocator: admitting or retiring a
        # stream then never synchronises the device
        prec = _lib.DMSGM_STATE_FP16 if self.precision == "fp16" else _lib.DMSGM_STATE_FP32
        nbytes = _lib.dmsgm_state_bytes(W, H, block, prec)
        with torch.cuda.device(self.device):
            raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-raw.data_ptr()) % 256
            m = Dmsgm(W, H, block, precision=self.precision, state_mem=raw[off:off + nbytes],
                      use_pdl=self.use_pdl)
            frames = torch.empty((2, H, W), dtype=torch.uint8, device=self.device)
            masks = torch.empty((2, H, mask_words(W)), dtype=torch.int32, device=self.device)
        # pinned result ring: a request's mask stays valid until RING more
        # frames of its stream -- or, once the stream is closed, of the next
        # stream that takes over its slot -- have completed
        ring = torch.empty((self.RING, H, mask_words(W)), dtype=torch.int32, pin_memory=True)
        self.slots[sid] = {"m": m, "frames": frames, "masks": masks, "n": 0, "raw": raw,
                           "ring": ring, "handle": m.handle.value, "key": (W, H, block),
                           "fptr": [frames[0].data_ptr(), frames[1].data_ptr()],
                           "mptr": [masks[0].data_ptr(), masks[1].data_ptr()]}

    RING = 8

    def close(self, sid):
        # called once every step of the stream has completed: keep the
        # device slot for the next stream of the same shape
        sl = self.slots.pop(sid)
        pool = self.free[sl["key"]]
        if len(pool) < self.POOL:
            pool.append(sl)
        else:
            sl["m"].close()
            sl.clear()

    def launch(self, reqs):
        """One native call enqueues the frames' host->device copies (h2d
        stream), one batched step (compute stream) and the masks' copies
        back (d2h stream); returns an event that completes with the step.
        The server keeps at most two steps in flight, so a stream's device
        slot is never reused before the step that last used it completed."""
        with torch.cuda.nvtx.range("serve_step"):
            return self._launch(reqs)

    def _launch(self, reqs):
        n = len(reqs)
        for lo in range(0, n, _lib.DMSGM_MAX_BATCH):
            part = reqs[lo:lo + _lib.DMSGM_MAX_BATCH]
            k = len(part)
            hs = np.empty(k, np.uint64)
            fh = np.empty(k, np.uint64)
            fd = np.empty(k, np.uint64)
            md = np.empty(k, np.uint64)
            mh = np.empty(k, np.uint64)
            Hs = np.empty((k, 9), np.float64)
            for i, r in enumerate(part):
                sl = self.slots[r.sid]
                j = sl["n"]
                sl["n"] = j + 1
                hs[i] = sl["handle"]
                fh[i] = r.frame.data_ptr()
                fd[i] = sl["fptr"][j & 1]
                md[i] = sl["mptr"][j & 1]
                r.mask_host = sl["ring"][j % self.RING]
                mh[i] = r.mask_host.data_ptr()
                Hs[i] = r.H.reshape(9)
            opts = _lib.dmsgm_batch_opts(0, 0, 1 if self.use_pdl else 0)
            rc = _lib.load_library().dmsgm_process_batch_host(
                k, hs.ctypes.data, fh.ctypes.data, fd.ctypes.data, Hs.ctypes.data,
                md.ctypes.data, mh.ctypes.data, _lib.ctypes.byref(opts), self.h2d.cuda_stream,
                self.compute.cuda_stream, self.d2h.cuda_stream)
            _lib._check(rc)
        ev_done = torch.cuda.Event()
        ev_done.record(self.d2h)
        return ev_done

    @staticmethod
    def wait(ev):
        ev.synchronize()


class PlainEngine(GpuEngine):
    """The plain per-stream path behind the same server, for comparison: no
    batching -- every request is its own host->device copy, one
    dmsgm_process launch and the mask's copy back, on one of `lanes` CUDA
    streams (a stream's frames always on the same one, which keeps its
    recurrence in order).  Admission, slots and pinned rings as GpuEngine."""

    def __init__(self, precision: str = "fp32", device: int = 0, use_pdl: bool = True,
                 lanes: int = 8):
        super().__init__(precision, device, use_pdl)
        self.lanes = [torch.cuda.Stream(device=self.device) for _ in range(lanes)]

    def warm(self):
        pass

    def _launch(self, reqs):
        used = {}
        for r in reqs:
            sl = self.slots[r.sid]
            j = sl["n"]
            sl["n"] = j + 1
            ls = self.lanes[r.sid % len(self.lanes)]
            used[id(ls)] = ls
            r.mask_host = sl["ring"][j % self.RING]
            dev_frame = sl["frames"][j & 1]
            dev_mask = sl["masks"][j & 1]
            with torch.cuda.stream(ls):
                dev_frame.copy_(r.frame, non_blocking=True)
                _lib.dmsgm_process(sl["m"].handle, dev_frame.data_ptr(), r.H, dev_mask.data_ptr(),
                                   ls.cuda_stream)
                r.mask_host.copy_(dev_mask, non_blocking=True)
        evs = []
        for ls in used.values():
            ev = torch.cuda.Event()
            ev.record(ls)
            evs.append(ev)
        return evs

    @staticmethod
    def wait(evs):
        for ev in evs:
            ev.synchronize()


class Server:
    """Admission by memory budget + continuous batching over an engine."""

    def __init__(self, engine, hbm_budget: int, max_batch: int = 1 << 30,
                 max_in_flight_steps: int = 2):
        self.engine = engine
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.max_steps = max_in_flight_steps
        self.used = 0
        self.waiting = collections.deque()       # streams not admitted yet
        self.active = collections.OrderedDict()  # sid -> StreamInfo
        self.known = {}
        self.cv = threading.Condition()
        self.done_q = collections.deque()
        self.in_flight_steps = 0
        self.running = True
        self.steps = 0
        self.step_sizes = []
        self.latencies = []
        self.pixels = 0
        self.failed = 0
        self.admit_log = []      # (time, sid) of each admission
        self.release_log = []    # (time, sid) of each release
        if hasattr(engine, "reserve"):
            engine.reserve(self.budget)
        if hasattr(engine, "warm"):
            engine.warm()
        self._sched = threading.Thread(target=self._schedule_loop, daemon=True)
        self._comp = threading.Thread(target=self._complete_loop, daemon=True)
        self._sched.start()
        self._comp.start()

    # ------------------------------------------------------------- client API
    def open_stream(self, sid: int, W: int, H: int, block: int = 4):
        with self.cv:
            if sid in self.known:
                raise ValueError(f"stream {sid} already open")
            info = StreamInfo(sid, W, H, block, self.engine.stream_bytes(W, H, block))
            if info.nbytes > self.budget:
                raise ValueError(f"stream {sid} needs {info.nbytes} bytes, budget {self.budget}")
            self.known[sid] = info
            self.waiting.append(info)
            self.cv.notify_all()

    def submit(self, sid: int, frame: torch.Tensor, H) -> Future:
        req = Request(sid, frame, np.asarray(H, dtype=np.float64), time.perf_counter())
        with self.cv:
            info = self.known.get(sid)
            if info is None or info.closing:
                raise ValueError(f"stream {sid} is not open")
            info.queue.append(req)
            self.cv.notify_all()
        return req.future

    def close_stream(self, sid: int):
        """No more frames; the stream's memory is released once its queued
        frames are done."""
        with self.cv:
            self.known[sid].closing = True
            self.cv.notify_all()

    def shutdown(self, timeout: float = 30.0):
        t_end = time.perf_counter() + timeout
        with self.cv:
            while (any(s.queue or s.in_flight for s in self.known.values())
                   and time.perf_counter() < t_end):
                self.cv.wait(0.05)
            self.running = False
            self.cv.notify_all()
        self._sched.join(timeout)
        self._comp.join(timeout)
        with self.cv:   # retire whatever is still resident
            for info in list(self.active.values()):
                if not info.in_flight:
                    self._release(info)

    def stats(self) -> dict:
        lat = np.array(self.latencies) * 1e3 if self.latencies else np.zeros(1)
        return {"frames": len(self.latencies), "steps": self.steps, "failed": self.failed,
                "mean_batch": float(np.mean(self.step_sizes)) if self.step_sizes else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "pixels": self.pixels}

    # ------------------------------------------------------------- internals
    def _reserve(self):
        """Streams that now fit the budget, with their memory accounted; the
        caller opens them outside the lock."""
        out = []
        while self.waiting:
            info = self.waiting[0]
            if self.used + info.nbytes > self.budget:
                break
            self.waiting.popleft()
            self.used += info.nbytes
            out.append(info)
        return out

    def _release(self, info):
        self.release_log.append((time.perf_counter(), info.sid))
        self.engine.close(info.sid)
        self.used -= info.nbytes
        del self.active[info.sid]
        del self.known[info.sid]

    def _schedule_loop(self):
        while True:
            opening = []
            with self.cv:
                while self.running:
                    for info in list(self.active.values()):
                        if info.closing and not info.queue and not info.in_flight:
                            self._release(info)
                    opening = self._reserve()
                    if opening:
                        break
                    # a stream may sit in two consecutive steps: the device runs
                    # steps in order, so its recurrence is kept
                    ready = [s for s in self.active.values()
                             if s.queue and s.in_flight < self.max_steps]
                    if ready and self.in_flight_steps < self.max_steps:
                        break
                    self.cv.wait(0.002)
                if not self.running and not opening:
                    return
            if opening:
                # admission (device memory, a handle, a pinned ring) runs
                # without the lock: submissions and completions go on
                for info in opening:
                    self.engine.open(info.sid, info.W, info.H, info.block)
                with self.cv:
                    for info in opening:
                        self.active[info.sid] = info
                        self.admit_log.append((time.perf_counter(), info.sid))
                    self.cv.notify_all()
                continue
            with self.cv:
                batch = []
                for s in ready[: self.max_batch]:
                    batch.append(s.queue.popleft())
                    s.in_flight += 1
                self.in_flight_steps += 1
            try:
                ev = self.engine.launch(batch)
            except Exception as e:   # the step failed: its requests fail, the loop goes on
                with self.cv:
                    for r in batch:
                        info = self.active.get(r.sid)
                        if info is not None:
                            info.in_flight -= 1
                    self.in_flight_steps -= 1
                    self.failed += len(batch)
                    self.cv.notify_all()
                for r in batch:
                    r.future.set_exception(e)
                continue
            with self.cv:
                self.steps += 1
                self.step_sizes.append(len(batch))
                self.done_q.append((ev, batch))
                self.cv.notify_all()

    def _complete_loop(self):
        while True:
            with self.cv:
                while self.running and not self.done_q:
                    self.cv.wait(0.01)
                if not self.done_q:
                    return
                ev, batch = self.done_q.popleft()
            err = None
            try:
                self.engine.wait(ev)
            except Exception as e:
                err = e
            t = time.perf_counter()
            with self.cv:
                for r in batch:
                    r.t_done = t
                    self.latencies.append(t - r.t_submit)
                    info = self.active.get(r.sid)
                    if info is not None:
                        info.in_flight -= 1
                        info.frames_done += 1
                        self.pixels += info.W * info.H
                self.in_flight_steps -= 1
                self.cv.notify_all()
            for r in batch:
                if err is None:
                    r.future.set_result(getattr(r, "mask_host", None))
                else:
                    r.future.set_exception(err)


def simulate(server: Server, n_streams: int, rate: float, fps: float, dur_lo: float,
             dur_hi: float, resolutions, pools, seed: int = 7, block: int = 4):
    """Drive `server` with `n_streams` streams arriving as a Poisson process
    (rate per second), each submitting frames at `fps` for U(dur_lo, dur_hi)
    seconds of wall time.  pools[(W, H)] = (frames pinned (K, H, W), Hs (K,3,3)):
    a stream cycles through its resolution's pool from a random offset.
    Returns (wall seconds, futures)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    events = []   # (time, kind, sid, payload)
    for sid in range(n_streams):
        t += rng.exponential(1.0 / rate)
        W, H = resolutions[rng.integers(len(resolutions))]
        dur = rng.uniform(dur_lo, dur_hi)
        nfr = max(1, int(dur * fps))
        off = int(rng.integers(len(pools[(W, H)][0])))
        events.append((t, 0, sid, (W, H, nfr, off)))
        for k in range(nfr):
            events.append((t + k / fps, 1, sid, k))
        events.append((t + (nfr - 1) / fps + 1e-6, 2, sid, None))
    events.sort(key=lambda e: (e[0], e[1]))
    meta = {}
    futures = []
    t0 = time.perf_counter()
    for (te, kind, sid, pl) in events:
        now = time.perf_counter() - t0
        if te > now:
            time.sleep(te - now)
        if kind == 0:
            W, H, nfr, off = pl
            meta[sid] = (W, H, off)
            server.open_stream(sid, W, H, block)
        elif kind == 1:
            W, H, off = meta[sid]
            fr, Hs = pools[(W, H)]
            i = (off + pl) % len(fr)
            futures.append(server.submit(sid, fr[i], np.eye(3) if pl == 0 else Hs[i]))
        else:
            server.close_stream(sid)
    for f in futures:
        f.result(timeout=120)
    wall = time.perf_counter() - t0
    return wall, futures

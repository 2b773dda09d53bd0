"""Many streams per launch: a runner that captures frame-steps of a set of
streams into one CUDA graph, and an autotuner for the batched kernel's
launch shape.

A "step" advances every stream of the batch by one frame in ONE launch of
the batched kernel (dmsgm_process_batch_ex), or in one launch per lane when
the streams are split over several CUDA streams (lanes); a captured graph
replays `steps` consecutive steps.  The plain path (one launch of the
single-stream kernel per stream per step, also captured) is kept alongside
for comparison.  All arithmetic happens in libdmsgm.so.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from .dmsgm import Dmsgm, new_mask

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


@dataclass(frozen=True)
class LaunchShape:
    ctas: int = 0          # CTAs (0 or >= work items: one item per CTA; fewer: persistent)
    use_pdl: bool = True
    lanes: int = 1         # CUDA streams the batch is split over, one launch each per step
    item_warps: int = 0    # warps (strip rows) per work item: 4 or 8 (0: 4)

    def opts(self) -> _lib.dmsgm_batch_opts:
        return _lib.dmsgm_batch_opts(0, self.ctas, 1 if self.use_pdl else 0, self.item_warps)


def _ptr_arrays(models, frames_t, masks_t):
    n = len(models)
    hs = (_lib.ctypes.c_void_p * n)(*[m.handle.value for m in models])
    fr = (_lib.ctypes.c_void_p * n)(*[f.data_ptr() for f in frames_t])
    mk = (_lib.ctypes.c_void_p * n)(*[k.data_ptr() for k in masks_t])
    return hs, fr, mk


class BatchRunner:
    """Streams of mixed size / block / precision stepped together.

    frames[i]: uint8 (T, H_i, W_i) device tensor of stream i; Hs[i]: (T, 3, 3)
    homographies.  Masks are written to per-stream device tensors
    (T, H_i, ceil(W_i/32)).
    """

    def __init__(self, specs, frames, Hs, precision="fp32", device="cuda"):
        self.specs = specs           # [(W, H, B)]
        self.frames = frames
        self.Hs = [np.ascontiguousarray(h, dtype=np.float64) for h in Hs]
        self.T = min(f.shape[0] for f in frames)
        self.precision = precision
        # programmatic dependent launch for the plain path's single-stream steps
        self.models = [Dmsgm(w, h, b, precision=precision, use_pdl=True) for (w, h, b) in specs]
        self.masks = [new_mask(h, w, device, n=self.T) for (w, h, b) in specs]
        self.pixels_per_step = sum(w * h for (w, h, b) in specs)
        self._H_steps = [np.stack([self.Hs[i][t] for i in range(len(specs))]).reshape(-1)
                         for t in range(self.T)]

    # -------------------------------------------------------------- launches
    def lane_sets(self, lanes: int) -> list[list[int]]:
        """The streams split over `lanes` launches with about equal pixels:
        largest stream first, each onto the lane with the fewest pixels."""
        load = [0] * lanes
        sets = [[] for _ in range(lanes)]
        for i in sorted(range(len(self.specs)), key=lambda i: -self.specs[i][0] * self.specs[i][1]):
            j = load.index(min(load))
            sets[j].append(i)
            load[j] += self.specs[i][0] * self.specs[i][1]
        return [sorted(s) for s in sets if s]

    def step_batched(self, t: int, shape: LaunchShape, stream: int, idx: list[int] | None = None):
        """One batched launch for streams `idx` (default: all) at frame t."""
        idx = list(range(len(self.models))) if idx is None else idx
        models = [self.models[i] for i in idx]
        hs, fr, mk = _ptr_arrays(models, [self.frames[i][t] for i in idx],
                                 [self.masks[i][t] for i in idx])
        Hs = self._H_steps[t] if len(idx) == len(self.models) else \
            np.ascontiguousarray(np.stack([self.Hs[i][t] for i in idx]).reshape(-1))
        opts = shape.opts()
        rc = _lib.load_library().dmsgm_process_batch_ex(
            len(models), hs, fr, Hs.ctypes.data, mk, _lib.ctypes.byref(opts), stream)
        _lib._check(rc)

    def step_plain(self, t: int, stream: int):
        for i, m in enumerate(self.models):
            _lib.dmsgm_process(m.handle, self.frames[i][t].data_ptr(), self.Hs[i][t],
                               self.masks[i][t].data_ptr(), stream)

    def capture(self, mode: str, shape: LaunchShape | None = None, steps: int | None = None,
                stream: torch.cuda.Stream | None = None, lanes: int = 8) -> torch.cuda.CUDAGraph:
        """Capture `steps` (default T, even) consecutive steps into a graph.
        mode "batched": one batched launch per step, or with shape.lanes > 1
        one per lane, each lane's streams (lane_sets) on a CUDA stream of
        their own; "plain": one launch per stream per step, all on the
        capturing stream; "plain_multi": the same launches with stream i's on
        CUDA stream i % lanes.  Side streams fork from and join back to the
        capturing stream, so independent streams' steps run side by side."""
        steps = steps or self.T
        assert steps % 2 == 0, "an even number of steps keeps the handles' parity consistent"
        stream = stream or torch.cuda.Stream()
        sh = stream.cuda_stream
        g = torch.cuda.CUDAGraph()
        shape = shape or LaunchShape()
        sets = self.lane_sets(shape.lanes) if mode == "batched" and shape.lanes > 1 else None
        nside = lanes if mode == "plain_multi" else (len(sets) if sets else 0)
        side = [torch.cuda.Stream() for _ in range(nside)]
        with torch.cuda.graph(g, stream=stream):
            if side:
                fork = torch.cuda.Event()
                fork.record(stream)
                for s in side:
                    s.wait_event(fork)
            for k in range(steps):
                t = k % self.T
                if mode == "batched" and sets:
                    for s, idx in zip(side, sets):
                        self.step_batched(t, shape, s.cuda_stream, idx)
                elif mode == "batched":
                    self.step_batched(t, shape, sh)
                elif mode == "plain":
                    self.step_plain(t, sh)
                else:
                    for i, m in enumerate(self.models):
                        _lib.dmsgm_process(m.handle, self.frames[i][t].data_ptr(), self.Hs[i][t],
                                           self.masks[i][t].data_ptr(), side[i % lanes].cuda_stream)
            for s in side:
                join = torch.cuda.Event()
                join.record(s)
                stream.wait_event(join)
        return g

    def warm(self, mode: str, shape: LaunchShape | None = None, stream=None):
        stream = stream or torch.cuda.current_stream()
        for t in range(2):
            if mode == "batched":
                self.step_batched(t, shape or LaunchShape(), stream.cuda_stream)
            else:
                self.step_plain(t, stream.cuda_stream)
        stream.synchronize()

    def close(self):
        for m in self.models:
            m.close()


def time_graph(g: torch.cuda.CUDAGraph, stream: torch.cuda.Stream, reps: int = 3) -> float:
    """Mean milliseconds per replay (CUDA events on the replay stream)."""
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            g.replay()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _key(specs, precision, sms):
    sig = sorted(f"{w}x{h}b{b}" for (w, h, b) in specs)
    return json.dumps([sig, precision, sms])


def autotune(runner: BatchRunner, candidates=None, steps: int = 8, use_cache: bool = True):
    """Pick the launch shape (CTA count, PDL, lanes, work-item size) of the batched kernel that gives
    the shortest step on this GPU for this stream mix; cached on disk by the
    mix, the precision and the SM count."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    key = _key(runner.specs, runner.precision, sms)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        d = cache[key]
        return (LaunchShape(d["ctas"], d["use_pdl"], d.get("lanes", 1), d.get("item_warps", 0)),
                d.get("results", []))
    if candidates is None:
        candidates = [LaunchShape(0, False)]   # one work item per CTA, no PDL
        for per_sm in (1, 2, 4, 8):            # persistent grids
            candidates.append(LaunchShape(per_sm * sms, True))
        for item_warps in (4, 8):    # one work item per CTA, the streams over `lanes` launches
            for lanes in (1, 2, 4, 8):
                if lanes <= len(runner.specs):
                    candidates.append(LaunchShape(1 << 30, True, lanes, item_warps))
    stream = torch.cuda.Stream()
    results = []
    for c in candidates:
        runner.warm("batched", c, stream)
        g = runner.capture("batched", c, steps=steps, stream=stream)
        ms = time_graph(g, stream, reps=3) / steps
        results.append({"ctas": c.ctas, "use_pdl": c.use_pdl, "lanes": c.lanes,
                        "item_warps": c.item_warps or 4, "ms_per_step": ms})
        del g
    best = min(results, key=lambda r: r["ms_per_step"])
    shape = LaunchShape(best["ctas"], best["use_pdl"], best["lanes"], best["item_warps"])
    if use_cache:
        cache[key] = {"ctas": shape.ctas, "use_pdl": shape.use_pdl, "lanes": shape.lanes,
                      "item_warps": shape.item_warps, "results": results}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return shape, results

#!/usr/bin/env python3
"""Benchmark of the GB300 DMSGM motion-mask path.

Workload (one "step"): one pass of the fused per-frame kernel over a
pre-staged seeded synthetic 1920x1080 uint8 stream of 300 frames, block 4,
FP32 state, theta_s = 2, theta_d = 4, age cap 30.  The 300 frames (622 MB)
are larger than L2, so every frame is read from HBM; the model state (2 x
2.3 MB) stays L2-resident across frames by the nature of the recurrence.
The step's 300 launches go through the C ABI (dmsgm_process) inside a
stream capture and are replayed as one CUDA graph.

Output: ONE JSON line (rank 0).  value = Mpix/s over all ranks; e2e = the
same metric through dmsgm_process_host (pinned host frames in, host masks
out, copies inside the timed region); roofline = the fused kernel's
algorithmic HBM bytes per launch / its average launch time vs the measured
copy bandwidth; cpu_baseline = the FP64 oracle on this host's cores.

--impl reference times the FP64 oracle (the only reference there is: the
paper ships no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DMSGM Mpix/s & %HBM peak (1080p, 4K); batched vs plain Mpix/s; p99 frame ms"
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (the roofline's own peak is the measured copy rate)
UNIT = "Mpix/s"


def bytes_per_pixel(block: int, precision: str) -> float:
    """Algorithmic HBM bytes per pixel of one frame step: the frame (1 B),
    the mask (1/8 B) and the state read + write of the pixel's block
    (2 x (4 values x s + 2 ages) / B^2)."""
    s = 2 if precision == "fp16" else 4
    return 1.0 + 1.0 / 8.0 + 2.0 * (4 * s + 2) / (block * block)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_tag: str, fingerprint: str):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_tag)
    if not e or e.get("fingerprint") != fingerprint:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled in the background."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.samples = []
        self.proc = None
        self.index = index
        self.t_lo = self.t_hi = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, lo, hi):
        self.t_lo, self.t_hi = lo, hi

    def stop(self):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((t, float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        inwin = [r for r in rows if self.t_lo is not None and self.t_lo - 0.05 <= r[0] <= self.t_hi + 0.05]
        use = inwin or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "in_timed_window": len(inwin)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(vals, device):
    """Element-wise maximum of per-rank timings over all ranks (identity on
    one rank).  The job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_rate(pixels_per_rank, world, ms):
    """Whole-job Mpix/s: every rank processes `pixels_per_rank` in at most
    `ms` milliseconds (weak scaling: one stream replica per GPU)."""
    return world * pixels_per_rank / (ms / 1e3) / 1e6


def cpu_oracle_rate(frames_np, Hs, block, budget_s=12.0, min_frames=3, threads=1):
    """Time the FP64 oracle frame by frame from the first frame until the
    time budget is spent, its block rows on `threads` host threads (0: all);
    returns (Mpix/s, frames, seconds, threads used)."""
    from oracle import oracle_step, set_threads
    used = set_threads(threads)
    T, H, W = frames_np.shape
    st = None
    t0 = time.perf_counter()
    n = 0
    while n < T:
        st, _ = oracle_step(frames_np[n], Hs[n], st, block=block)
        n += 1
        el = time.perf_counter() - t0
        if n >= min_frames and el >= budget_s:
            break
    el = time.perf_counter() - t0
    return n * W * H / el / 1e6, n, el, used


# --------------------------------------------------------------------- our arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm, build as pbuild
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    W, H, B, T, prec = args.width, args.height, args.block, args.frames, args.precision
    frames, Hs = make_stream(spec_for(W, H, T, seed=args.seed + rank), device=dev)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    m = dmsgm.Dmsgm(W, H, B, precision=prec, use_pdl=args.pdl, tile_rows=args.tile_rows)
    masks = dmsgm.new_mask(H, W, dev, n=T)

    def one_pass():
        for t in range(T):
            m.process(frames[t], Hs[t], masks[t], stream=stream)

    # first pass eager (initialises the state), then capture one pass
    with torch.cuda.stream(stream):
        one_pass()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        one_pass()
    stream.synchronize()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            g.replay()
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    h0 = time.time()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            g.replay()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    h1 = time.time()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if sampler:
        sampler.mark(h0, h1)

    # per-frame latency distribution (one eager pass, events around frames)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(T + 1)]
    with torch.cuda.stream(stream):
        for t in range(T):
            evs[t].record(stream)
            m.process(frames[t], Hs[t], masks[t], stream=stream)
        evs[T].record(stream)
    stream.synchronize()
    fr_ms = np.array([evs[t].elapsed_time(evs[t + 1]) for t in range(T)])

    # end to end through host buffers: pinned frames in, host masks out
    host_frames = frames.cpu().pin_memory()
    host_masks = torch.zeros((T, H, dmsgm.mask_words(W)), dtype=torch.int32, pin_memory=True)
    me = dmsgm.Dmsgm(W, H, B, precision=prec, use_pdl=args.pdl, tile_rows=args.tile_rows)
    for _ in range(max(1, min(args.warmup, 2))):
        me.process_host(host_frames, Hs, host_masks, stream=stream)
    stream.synchronize()
    if world > 1:
        dist.barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 10))
    f0.record(stream)
    for _ in range(e2e_steps):
        me.process_host(host_frames, Hs, host_masks, stream=stream)
    f1.record(stream)
    f1.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    if world > 1:
        dist.barrier()
    if sampler:
        sampler.stop()

    # aggregate: max time over ranks
    ms, e2e_ms = reduce_max([ms, e2e_ms], dev)
    npx = W * H
    value = job_rate(args.steps * T * npx, world, ms)
    e2e_val = job_rate(e2e_steps * T * npx, world, e2e_ms)

    if rank == 0:
        peak, peak_kind = load_peaks()
        bpp = bytes_per_pixel(B, prec)
        per_launch_bytes = bpp * npx
        avg_launch_s = ms / 1e3 / (args.steps * T)
        achieved = per_launch_bytes / avg_launch_s / 1e9
        tag = f"dmsgm_step_kernel {W}x{H} B{B} {prec}"
        traffic = ncu_traffic(tag, pbuild.kernel_fingerprint(f"dmsgm_step_b{B}.cu"))
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f16-state/f32-math", "data": "synthetic",
            "config": {"workload": f"plain DMSGM {W}x{H} uint8, block {B}, {prec} state, "
                                   f"{T} pre-staged frames per step, one fused kernel per frame "
                                   f"replayed as a CUDA graph",
                       "width": W, "height": H, "block": B, "frames_per_step": T,
                       "precision": prec, "theta_s": 2.0, "theta_d": 4.0, "age_max": 30,
                       "seed": args.seed, "pdl": bool(args.pdl),
                       "l2": f"inputs larger than L2: {T} frames = {T * npx / 1e6:.0f} MB per step; "
                             f"model state {2 * m.info().state_bytes / 2e6:.1f} MB stays "
                             f"L2-resident between frames (recurrence)",
                       "parallelism": f"replicas x{world} (one stream per GPU)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "nominal_gbs": NOMINAL_HBM_GBS,
                         "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "bytes_per_launch": int(per_launch_bytes),
                         "bytes_per_pixel": bpp, "avg_launch_us": round(avg_launch_s * 1e6, 3),
                         "traffic": traffic, "kernel": "dmsgm_step_kernel"},
            "frame_ms": {"p50": round(float(np.percentile(fr_ms, 50)), 5),
                         "p99": round(float(np.percentile(fr_ms, 99)), 5),
                         "note": "per-frame device time, eager launches, events between frames"},
            "e2e": {"value": round(e2e_val, 1), "unit": UNIT,
                    "h2d_bytes_per_step": T * npx,
                    "d2h_bytes_per_step": T * H * dmsgm.mask_words(W) * 4,
                    "api": "dmsgm_process_host", "steps": e2e_steps},
            "gpu_launches": args.steps * T,
            "clocks": sampler.summary() if sampler else None,
        }
        if args.cpu_baseline:
            fn = frames.cpu().numpy()
            rate, nfr, el, _ = cpu_oracle_rate(fn, Hs, B, budget_s=args.cpu_seconds)
            out["cpu_baseline"] = {"value": round(rate, 3), "unit": UNIT, "cores": 1,
                                   "kind": "oracle",
                                   "sample": f"first {nfr} frames of the same {W}x{H} stream, "
                                             f"FP64 C oracle, 1 thread, {el:.1f} s"}
            # the same oracle with its block rows on every host thread (as the
            # paper's CPU version splits rows over TBB tasks)
            rate, nfr, el, used = cpu_oracle_rate(fn, Hs, B, budget_s=args.cpu_seconds / 2,
                                                  threads=0)
            out["cpu_baseline_parallel"] = {
                "value": round(rate, 3), "unit": UNIT, "cores": used, "kind": "oracle",
                "sample": f"first {nfr} frames of the same {W}x{H} stream, FP64 C oracle, "
                          f"OpenMP over block rows, {used} threads, {el:.1f} s"}
        if args.extra:
            out["extra"] = run_extras(args, dev, stream)
        if args.batched:
            out["batched"] = run_batched(args, dev)
        if args.serve:
            out["serving"] = run_serving(args, dev)
        if args.target:
            # last in the line, so that a tail of the output keeps it
            out["target_4k"] = run_target_4k(args, dev, stream, load_peaks()[0],
                                             with_oracle=bool(args.cpu_baseline))
        print(json.dumps(out), flush=True)
    m.close()
    me.close()
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, dev):
    """64 streams of mixed size (16 each of 320x240, 640x480, 1280x720,
    1920x1080), block 4 or 8 drawn per stream, seeds 1000 + k: all streams
    advance one frame per step in one batched launch (or one per lane when
    the autotuner splits the streams over CUDA streams), steps captured as a
    CUDA graph, launch shape autotuned; against the plain path (one launch
    per stream per step, also captured, on one or 8 CUDA streams)."""
    import torch
    from paper_1702_05156_gb300.batch import BatchRunner, autotune, time_graph
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    peak, _ = load_peaks()
    rng = np.random.Generator(np.random.PCG64(1000))
    sizes = [(320, 240)] * 16 + [(640, 480)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 16
    sizes = sizes[: args.batch_streams]
    specs, frames, Hs = [], [], []
    for k, (w, h) in enumerate(sizes):
        b = 4 if rng.random() < 0.5 else 8
        fr, H = make_stream(spec_for(w, h, args.batch_frames, seed=1000 + k), device=dev)
        specs.append((w, h, b))
        frames.append(fr)
        Hs.append(H)
    r = BatchRunner(specs, frames, Hs)
    shape, tune = autotune(r, steps=8, use_cache=False)
    stream = torch.cuda.Stream(device=dev)
    T = args.batch_frames
    out = {"streams": len(specs), "frames": T, "pixels_per_step": r.pixels_per_step}
    bytes_step = sum(bytes_per_pixel(b, "fp32") * w * h for (w, h, b) in specs)
    for mode in ("batched", "plain", "plain_multi"):
        r.warm("plain" if mode == "plain_multi" else mode, shape, stream)
        g = r.capture(mode, shape, steps=T, stream=stream)
        ms = time_graph(g, stream, reps=2)
        per_step = ms / T
        out[mode] = {"mpix_s": round(r.pixels_per_step / (per_step / 1e3) / 1e6, 1),
                     "ms_per_step": round(per_step, 4),
                     "achieved_gbs": round(bytes_step / (per_step / 1e3) / 1e9, 1),
                     "frac": round(bytes_step / (per_step / 1e3) / 1e9 / peak, 4),
                     "launches_per_step": len(r.lane_sets(shape.lanes)) if mode == "batched" else len(specs)}
        del g
    out["plain"]["note"] = "one CUDA stream, programmatic dependent launch"
    out["plain_multi"]["note"] = "stream i on CUDA stream i % 8, forked and joined in the graph"
    # the same steps launched eagerly from Python (no graph), as a server
    # whose stream set changes every step launches them
    out["eager"] = run_batched_eager(r, shape, stream, peak, bytes_step)
    best_plain = max(out["plain"]["mpix_s"], out["plain_multi"]["mpix_s"])
    out["speedup_batched_vs_plain"] = round(out["batched"]["mpix_s"] / best_plain, 3)
    out["bytes_per_step"] = int(bytes_step)
    one_per_item = shape.ctas == 0 or shape.ctas >= (1 << 30)
    out["launch_shape"] = {"ctas": "one per work item" if one_per_item else shape.ctas,
                           "use_pdl": shape.use_pdl, "lanes": shape.lanes,
                           "item_warps": shape.item_warps or 4}
    out["autotune"] = [{"ctas": "one per work item" if t["ctas"] == 0 or t["ctas"] >= (1 << 30) else t["ctas"],
                        "use_pdl": t["use_pdl"], "lanes": t["lanes"],
                        "item_warps": t["item_warps"], "ms_per_step": round(t["ms_per_step"], 5)}
                       for t in tune]
    out["blocks"] = {"b4": sum(1 for s in specs if s[2] == 4), "b8": sum(1 for s in specs if s[2] == 8)}
    r.close()
    del frames
    torch.cuda.empty_cache()
    return out


def run_batched_eager(r, shape, stream, peak, bytes_step, steps=40):
    """Steps issued one by one from Python through the public calls, timed by
    CUDA events on the issuing stream (host launch cost included): the
    batched form (one call per lane per step) against the plain path (one
    dmsgm_process per stream per step, spread over 8 CUDA streams)."""
    import torch
    from paper_1702_05156_gb300 import _lib

    lanes = [torch.cuda.Stream() for _ in range(8)]
    sets = r.lane_sets(shape.lanes) if shape.lanes > 1 else [None]
    out = {}
    for mode in ("batched", "plain_multi"):
        def one(t):
            if mode == "batched":
                if sets[0] is None:
                    r.step_batched(t, shape, stream.cuda_stream)
                else:
                    for ln, idx in zip(lanes, sets):
                        r.step_batched(t, shape, ln.cuda_stream, idx)
            else:
                for i, m in enumerate(r.models):
                    _lib.dmsgm_process(m.handle, r.frames[i][t].data_ptr(), r.Hs[i][t],
                                       r.masks[i][t].data_ptr(), lanes[i % 8].cuda_stream)
        for t in range(4):
            one(t % r.T)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        fork = torch.cuda.Event()
        e0.record(stream)
        fork.record(stream)
        for ln in lanes:
            ln.wait_event(fork)
        for k in range(steps):
            one(k % r.T)
        for ln in lanes:
            j = torch.cuda.Event()
            j.record(ln)
            stream.wait_event(j)
        e1.record(stream)
        e1.synchronize()
        per_step = e0.elapsed_time(e1) / steps
        out[mode] = {"mpix_s": round(r.pixels_per_step / (per_step / 1e3) / 1e6, 1),
                     "ms_per_step": round(per_step, 4),
                     "frac": round(bytes_step / (per_step / 1e3) / 1e9 / peak, 4)}
    out["speedup_batched_vs_plain"] = round(out["batched"]["mpix_s"] / out["plain_multi"]["mpix_s"], 3)
    out["note"] = (f"{steps} steps launched one by one from Python (ctypes), no graph; the "
                   "host's launch cost is inside the timed region")
    return out


def run_serving(args, dev):
    """256 streams, resolutions uniform over {320x240, 640x480, 1280x720,
    1920x1080, 3840x2160}, Poisson arrivals (20 streams/s), 30 fps for
    U(5, 30) s each, admitted under a fixed HBM budget, served by the
    continuous-batching loop; frames come from pinned host memory and masks
    go back to it.  Three runs of the same arrival sequence: the offered load
    (real time), and time compressed by --serve-saturate (arrivals and frame
    rate that many times faster, durations that many times shorter: the same
    frames, far more than the server can take, so the HBM budget and the
    queues bind) for the batched engine and for the plain per-stream engine
    (one copy, launch and copy back per frame on 8 CUDA streams)."""
    import torch
    from paper_1702_05156_gb300.serve import GpuEngine, PlainEngine, Server, simulate
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    res = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    pools = {}
    for i, (w, h) in enumerate(res):
        fr, H = make_stream(spec_for(w, h, args.serve_pool, seed=100000 + i), device=dev)
        pools[(w, h)] = (fr.cpu().pin_memory(), H)

    def one(engine, sp):
        srv = Server(engine, hbm_budget=int(args.serve_budget_gb * 2 ** 30))
        # the cyclic garbage collector stops every thread while it scans the
        # ~10^5 live request objects; a latency-sensitive application freezes
        # its setup and keeps it off while serving
        import gc
        gc.collect()
        gc.freeze()
        gc.disable()
        try:
            wall, futs = simulate(srv, args.serve_streams, 20.0 * sp, 30.0 * sp, 5.0 / sp, 30.0 / sp,
                                  res, pools, seed=7)
        finally:
            gc.enable()
            gc.unfreeze()
        srv.shutdown()
        st = srv.stats()
        return {"time_compression": sp, "arrival_rate_per_s": 20.0 * sp, "fps": 30.0 * sp,
                "wall_s": round(wall, 2), "frames": st["frames"], "steps": st["steps"],
                "mean_batch": round(st["mean_batch"], 2), "p50_ms": round(st["p50_ms"], 3),
                "p99_ms": round(st["p99_ms"], 3), "max_ms": round(st["max_ms"], 3),
                "served_mpix_s": round(st["pixels"] / wall / 1e6, 1), "failed": st["failed"]}

    out = {"streams": args.serve_streams, "hbm_budget_gb": args.serve_budget_gb,
           "offered": one(GpuEngine(device=dev.index or 0), 1.0)}
    if args.serve_saturate > 0:
        sp = args.serve_saturate
        out["saturated_batched"] = one(GpuEngine(device=dev.index or 0), sp)
        out["saturated_plain"] = one(PlainEngine(device=dev.index or 0), sp)
        out["served_vs_plain"] = round(out["saturated_batched"]["served_mpix_s"]
                                       / max(out["saturated_plain"]["served_mpix_s"], 1e-9), 3)
    out["note"] = ("latency = host submit -> mask back in pinned host memory; at the offered "
                   "load the served Mpix/s is the load itself; the saturated runs measure what "
                   "the server delivers; Python's cyclic garbage collector is frozen and off "
                   "while serving")
    return out


def run_extras(args, dev, stream):
    """Other configurations of the same kernel, reported beside the headline:
    4K at block 4/8, FP32/FP16 state (one pass of 100 frames per step),
    blocks 1, 2 and 16, the mixture-variance option, the preprocessing
    filters on their own, and the step with the preprocessing fused into its
    tile or run as a separate pass."""
    import torch
    from paper_1702_05156_gb300 import dmsgm
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    res = {}
    peak, _ = load_peaks()
    W, H, T = 3840, 2160, args.extra_frames
    frames, Hs = make_stream(spec_for(W, H, T, seed=args.seed), device=dev)
    masks = dmsgm.new_mask(H, W, dev, n=T)

    def graph_time(one_pass, reps):
        """Seconds per pass of a captured pass (two warm replays first)."""
        with torch.cuda.stream(stream):
            one_pass()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            one_pass()
        with torch.cuda.stream(stream):
            for _ in range(2):
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
        return e0.elapsed_time(e1) / 1e3 / reps

    # 4K single stream: block 4 / 8, FP32 / FP16 state; then the widened
    # forms: blocks 1, 2 and 16 (FP32, fewer frames for block 1 and 2) and
    # the mixture-variance option (block 4)
    # (blocks 4 and 8 in FP32 and FP16 are the target_4k line)
    runs = [(16, "fp32", False, T), (2, "fp32", False, min(T, 20)), (1, "fp32", False, min(T, 10)),
            (4, "fp32", True, T)]
    if args.extra in (2, 3):   # the preprocessing or the motion-estimation forms only
        runs = []
    for B, prec, spread, n in runs:
        m = dmsgm.Dmsgm(W, H, B, precision=prec, use_pdl=args.pdl, mix_spread=spread)

        def one_pass():
            for t in range(n):
                m.process(frames[t], Hs[t], masks[t], stream=stream)
        per = graph_time(one_pass, 5 if n >= 50 else 3) / n
        bpp = bytes_per_pixel(B, prec)
        ach = bpp * W * H / per / 1e9
        key = f"4k_b{B}_{prec}" + ("_spread" if spread else "")
        res[key] = {"mpix_s": round(W * H / per / 1e6, 1), "frame_us": round(per * 1e6, 3),
                    "bytes_per_frame": int(bpp * W * H), "achieved_gbs": round(ach, 1),
                    "frac": round(ach / peak, 4)}
        m.close()
    if args.extra != 3:
        res.update(run_pre_extras(args, dev, stream, frames, Hs, masks, graph_time, peak))
    if args.extra in (1, 3):
        res.update(run_homog_extras(args, dev, stream, frames, Hs))
    del frames, masks
    torch.cuda.empty_cache()
    return res


def precision_report(frames, Hs, B, prec, pdl, every):
    """Part of the oracle leg: the step's FP32 / FP16-state results against
    the FP64 oracle, teacher-forced at every `every`-th frame of the stream
    (the oracle steps from the GPU's own previous state), with the parity
    tests' bands (tests/parity_util.py): blocks whose decisions sit within
    FP32 reach of a threshold are exempt and counted; over the others, the
    largest relative error of the means and variances (floor 1e-5 * 255),
    the blocks whose ages differ, and the mask pixels that differ (and how
    many of them lie outside the 1e-4 threshold band)."""
    import torch
    from oracle import set_threads
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_util import StepReport, compare_step
    from paper_1702_05156_gb300 import dmsgm
    set_threads(0)
    T, H, W = frames.shape
    m = dmsgm.Dmsgm(W, H, B, precision=prec, use_pdl=pdl)
    mask = dmsgm.new_mask(H, W, frames.device)
    rep = StepReport()
    checked = []
    prev = None
    rel = 1e-5 if prec == "fp32" else 6e-4
    for t in range(T):
        sample = (t + 1) % every == 0
        if sample:
            prev = m.get_state()
        m.process(frames[t], Hs[t], mask)
        if not sample:
            continue
        got = m.get_state()
        rep.add(compare_step(prev, got, dmsgm.unpack_mask(mask, W), frames[t].cpu().numpy(), Hs[t],
                             block=B, rel=rel))
        checked.append(t)
    m.close()
    torch.cuda.empty_cache()
    return {"frames_checked": checked, "blocks": rep.blocks, "exempt_blocks": rep.exempt,
            "mu_rel_max": rep.max_rel_mu, "var_rel_max": rep.max_rel_var,
            "age_mismatch_blocks": rep.age_mismatch, "state_out_of_tolerance": rep.state_out_of_tol,
            "tolerance_rel": rel, "mask_disagree_frac": rep.mask_mismatch / max(rep.pixels, 1),
            "mask_out_of_band": rep.mask_out_of_band,
            "method": f"teacher-forced every {every}th frame against the FP64 oracle, "
                      "bands of the parity tests"}


def run_target_4k(args, dev, stream, peak, with_oracle):
    """The 3840x2160 precision variant: blocks 4 and 8, FP32 and FP16 state,
    a stream of `target_frames` pre-staged frames per step replayed as a CUDA
    graph (per-frame device time, HBM bytes per frame and the fraction of the
    measured HBM peak), the SM clocks during the timing, and -- in the oracle
    leg -- the errors against the FP64 oracle."""
    import torch
    from paper_1702_05156_gb300 import dmsgm
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    W, H, T = 3840, 2160, args.target_frames
    frames, Hs = make_stream(spec_for(W, H, T, seed=args.seed), device=dev)
    masks = dmsgm.new_mask(H, W, dev, n=T)
    out = {"workload": f"plain DMSGM {W}x{H} uint8, {T} pre-staged frames per step "
                       f"({T * W * H / 1e9:.2f} GB, larger than L2), one fused kernel per frame, "
                       "CUDA graph", "frames": T}
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    time.sleep(0.3)
    t_lo = time.time()
    res = {}
    for B, prec in ((4, "fp32"), (4, "fp16"), (8, "fp32"), (8, "fp16")):
        m = dmsgm.Dmsgm(W, H, B, precision=prec, use_pdl=args.pdl)

        def one_pass():
            for t in range(T):
                m.process(frames[t], Hs[t], masks[t], stream=stream)
        with torch.cuda.stream(stream):
            one_pass()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            one_pass()
        with torch.cuda.stream(stream):
            for _ in range(3):
                g.replay()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                g.replay()
        e1.record(stream)
        e1.synchronize()
        per = e0.elapsed_time(e1) / 1e3 / (reps * T)
        bpp = bytes_per_pixel(B, prec)
        ach = bpp * W * H / per / 1e9
        res[f"b{B}_{prec}"] = {"frame_us": round(per * 1e6, 3), "mpix_s": round(W * H / per / 1e6, 1),
                               "bytes_per_frame": int(bpp * W * H), "achieved_gbs": round(ach, 1),
                               "frac": round(ach / peak, 4), "status": m.status()}
        del g
        m.close()
    t_hi = time.time()
    sampler.mark(t_lo, t_hi)
    sampler.stop()
    out["clocks"] = sampler.summary()
    if with_oracle:
        for B, prec in ((4, "fp32"), (4, "fp16"), (8, "fp32"), (8, "fp16")):
            res[f"b{B}_{prec}"]["vs_oracle"] = precision_report(frames, Hs, B, prec, args.pdl,
                                                                args.target_every)
    out["configs"] = res
    del frames, masks
    torch.cuda.empty_cache()
    return out


def run_pre_extras(args, dev, stream, frames, Hs, masks, graph_time, peak):
    """The preprocessing forms: the filter alone, and the step with it fused
    into its tile or as a separate pass."""
    import torch
    from paper_1702_05156_gb300 import dmsgm
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    res = {}
    W, H, T = 3840, 2160, args.extra_frames
    # the Sec. 2.1 preprocessing on its own (5 x 5 Gaussian, sigma 1, then
    # the 3 x 3 median), HD and 4K: 2 bytes per pixel (read + write)
    for (w, h) in ((3840, 2160), (1920, 1080)):
        src = frames[0, :h, :w].contiguous()
        dst = torch.empty_like(src)
        per = graph_time(lambda: [dmsgm.prefilter(src, 5, 1.0, True, out=dst, stream=stream)
                                  for _ in range(20)], 5) / 20
        ach = 2 * w * h / per / 1e9
        res[f"prefilter_{w}x{h}"] = {"mpix_s": round(w * h / per / 1e6, 1),
                                     "frame_us": round(per * 1e6, 3), "achieved_gbs": round(ach, 1),
                                     "frac": round(ach / peak, 4)}
    # the step with the same preprocessing, block 4, FP32: filtered inside the
    # step kernel's tile (fused), and as its own pass before the step
    for (w, h, name) in ((3840, 2160, "4k"), (1920, 1080, "hd")):
        n = min(T, 50)
        if (w, h) == (W, H):
            fr, hs = frames, Hs
        else:
            fr, hs = make_stream(spec_for(w, h, n, seed=args.seed), device=dev)
        mk = dmsgm.new_mask(h, w, dev, n=n)
        for sep in (False, True):
            m = dmsgm.Dmsgm(w, h, 4, use_pdl=args.pdl, prefilter=(5, 1.0, True),
                            prefilter_separate=sep)

            def one_pass():
                for t in range(n):
                    m.process(fr[t], hs[t], mk[t], stream=stream)
            per = graph_time(one_pass, 5) / n
            res[f"{name}_b4_fp32_pre_" + ("separate" if sep else "fused")] = {
                "mpix_s": round(w * h / per / 1e6, 1), "frame_us": round(per * 1e6, 3),
                "fused": m.info().pre_fused}
            m.close()
        del fr, hs, mk
    return res


def run_homog_extras(args, dev, stream, frames, Hs):
    """The motion-estimation front end (corners, pyramidal Lucas-Kanade,
    RANSAC) per frame pair, HD and 4K: device time per estimate (each call
    ends with its result on the host), and the estimate's distance from the
    stream's known camera motion at the frame corners."""
    import time

    import numpy as np
    import torch
    from paper_1702_05156_gb300.homog import HomographyEstimator
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    res = {}
    for (w, h, name) in ((1920, 1080, "hd"), (3840, 2160, "4k")):
        n = 12
        if (w, h) == (3840, 2160):
            fr, hs = frames[:n], np.asarray(Hs[:n])
        else:
            fr, hs = make_stream(spec_for(w, h, n, seed=args.seed), device=dev)
            hs = np.asarray(hs)
        # the stand-in stream's moving rectangles hold the strongest corners;
        # a 0.1 % quality cut keeps the background texture's as well
        est = HomographyEstimator(w, h, quality=0.001, thresh=1.0)
        corners = np.array([[0, 0], [w, 0], [0, h], [w, h]], float)

        def apply(Hm, p):
            q = np.c_[p, np.ones(len(p))] @ Hm.T
            return q[:, :2] / q[:, 2:]
        with torch.cuda.stream(stream):
            for t in range(1, 4):   # warm-up
                est.estimate(fr[t - 1], fr[t], stream=stream)
            torch.cuda.synchronize()
            errs, ins, t0 = [], [], time.perf_counter()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for t in range(1, n):
                Hm, r = est.estimate(fr[t - 1], fr[t], stream=stream)
                errs.append(float(np.abs(apply(Hm, corners) - apply(hs[t], corners)).max()))
                ins.append(r.inliers)
            e1.record(stream)
            e1.synchronize()
            wall = (time.perf_counter() - t0) / (n - 1)
        dev_s = e0.elapsed_time(e1) / 1e3 / (n - 1)
        res[f"homog_{name}"] = {"pair_us": round(dev_s * 1e6, 1), "wall_us": round(wall * 1e6, 1),
                                "mpix_s": round(w * h / wall / 1e6, 1),
                                "corner_err_px_max": round(max(errs), 3),
                                "inliers_mean": round(float(np.mean(ins)), 1),
                                "params": "quality 0.001, ransac thresh 1 px, other defaults"}
        est.close()
        del fr
    return res


# --------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    from oracle import build_oracle, oracle_step, set_threads
    from paper_1702_05156_gb300.synth import make_stream, spec_for

    build_oracle()
    threads = set_threads(0)   # every host thread (OpenMP over block rows)
    W, H, B = args.width, args.height, args.block
    per_step = args.ref_frames
    need = per_step * (args.steps + args.warmup)
    T = min(args.frames, need)
    frames, Hs = make_stream(spec_for(W, H, T, seed=args.seed), device="cpu")
    fn = frames.numpy()
    st = None
    idx = 0

    def step():
        nonlocal st, idx
        for _ in range(per_step):
            st, _ = oracle_step(fn[idx % T], Hs[idx % T], None if idx == 0 else st, block=B)
            idx += 1
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps * per_step * W * H / el / 1e6
    sample = (f"{per_step} frames per step of the {W}x{H} block-{B} stream, FP64 C oracle, "
              f"OpenMP over block rows, {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el * 1e3 / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"plain DMSGM {W}x{H} uint8, block {B}, FP64 oracle (the paper "
                               f"ships no code; the reference arm is the oracle written from it)",
                   "width": W, "height": H, "block": B},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }), flush=True)
    del torch


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--block", type=int, default=4)
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--pdl", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--extra", type=int, default=1,
                    help="1: all extra configurations, 2: the preprocessing forms only, "
                         "3: the motion-estimation front end only, 0: none")
    ap.add_argument("--extra-frames", type=int, default=100)
    ap.add_argument("--target", type=int, default=1,
                    help="1: the 3840x2160 block 4 / 8, FP32 / FP16 line (target_4k)")
    ap.add_argument("--target-frames", type=int, default=500)
    ap.add_argument("--target-every", type=int, default=50,
                    help="oracle comparison of target_4k at every n-th frame")
    ap.add_argument("--ref-frames", type=int, default=4)
    ap.add_argument("--batched", type=int, default=1)
    ap.add_argument("--batch-streams", type=int, default=64)
    ap.add_argument("--batch-frames", type=int, default=200)
    ap.add_argument("--serve", type=int, default=1)
    ap.add_argument("--serve-streams", type=int, default=256)
    ap.add_argument("--serve-saturate", type=float, default=40.0,
                    help="time compression of the saturated serving runs (0: none)")
    ap.add_argument("--serve-pool", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    ap.add_argument("--config", default=None,
                    help="JSON file of argument defaults (keys: the option names with '_'); "
                         "options given on the command line override it")
    pre, _ = ap.parse_known_args()
    if pre.config:
        with open(pre.config) as f:
            cfg = json.load(f)
        known = {a.dest for a in ap._actions}
        unknown = sorted(set(cfg) - known)
        if unknown:
            ap.error(f"--config: unknown keys {unknown}")
        ap.set_defaults(**cfg)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

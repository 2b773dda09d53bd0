"""GPU: the batched runner and the serving loop give each stream exactly the
results it gets alone (the batched kernel runs the same per-block math)."""
import numpy as np
import pytest
import torch

from paper_1702_05156_gb300.synth import StreamSpec, make_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_1702_05156_gb300 import dmsgm
    return dmsgm


CFGS = [(320, 240, 4), (640, 480, 8), (1280, 720, 4), (320, 240, 8), (48, 24, 4)]


def _streams(T):
    return [make_stream(StreamSpec(w, h, T, seed=300 + i), device="cuda")
            for i, (w, h, b) in enumerate(CFGS)]


def _solo(lib, streams, T):
    out = []
    for (w, h, b), (fr, Hs) in zip(CFGS, streams):
        m = lib.Dmsgm(w, h, b)
        out.append(torch.stack([m.process(fr[t], Hs[t]).clone() for t in range(T)]).cpu())
        m.close()
    return out


def test_served_equals_alone(lib):
    from paper_1702_05156_gb300.serve import GpuEngine, Server
    T = 6
    streams = _streams(T)
    ref = _solo(lib, streams, T)
    srv = Server(GpuEngine(), hbm_budget=1 << 30)
    futs = {}
    for sid, (w, h, b) in enumerate(CFGS):
        srv.open_stream(sid, w, h, b)
    hosts = [fr.cpu().pin_memory() for fr, _ in streams]
    for t in range(T):                      # interleaved arrival
        for sid in range(len(CFGS)):
            futs[(sid, t)] = srv.submit(sid, hosts[sid][t], streams[sid][1][t])
    for sid in range(len(CFGS)):
        srv.close_stream(sid)
    for (sid, t), f in futs.items():
        assert torch.equal(f.result(timeout=60), ref[sid][t]), (sid, t)
    srv.shutdown()
    assert srv.stats()["frames"] == T * len(CFGS)


def test_batch_runner_graph_equals_alone(lib):
    from paper_1702_05156_gb300.batch import BatchRunner, LaunchShape
    T = 4
    streams = _streams(T)
    ref = _solo(lib, streams, T)
    r = BatchRunner(CFGS, [fr for fr, _ in streams], [h for _, h in streams])
    s = torch.cuda.Stream()
    for mode_shape in (LaunchShape(0, True), LaunchShape(1 << 30, False), LaunchShape(3, True),
                       LaunchShape(1 << 30, True, 2), LaunchShape(1 << 30, True, 2, 8),
                       LaunchShape(0, True, 1, 8)):
        for m in r.models:
            m.reset()
        g = r.capture("batched", mode_shape, steps=T, stream=s)
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        for i in range(len(CFGS)):
            assert torch.equal(r.masks[i].cpu(), ref[i]), (mode_shape, i)
    r.close()


def test_bench_batched_workload_equals_alone(lib):
    """The bench's batched workload at full size -- 64 streams, 16 each of
    320x240, 640x480, 1280x720 and 1920x1080, block 4 or 8 drawn per stream
    from the same seeded generator -- in the launch configurations the
    autotuner picks from (one work item per CTA on one, two and four lanes,
    items of 4 or 8 warps, captured as a graph): every stream's masks and
    final state equal the stream processed alone, bit for bit."""
    from paper_1702_05156_gb300.batch import BatchRunner, LaunchShape
    from paper_1702_05156_gb300.synth import spec_for
    T = 4
    rng = np.random.Generator(np.random.PCG64(1000))
    sizes = [(320, 240)] * 16 + [(640, 480)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 16
    specs, frames, Hs = [], [], []
    for k, (w, h) in enumerate(sizes):
        b = 4 if rng.random() < 0.5 else 8
        fr, H = make_stream(spec_for(w, h, T, seed=1000 + k), device="cuda")
        specs.append((w, h, b))
        frames.append(fr)
        Hs.append(H)
    ref, ref_state = [], []
    for (w, h, b), fr, H in zip(specs, frames, Hs):
        m = lib.Dmsgm(w, h, b)
        ref.append(torch.stack([m.process(fr[t], H[t]).clone() for t in range(T)]).cpu())
        ref_state.append(m.get_state())
        m.close()
    r = BatchRunner(specs, frames, Hs)
    s = torch.cuda.Stream()
    for shape in (LaunchShape(1 << 30, True), LaunchShape(1 << 30, True, 2),
                  LaunchShape(1 << 30, True, 4), LaunchShape(1 << 30, True, 2, 8)):
        for m in r.models:
            m.reset()
        g = r.capture("batched", shape, steps=T, stream=s)
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        for i in range(len(specs)):
            assert torch.equal(r.masks[i].cpu(), ref[i]), (shape, i, specs[i])
            st = r.models[i].get_state()
            for key in st:
                assert np.array_equal(st[key], ref_state[i][key]), (shape, i, key)
            assert r.models[i].status() == 0
        del g
    r.close()


def _serve(lib, engine, budget, T, waves=1):
    """Open every stream at once, submit its frames in `waves` bursts (the
    later ones while earlier frames are on the GPU), close it; returns the
    server and the masks per (stream, frame)."""
    import time
    from paper_1702_05156_gb300.serve import Server
    streams = _streams(T)
    srv = Server(engine, hbm_budget=budget)
    hosts = [fr.cpu().pin_memory() for fr, _ in streams]
    for sid, (w, h, b) in enumerate(CFGS):
        srv.open_stream(sid, w, h, b)
    futs = {}
    per = (T + waves - 1) // waves
    for wv in range(waves):
        for sid in range(len(CFGS)):
            for t in range(wv * per, min(T, (wv + 1) * per)):
                futs[(sid, t)] = srv.submit(sid, hosts[sid][t], streams[sid][1][t])
        time.sleep(0.002)
    for sid in range(len(CFGS)):
        srv.close_stream(sid)
    got = {k: f.result(timeout=60).clone() for k, f in futs.items()}
    srv.shutdown()
    return srv, streams, got


def test_binding_budget_admits_streams_as_memory_frees(lib):
    """A budget that holds the two largest streams at most: the others wait,
    are admitted as earlier streams retire, and each result equals the
    stream's result alone."""
    from paper_1702_05156_gb300.serve import GpuEngine
    T = 6
    eng = GpuEngine()
    sizes = sorted((eng.stream_bytes(w, h, b) for (w, h, b) in CFGS), reverse=True)
    budget = sizes[0] + sizes[1] + 1
    srv, streams, got = _serve(lib, eng, budget, T, waves=2)
    ref = _solo(lib, streams, T)
    for (sid, t), m in got.items():
        assert torch.equal(m, ref[sid][t]), (sid, t)
    assert srv.stats()["frames"] == T * len(CFGS) and srv.stats()["failed"] == 0
    # resident streams never exceeded the budget: replay admissions and releases
    events = sorted([(t, 1, sid) for t, sid in srv.admit_log] +
                    [(t, -1, sid) for t, sid in srv.release_log])
    used = peak = 0
    admitted_after_release = 0
    released = 0
    for t, kind, sid in events:
        w, h, b = CFGS[sid]
        used += kind * eng.stream_bytes(w, h, b)
        peak = max(peak, used)
        released += kind < 0
        admitted_after_release += kind > 0 and released > 0
    assert peak <= budget
    assert admitted_after_release >= 1     # some stream waited for memory to free
    assert len(srv.admit_log) == len(CFGS)


def test_plain_engine_equals_alone(lib):
    """The plain per-stream engine (one copy, launch and copy back per frame
    on several CUDA streams) under the same server gives the same results."""
    from paper_1702_05156_gb300.serve import PlainEngine
    T = 6
    srv, streams, got = _serve(lib, PlainEngine(lanes=3), 1 << 30, T, waves=3)
    ref = _solo(lib, streams, T)
    for (sid, t), m in got.items():
        assert torch.equal(m, ref[sid][t]), (sid, t)

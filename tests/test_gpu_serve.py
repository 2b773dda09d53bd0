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
    for mode_shape in (LaunchShape(0, True), LaunchShape(1 << 30, False), LaunchShape(3, True)):
        for m in r.models:
            m.reset()
        g = r.capture("batched", mode_shape, steps=T, stream=s)
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        for i in range(len(CFGS)):
            assert torch.equal(r.masks[i].cpu(), ref[i]), (mode_shape, i)
    r.close()

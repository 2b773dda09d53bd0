"""The multi-rank path of bench.py on CPU: two gloo ranks, one stream
replica each; the job time is the slowest rank's and the rate counts every
rank's pixels."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + 5.0 * rank, 3.0 - rank]          # rank 1 is slower in the first
    out = bench.reduce_max(ms, torch.device("cpu"))
    rate = bench.job_rate(1_000_000, world, out[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out, rate))


def test_two_rank_max_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for rank, out, rate in res:
        assert out == [15.0, 3.0]
        assert rate == pytest.approx(2 * 1_000_000 / 0.015 / 1e6)


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the reference arm; another rank
    prints nothing and exits 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_reduce_is_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2.5], torch.device("cpu")) == [1.5, 2.5]
    assert bench.job_rate(2_000_000, 1, 1000.0) == pytest.approx(2.0)


def test_config_file_sets_defaults_and_rejects_unknown_keys(tmp_path):
    """bench.py --config: a JSON file of option defaults; unknown keys are an
    argument error (exit 2) before any work."""
    bad = tmp_path / "bad.json"
    bad.write_text('{"stepz": 3}')
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--config", str(bad)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "unknown keys" in r.stderr
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_cfg", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    good = tmp_path / "good.json"
    good.write_text('{"steps": 4, "width": 640, "height": 480}')
    seen = {}

    def fake_run(args):
        seen.update(vars(args))
        raise SystemExit(0)
    orig_argv = sys.argv
    try:
        sys.argv = ["bench.py", "--config", str(good), "--steps", "7"]
        b.run_gpu = fake_run
        with pytest.raises(SystemExit):
            b.main()
    finally:
        sys.argv = orig_argv
    assert seen["steps"] == 7 and seen["width"] == 640 and seen["height"] == 480

"""Multi-rank path of bench.py (replicas, one box per rank): the job time is
the slowest rank's and the rate counts every rank's steps.  Runs as two gloo
ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 200.0][rank]
    ms = bench.max_over_ranks(ms_local, world, torch.device("cpu"))
    q.put((rank, ms, bench.whole_job_rate(10, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 200.0
        assert rate == pytest.approx(2 * 10 / 0.2)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_stored_traffic_applies_only_to_the_current_kernel_sources():
    """The DRAM traffic that bench.py reports for its roofline kernel comes from
    a committed capture; it is reported only while that capture's digest is the
    one of the kernel's current sources, and then it is close to the
    algorithmic bytes."""
    import json
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "traffic_xpass_fp32_N1024.json")) as f:
        tf = json.load(f)
    got = bench.stored_traffic("xpass", 1024)
    if tf["kernel_digest"] == bench._kernel_digest():
        assert got == tf["bytes_per_launch"]
        assert 0.9 < tf["bytes_per_launch"] / tf["algorithmic_bytes"] < 1.2
    else:
        assert got is None
    assert bench.stored_traffic("xpass", 12345) is None

"""The N > 1 path of bench.py without a GPU: world-size-2 gloo ranks run
independent replicas; the whole-job value uses the slowest rank's time."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms = b.max_over_ranks(torch, dist, local_ms)
    value = b.whole_job_value(world, 1000, ms)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 150.0
        assert abs(value - 2 * 1000 / 0.150) < 1e-6


def test_single_rank_value():
    b = _bench()
    assert b.max_over_ranks(None, None, 3.5) == 3.5
    assert abs(b.whole_job_value(1, 500 * 512 ** 3, 612.0) - 500 * 512 ** 3 / 0.612) < 1

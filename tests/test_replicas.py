"""The multi-rank host logic of the benchmark, on CPU: two gloo ranks (one process each)
time different amounts, and every rank must report the slowest time and the whole-job
throughput of the two replicas (weak scaling: each rank advances its own lattice)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    worst = bench.max_over_ranks(ms, torch.device("cpu"))
    out[rank] = (worst, bench.job_mlups(1 << 20, world, 10, worst))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    want = 2 * (1 << 20) * 10 / 0.150 / 1e6
    for r in range(world):
        assert res[r][0] == 150.0
        assert abs(res[r][1] - want) < 1e-9 * want


def test_single_process_is_unchanged():
    import bench

    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.default_width("d2q9", "fp16", 8192) == 8
    assert bench.default_width("d2q9", "fp32", 4098) == 2
    assert bench.default_width("d3q19", "bf16", 255) == 1

"""The multi-GPU path of bench.py is replicas only (one process per GPU, no data-path
collective): each rank times its own replica, the job's time is the maximum over ranks
and the value counts every rank's iterations.  Checked here with two gloo ranks on CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    ms = [12.5, 19.75][rank]                    # the ranks' own timed regions
    dist.barrier()
    out[rank] = bench.max_over_ranks(ms, dist, "cpu")
    ref = bench.run_reference(None, rank, world) if rank == 1 else "rank0"
    out[2 + rank] = ref is None or ref == "rank0"
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_iterations():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 19.75
    assert out[2] and out[3]                    # the reference arm runs on rank 0 only
    bench = _bench()
    assert bench.job_throughput(10, world, 19.75) == pytest.approx(10 * 2 / 19.75e-3)
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0

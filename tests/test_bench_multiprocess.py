"""The replica path of bench.py under torch.distributed: two CPU ranks (gloo) with
different timed regions; the job time is the maximum and the throughput counts every
rank's solves."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max, value = bench.aggregate(1000.0 * (rank + 1), steps=3, world=world)
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get() for _ in range(world))
    for rank, ms_max, value in out:
        assert ms_max == pytest.approx(2000.0)
        assert value == pytest.approx(world * 3 / 2.0)


def test_single_process_aggregate():
    import bench
    ms, v = bench.aggregate(500.0, steps=2, world=1)
    assert ms == 500.0 and v == pytest.approx(4.0)


def test_bench_defines_every_leg():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for name in ("gpu_arm", "spmv_measure", "batched_measure", "roofline", "traffic_for",
                 "oracle_sample", "reference_arm", "make_config", "aggregate"):
        assert callable(getattr(mod, name)), name

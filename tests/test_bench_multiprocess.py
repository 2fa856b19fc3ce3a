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
    for name in ("gpu_arm", "spmv_measure", "batched_measure", "legs_measure", "roofline",
                 "hot_loop_roofline", "traffic_for", "oracle_baseline", "OracleReplay",
                 "reference_arm", "make_config", "aggregate", "cpu_info"):
        assert callable(getattr(mod, name)), name


def test_roofline_names_the_dominant_family_and_its_rate():
    """The roofline object of the bench line: the family with the largest device time,
    achieved = work per launch / average launch time, frac = achieved / peak."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    nf = len(mod.NAMES)
    prof = {"ms": [0.0] * nf, "launches": [0] * nf, "work": [0.0] * nf}
    # family 0 (an A pass, bytes): 100 launches of 1 GB in 200 ms -> 500 GB/s
    prof["ms"][0], prof["launches"][0], prof["work"][0] = 200.0, 100, 100 * 1e9
    # family 3 (GEMM, flops): 10 launches of 1 TFLOP in 1000 ms -> 10 TFLOP/s, dominant
    prof["ms"][3], prof["launches"][3], prof["work"][3] = 1000.0, 10, 10 * 1e12
    r = mod.roofline(prof)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel"):
        assert key in r, key
    assert r["kernel"] == mod.NAMES[3] and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(10.0)
    assert r["frac"] == pytest.approx(10.0 / r["peak"], rel=1e-3)
    assert r["families"][mod.NAMES[0]]["GBps"] == pytest.approx(500.0)


def test_oracle_replay_strata_follow_the_schedule():
    """The CPU baseline's strata: the sketch, every rank step, and per rebuild the build
    and a phase sample scaled by the phase length, in driver order; running them all on a
    small problem covers every stratum, and the assembled solve time is their scaled sum."""
    import importlib.util
    import os

    from oracle import aplicur_oracle as O
    from paper_2604_05065_gb300 import workloads as wl
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod3", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    p = wl.config1(scale=4)
    res = O.aplicur(p.dense, p.b, p.mu, p.sketch_dim, O.Options(seed=1), tol=1e-8)
    gold = {"rank_steps": res.rank_steps,
            "bench_tol": {"phases": [ph["iters"] for ph in res.phases]}}
    rep = mod.OracleReplay(p, gold)
    names = [nm for nm, _, _ in rep.strata]
    nb = sum(1 for st in res.rank_steps if st["rebuild"])
    assert names[0] == "sketch" and len(names) == 1 + len(res.rank_steps) + 2 * nb
    assert sum(1 for nm in names if nm.startswith("rank step")) == len(res.rank_steps)
    while not rep.covered():
        rep.run_next()
    tot = sum(sum(v) / len(v) * sc for (nm, _, sc) in rep.strata for v in [rep.times[nm]])
    assert rep.solve_seconds() == pytest.approx(tot)
    ph = [sc for nm, _, sc in rep.strata if nm.startswith("phase")]
    iters = gold["bench_tol"]["phases"]
    assert ph == pytest.approx([(k + 2) / (rep.SAMPLE_ITERS + 2) for k in iters[:len(ph)]])


def test_bench_package_names_exist():
    """Every package attribute bench.py uses is exported (a missing name would only show
    on the GPU machine)."""
    import inspect
    import re

    import bench
    import paper_2604_05065_gb300 as pkg
    names = set(re.findall(r"pkg\.([A-Za-z_][A-Za-z_0-9]*)", inspect.getsource(bench)))
    assert names and all(hasattr(pkg, n) for n in names), [n for n in names if not hasattr(pkg, n)]

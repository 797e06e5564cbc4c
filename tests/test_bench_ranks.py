"""The multi-process path of bench.py on the CPU: two gloo ranks agree on the
job's time (the largest per-rank time) and on the whole-job value, and the
reference arm runs on rank 0 only (the other ranks do no work)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 150.5][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_value(world, 10, 1000, ms)
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.5, 150.5]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 10 * 1000 / 0.1505)


def test_single_process_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 4, 250, 1000.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload, tile, warmup, steps = "planted60", 16, 1, 1
    assert bench.run_reference(Args(), 1) is None
    out = bench.run_reference(Args(), 0)
    assert out["impl"] == "reference" and out["value"] > 0


def test_host_cores_reads_the_cgroup_quota():
    sys.path.insert(0, ROOT)
    import pathlib
    import bench
    work = pathlib.Path(ROOT) / "tests" / "_build"
    work.mkdir(exist_ok=True)
    f = work / f"cpu.max.{os.getpid()}"
    free = bench.host_cores(str(work / "absent"))
    assert free >= 1
    f.write_text("max 100000\n")
    assert bench.host_cores(str(f)) == free
    f.write_text("150000 100000\n")
    assert bench.host_cores(str(f)) == min(free, 2)
    f.write_text("50000 100000\n")
    assert bench.host_cores(str(f)) == 1
    f.unlink()

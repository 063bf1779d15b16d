"""Multi-process path of bench.py on the CPU: two gloo ranks on 127.0.0.1.

The hot path runs as independent replicas (one per GPU, no collective in the
data path); the job's time is the slowest rank's, taken after a barrier, and
its value is all ranks' units over that time.  These tests run the same
helpers bench.py uses on a world of two CPU processes.
"""
import os
import socket
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank "timed region": rank 1 is the slow one
        dist.barrier()
        t0 = time.perf_counter()
        time.sleep(0.05 + 0.15 * rank)
        dt = time.perf_counter() - t0
        dist.barrier()
        t_max = bench.max_over_ranks(dt, dist, "cpu")
        units = 1000 * (rank + 1)  # unequal units must not matter: the job counts units_per_rank x world
        value = bench.whole_job_rate(1000, world, t_max)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r %r %r\n" % (dt, t_max, value, units))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(2)]
    dts = [float(r[0]) for r in rows]
    t_max = [float(r[1]) for r in rows]
    values = [float(r[2]) for r in rows]
    # both ranks agree on the slowest rank's time, which is rank 1's
    assert t_max[0] == t_max[1] == max(dts)
    assert dts[1] > dts[0]
    assert values[0] == values[1] == pytest.approx(2 * 1000 / max(dts))


def test_helpers_without_process_group():
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.whole_job_rate(300, 4, 2.0) == 600.0

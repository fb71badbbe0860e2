"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
evaluates its own replica (distinct seeds), the job's time is the slowest
rank's, and the whole-job value counts the candidates of every rank."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 95.5][rank]  # the ranks' own timed totals
    total = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{total} {bench.replica_seed(1, rank)}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(2)]
    totals = [float(r[0]) for r in rows]
    seeds = [int(r[1]) for r in rows]
    assert totals == [120.0, 120.0]  # both ranks see the slowest rank's time
    assert seeds[0] != seeds[1]      # independent replicas
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 10 steps x 1,000 candidates in 120 ms
    assert bench.job_value(1000, 2, 10, 120.0) == pytest.approx(1000 * 2 * 10 / 0.120)
    assert bench.max_over_ranks(7.0, None, None) == 7.0

"""Multi-rank path of bench.py on CPU: world size 2 over gloo (no GPU).

Each rank traces its own wavefront (replicas, weak scaling); the job's time is
the slowest rank's, and its throughput counts every rank's rays.
"""
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
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = bench.dist_env()
    local_ms = [120.0, 150.0][rank]
    m = bench.max_over_ranks(local_ms, "cpu")
    v = bench.whole_job_mrays(w, 1_000_000, 10, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, m, v))


def test_two_ranks_take_the_slowest_time_and_all_rays():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    for _, _, m, v in out:
        assert m == 150.0
        assert v == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e6)


def test_one_rank_without_a_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, "cpu") == 42.0
    assert bench.whole_job_mrays(1, 1000, 4, 2.0) == pytest.approx(2.0)

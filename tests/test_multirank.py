"""Multi-GPU form of the benchmark: replicas only.  The path shards by event with
no exchange step (events are independent; arXiv 2101.11489 section 3 runs many
events concurrently), so each rank processes its own events and the only
cross-rank operation is the maximum of the per-rank timings.  This host logic is
checked here on CPU with two gloo ranks, rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, root, q):
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = list(bench.shard(rank, 5))
    env = bench.dist_env()
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ids, env, got))


def test_two_gloo_ranks_shard_events_and_take_the_maximum_time():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ROOT, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, ids, env, got = q.get(timeout=120)
        res[rank] = (ids, env, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == [0, 1, 2, 3, 4] and res[1][0] == [5, 6, 7, 8, 9]  # disjoint, no event twice
    assert res[0][1][:2] == (0, 2) and res[1][1][:2] == (1, 2)
    for r in (0, 1):
        assert res[r][2] == [2.0, 10.0]  # both ranks see the maximum of both


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert list(bench.shard(0, 3)) == [0, 1, 2]
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, workload = 1, 1, "batch64"

    assert bench.run_reference(A(), 1, 2, 2, 64) is None
    assert capsys.readouterr().out == ""

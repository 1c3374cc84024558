"""The multi-rank path on CPU (two gloo ranks, no GPU): the sweep's discharges
are dealt to the ranks disjointly and in balance, and the benchmark's
weak-scaling aggregate takes the slowest rank's time and all ranks' work."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2310_04957_gb300 import sweep

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = sweep.design(64, seed=4)
    weights = [p["n_per_species"] for p in pts]
    mine = sweep.shard(weights, rank, world)
    work = float(sum(weights[k] for k in mine))
    t, w = bench.across_ranks(10.0 + rank, work, dist, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, work, t, w))


def test_two_gloo_ranks_shard_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [set(r[1]) for r in res]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(64))
    works = [r[2] for r in res]
    assert max(works) / min(works) < 1.05  # balanced by particle count
    for _, _, _, t, w in res:
        assert t == 11.0  # the slowest rank's time
        assert w == pytest.approx(sum(works))  # every rank's work


def test_shard_single_rank_takes_everything():
    from paper_2310_04957_gb300 import sweep

    assert sweep.shard([3, 1, 2], 0, 1) == [0, 1, 2]
    assert sweep.shard([5, 5, 5, 5], 1, 4) == [1]

"""Host logic of the multi-GPU benchmark, with two gloo ranks on the CPU.

Each rank counts its own read set (no collective on the data path); the
benchmark only reduces the timing (max over ranks) and the work (sum over
ranks).  Here two CPU processes check the seed assignment and both reductions.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench

    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    dev = torch.device("cpu")
    seed = bench.shard_seed(r)
    # per-rank "measurements": rank 1 is slower and counts more windows
    t = 1.0 + r
    windows = 1000 * (r + 1)
    t_max = bench.reduce_max(t, dist, dev)
    w_sum = bench.reduce_sum(float(windows), dist, dev)
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
    dist.all_gather(seeds, torch.tensor([seed], dtype=torch.int64))
    bench.barrier(dist)
    q.put((r, w, local, t_max, w_sum, [int(s.item()) for s in seeds]))
    dist.destroy_process_group()


def test_two_rank_reductions_and_seeds():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, w, local, t_max, w_sum, seeds) in enumerate(out):
        assert rank == r and w == world and local == r
        assert t_max == 2.0  # the slowest rank's time
        assert w_sum == 3000.0  # windows of all ranks
        assert seeds[0] == 2  # rank 0 counts the canonical workload
        assert len(set(seeds)) == world  # every rank has its own read set
    # the aggregate the benchmark prints: all ranks' work over the slowest time
    assert out[0][4] / out[0][3] == 1500.0


def test_single_process_needs_no_process_group():
    import bench

    assert bench.init_dist(1, "gloo") is None
    assert bench.reduce_max(3.5, None, None) == 3.5
    assert bench.reduce_sum(2.0, None, None) == 2.0
    bench.barrier(None)

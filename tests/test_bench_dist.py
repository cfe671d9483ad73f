"""Host logic of the multi-GPU benchmark, with two gloo ranks on the CPU.

The one job is sharded by hash range: each rank owns a contiguous range of
the 64 hash shards (no collective on the data path); the benchmark reduces
only the timing (max over ranks), counts the job's windows once, and after
the timed steps gathers the ranks' results for a merge by key.  Here two CPU
processes check the shard assignment, the reduction and the gather + merge
of disjoint sorted results.
"""
import os
import socket

import numpy as np
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
    import paper_1712_03254_gb300 as kc

    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    dev = torch.device("cpu")
    knobs = bench.owner_knobs(r, w)
    # per-rank "measurements": rank 1 is slower
    t_max = bench.reduce_max(1.0 + r, dist, dev)
    # each rank's result: the keys of its own shards (here: keys = shard * 1000 + i, i < 3)
    keys = np.array([s * 1000 + i for s in range(knobs["own_lo"], knobs["own_hi"]) for i in range(3)], np.uint64)
    counts = (keys % 7 + 2).astype(np.uint32).reshape(-1, 1)
    gathered = [None] * w
    dist.all_gather_object(gathered, (keys, counts))
    mk, mc = kc.merge_results(gathered, 1)
    bench.barrier(dist)
    q.put((r, w, local, knobs, t_max, mk.tolist(), mc[:, 0].tolist()))
    dist.destroy_process_group()


def test_two_rank_shards_reduction_and_merge():
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
    out.sort(key=lambda x: x[0])
    import bench

    assert [o[3] for o in out] == [{"own_bits": bench.OWN_BITS, "own_lo": 0, "own_hi": 32},
                                   {"own_bits": bench.OWN_BITS, "own_lo": 32, "own_hi": 64}]
    want = [s * 1000 + i for s in range(64) for i in range(3)]
    for r, (rank, w, local, knobs, t_max, mk, mc) in enumerate(out):
        assert rank == r and w == world and local == r
        assert t_max == 2.0  # the slowest rank's time
        assert mk == want  # the union of both ranks' shards, in key order
        assert mc == [k % 7 + 2 for k in want]


def test_single_process_needs_no_process_group():
    import bench

    assert bench.init_dist(1, "gloo") is None
    assert bench.reduce_max(3.5, None, None) == 3.5
    assert bench.owner_knobs(0, 1) == {}
    bench.barrier(None)

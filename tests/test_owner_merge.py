"""Hash-range ownership and the merge of per-owner results, on the CPU.

A job shards by key: handle r of N owns the keys whose top own_bits hash bits
fall in its shard range, counts only those (its own filter slice and tables,
no synchronisation with the others: Section II-B, partitions by k-mer with
owner-private structures), and the job's result is the key-ordered union of
the owners' results.  Here:

* kc_merge_results (host code of the library) against numpy on disjoint runs,
  one and two samples, many threads, and its refusals (overlapping or
  unsorted runs);
* the shard ranges that owned_shards hands to the ranks tile the hash space;
* the arguments kc_create_ex refuses before touching a GPU;
* two gloo ranks on the CPU, each counting its owned range with the oracle
  (restricted to those hash shards), gathering the results and merging them
  with kc_merge_results: the merge equals the unrestricted oracle's result,
  and the owners' filters OR to the whole filter.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

import paper_1712_03254_gb300 as kc


def _disjoint_runs(rng, n_runs, n_keys, n_samples):
    keys = np.unique(rng.integers(0, 1 << 62, size=n_keys, dtype=np.uint64))
    owner = rng.integers(0, n_runs, size=keys.size)
    counts = rng.integers(1, 1 << 31, size=(keys.size, n_samples), dtype=np.uint32)
    runs = [(keys[owner == r], counts[owner == r]) for r in range(n_runs)]
    return runs, keys, counts


@pytest.mark.parametrize("n_runs,n_keys,n_samples", [(1, 10, 1), (2, 1000, 1), (4, 5000, 2), (8, 3_000_000, 2)])
def test_merge_results_equals_sorted_union(n_runs, n_keys, n_samples):
    rng = np.random.default_rng(n_runs * 7 + n_samples)
    runs, keys, counts = _disjoint_runs(rng, n_runs, n_keys, n_samples)
    got_k, got_c = kc.merge_results(runs, n_samples)
    assert np.array_equal(got_k, keys)
    assert np.array_equal(got_c, counts)


def test_merge_results_empty_and_single_empty_runs():
    e = (np.zeros(0, np.uint64), np.zeros((0, 1), np.uint32))
    k, c = kc.merge_results([e, e], 1)
    assert k.size == 0 and c.shape == (0, 1)
    k, c = kc.merge_results([e, (np.array([3, 4], np.uint64), np.array([[1], [2]], np.uint32))], 1)
    assert list(k) == [3, 4] and list(c[:, 0]) == [1, 2]


def test_merge_results_refuses_overlap_and_disorder():
    a = (np.array([1, 5, 9], np.uint64), np.ones((3, 1), np.uint32))
    b = (np.array([2, 5], np.uint64), np.ones((2, 1), np.uint32))
    with pytest.raises(kc.KcError, match="two runs"):
        kc.merge_results([a, b], 1)
    c = (np.array([7, 3], np.uint64), np.ones((2, 1), np.uint32))
    with pytest.raises(kc.KcError, match="ascending"):
        kc.merge_results([a, c], 1)
    # the duplicate straddling the threads' key ranges is still found
    rng = np.random.default_rng(5)
    runs, keys, _ = _disjoint_runs(rng, 4, 2_000_000, 1)
    k0, c0 = runs[0]
    dup = keys[keys.size // 2]
    if dup not in k0:
        k0 = np.sort(np.append(k0, dup))
        c0 = np.ones((k0.size, 1), np.uint32)
    runs[0] = (k0, c0)
    with pytest.raises(kc.KcError, match="two runs"):
        kc.merge_results(runs, 1)


@pytest.mark.parametrize("own_bits,world", [(1, 1), (1, 2), (6, 2), (6, 3), (6, 4), (6, 8), (4, 16)])
def test_owned_shards_tile_the_hash_space(own_bits, world):
    ranges = [kc.owned_shards(r, world, own_bits) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == 1 << own_bits
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a < b
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_owned_shards_rejects_more_ranks_than_shards():
    with pytest.raises(ValueError):
        kc.owned_shards(0, 3, 1)


@pytest.mark.parametrize("fields", [
    dict(own_bits=7, own_lo=0, own_hi=1, part_bits=6),       # more shard bits than partition bits
    dict(own_bits=2, own_lo=2, own_hi=2),                    # empty range
    dict(own_bits=2, own_lo=1, own_hi=5),                    # past the last shard
    dict(own_bits=0, own_lo=1, own_hi=2),                    # a range without shard bits
    dict(own_bits=2, own_lo=0, own_hi=1, strategy=1),        # the direct strategy has no partitions
])
def test_create_rejects_bad_ownership_before_cuda(fields):
    L = kc.lib()
    cfg = kc.Config()
    L.kc_default_config(ctypes.byref(cfg))
    for k, v in fields.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    assert L.kc_create_ex(31, 1, 1 << 24, 4, 2, ctypes.byref(cfg), None, ctypes.byref(h)) == 1  # KC_ERR_ARG
    assert not h.value


# ---------------------------------------------------------------- two gloo ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


OWN_BITS = 6


def _owner_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth

    w = synth.paired(scale=0.002)  # two samples, the joint table
    lo, hi = kc.owned_shards(rank, world, OWN_BITS)
    o = oracle.count(w, restrict=(OWN_BITS, range(lo, hi)))
    keys, counts = o.result()
    mine = (keys, counts, o.bloom(), o.counted)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        mk, mc = kc.merge_results([(g[0], g[1]) for g in gathered], len(w.samples))
        full = oracle.count(w)
        fk, fc = full.result()
        bloom_or = np.zeros_like(full.bloom())
        for g in gathered:
            bloom_or |= g[2]
        q.put(dict(keys_equal=bool(np.array_equal(mk, fk)), counts_equal=bool(np.array_equal(mc, fc)),
                   bloom_equal=bool(np.array_equal(bloom_or, full.bloom())),
                   counted=sum(g[3] for g in gathered), windows=full.windows, n=int(fk.size),
                   sizes=[int(g[0].size) for g in gathered]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_owners_merge_to_the_whole_result():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_owner_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out["keys_equal"] and out["counts_equal"] and out["bloom_equal"]
    assert out["counted"] == out["windows"]  # every window is counted by exactly one owner
    assert all(s > 0 for s in out["sizes"]) and sum(out["sizes"]) == out["n"]

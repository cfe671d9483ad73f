"""Batched finalize: jobs counted together give the results they give alone.

Several partitioned jobs (different k, sample counts, filter sizes, bits per
key, min_count) are finalized by one kc_batch: one persistent consumer launch
over all their partitions and one replay of the captured sort graph.  Each
job's table and filter must equal the oracle's bit for bit.
"""
import random

import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kc.lib()


def _jobs(seed, n):
    rng = random.Random(seed)
    jobs = []
    for i in range(n):
        G = rng.choice([20_000, 60_000, 150_000])
        g = synth.genome(seed * 100 + i, G)
        n_reads = rng.choice([500, 3000, 12000])
        rs = synth.reads(seed * 100 + i, g, n_reads, 60, 160, 0.01, 0.001)
        k = rng.choice([15, 25, 31])
        samples = [rs] if rng.random() < 0.6 else [rs.slice(0, n_reads // 2), rs.slice(n_reads // 2, n_reads)]
        w = synth.Workload(f"job{i}", samples, k, 1 << rng.choice([18, 20, 22]), rng.choice([3, 4, 4, 6]),
                           rng.choice([1, 2, 3]))
        jobs.append(w)
    return jobs


def _counter(w, **kw):
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", **kw)
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    return c


def _check(c, o):
    gk, gc = c.dump()
    ok, oc = o.result()
    assert np.array_equal(gk, ok)
    assert np.array_equal(gc, oc)
    assert np.array_equal(c.export_bloom(), o.bloom())


def test_batch_equals_oracle_and_alone(oracle_mod):
    jobs = _jobs(7, 6)
    oracles = [oracle_mod.count(w) for w in jobs]
    counters = [_counter(w) for w in jobs]
    b = kc.KcBatch()
    b.finalize(counters)
    for c, o in zip(counters, oracles):
        _check(c, o)
    # each alone, through kc_finalize (a batch of one)
    for w, o in zip(jobs, oracles):
        c = _counter(w)
        c.finalize()
        _check(c, o)


def test_batch_object_reused_across_batches(oracle_mod):
    b = kc.KcBatch()
    for seed, n in ((11, 2), (12, 5), (13, 1), (14, 8)):
        jobs = _jobs(seed, n)
        counters = [_counter(w) for w in jobs]
        b.finalize(counters)
        for c, w in zip(counters, jobs):
            _check(c, oracle_mod.count(w))
        # handles go on: reset and count again alone
        for c, w in zip(counters, jobs):
            c.reset()
            for s, rs in enumerate(w.samples):
                c.add_readset(s, rs)
            c.finalize()
            _check(c, oracle_mod.count(w))


def test_uniform_bits_per_key_batch(oracle_mod):
    jobs = _jobs(21, 4)
    for w in jobs:
        w.n_hashes = 4
    counters = [_counter(w) for w in jobs]
    kc.KcBatch().finalize(counters)
    for c, w in zip(counters, jobs):
        _check(c, oracle_mod.count(w))


def test_batch_mixes_split_fallback_and_plain_jobs(oracle_mod):
    """1024-slot tables and few partitions: some jobs' partitions are counted
    as sub-ranges (each job learning its own split level), one job falls back
    to global tables, small jobs need neither; one launch serves them all."""
    jobs = _jobs(31, 6)
    # filters of 2^18, 2^18, 2^22, 2^18, 2^22, 2^22 bits (slices of at most 2^13 words)
    kws = [dict(part_bits=1, smem_table_log2=10), dict(part_bits=2, smem_table_log2=10),
           dict(part_bits=3, smem_table_log2=10, split_max=-1), dict(part_bits=3, smem_table_log2=11),
           dict(), dict(part_bits=3, smem_table_log2=10, split_max=2)]
    counters = [_counter(w, **kw) for w, kw in zip(jobs, kws)]
    kc.KcBatch().finalize(counters)
    for c, w in zip(counters, jobs):
        _check(c, oracle_mod.count(w))
    st = [c.stats() for c in counters]
    assert sum(x["split_partitions"] for x in st) > 0
    assert st[2]["split_partitions"] == 0


def test_batch_rejects_bad_lists():
    w = _jobs(31, 1)[0]
    c = _counter(w)
    d = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, strategy="direct")
    b = kc.KcBatch()
    with pytest.raises(kc.KcError) as e:
        b.finalize([c, c])
    assert e.value.name == "KC_ERR_ARG"
    with pytest.raises(kc.KcError) as e:
        b.finalize([c, d])
    assert e.value.name == "KC_ERR_ARG"
    b.finalize([c])
    with pytest.raises(kc.KcError) as e:
        b.finalize([c])
    assert e.value.name == "KC_ERR_STATE"

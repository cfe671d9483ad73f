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


def _counter_batches(w, n_batches, **kw):
    """A counter fed each sample in n_batches kc_add_reads calls."""
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", **kw)
    for s, rs in enumerate(w.samples):
        cuts = np.linspace(0, rs.n_reads, n_batches + 1).astype(int)
        for a, b in zip(cuts[:-1], cuts[1:]):
            c.add_readset(s, rs.slice(a, b))
    return c


def test_batched_ingest_equals_oracle(oracle_mod):
    """kc_config.batched_ingest: kc_add_reads keeps the reads and the batch's
    finalize extracts and groups every job's batches in one launch per phase
    (mixed k, samples, partition bits -- one job with two grouping levels --
    and several kc_add_reads calls per sample); each job equals the oracle."""
    jobs = _jobs(41, 6)
    kws = [dict(), dict(part_bits=14), dict(part_bits=5), dict(), dict(part_bits=1), dict()]
    counters = [_counter_batches(w, 1 + i % 3, batched_ingest=True, **kw) for i, (w, kw) in enumerate(zip(jobs, kws))]
    kc.KcBatch().finalize(counters)
    for c, w in zip(counters, jobs):
        o = oracle_mod.count(w)
        _check(c, o)
        assert c.stats()["windows"] == o.windows


def test_batched_ingest_alone_mixed_and_reused(oracle_mod):
    """A batched-ingest job finalized alone (kc_finalize), a batch mixing
    batched-ingest jobs with jobs grouped at kc_add_reads, and a handle reset
    and reused: all equal the oracle."""
    jobs = _jobs(43, 5)
    w = jobs[0]
    c = _counter_batches(w, 2, batched_ingest=True)
    c.finalize()
    _check(c, oracle_mod.count(w))
    counters = [_counter_batches(x, 2, batched_ingest=(i % 2 == 0)) for i, x in enumerate(jobs)]
    kc.KcBatch().finalize(counters)
    for cc, x in zip(counters, jobs):
        _check(cc, oracle_mod.count(x))
    # the handle reset and fed again
    c.reset()
    for s, rs in enumerate(w.samples):
        cuts = np.linspace(0, rs.n_reads, 3).astype(int)
        for a, b in zip(cuts[:-1], cuts[1:]):
            c.add_readset(s, rs.slice(a, b))
    c.finalize()
    _check(c, oracle_mod.count(w))


def test_batched_ingest_owned_ranges(oracle_mod):
    """Batched ingest of handles owning hash ranges of the same reads: their
    merged results equal the oracle's, their filters OR to its filter."""
    w = _jobs(47, 1)[0]
    o = oracle_mod.count(w)
    counters = []
    for r in range(3):
        lo, hi = kc.owned_shards(r, 3, 4)
        counters.append(_counter_batches(w, 2, batched_ingest=True, own_bits=4, own_lo=lo, own_hi=hi))
    kc.KcBatch().finalize(counters)
    runs = [c.dump() for c in counters]
    keys, counts = kc.merge_results(runs, len(w.samples))
    ok, oc = o.result()
    assert np.array_equal(keys, ok)
    assert np.array_equal(counts, oc)
    bloom = np.zeros_like(o.bloom())
    for c in counters:
        bloom |= c.export_bloom()
    assert np.array_equal(bloom, o.bloom())
    assert sum(c.stats()["owned_windows"] for c in counters) == o.windows


def test_batch_ingest_then_finalize(oracle_mod):
    """kc_batch_ingest on one batch object groups the kept reads of every
    job (no wait for the device); a second batch object finalizes them, as
    the server's extract and finalize threads do."""
    jobs = _jobs(53, 4)
    counters = [_counter_batches(w, 2, batched_ingest=True) for w in jobs]
    ext, fin = kc.KcBatch(), kc.KcBatch()
    ext.ingest(counters + [_counter_batches(jobs[0], 1)])  # a handle grouped at kc_add_reads is left alone
    ext.ingest(counters)  # nothing kept any more: no work
    fin.finalize(counters)
    for c, w in zip(counters, jobs):
        _check(c, oracle_mod.count(w))
    with pytest.raises(kc.KcError) as e:
        ext.ingest([counters[0], counters[0]])
    assert e.value.name == "KC_ERR_ARG"


def test_kept_result_arrays_too_short_or_fallback(oracle_mod):
    """A handle keeps its result arrays across kc_reset, and the next job's
    sort runs right behind its consumer into them: a larger job finds them
    too short and is sorted again into larger ones; a job whose partitions
    overflow their tables (1024 slots) falls back after the early sort; a
    smaller job fits.  Every result equals the oracle's."""
    g = synth.genome(81, 150_000)
    small = synth.reads(81, g, 2_000, 100, 150, 0.01, 0.001)
    big = synth.reads(82, g, 20_000, 100, 150, 0.01, 0.001)
    ws = [synth.Workload(n, [r], k=25, bloom_bits=1 << 22, n_hashes=4, min_count=2)
          for n, r in (("small", small), ("big", big), ("small-again", small))]
    c = kc.KmerCounter(25, 1, 1 << 22, 4, 2, strategy="partitioned")
    for w in ws:
        c.reset()
        c.add_readset(0, w.samples[0])
        c.finalize()
        _check(c, oracle_mod.count(w))
    # 2^18-bit filters in 4 partitions (slices of 1024 words), 1024-slot tables, no splits
    wf = [synth.Workload(n, [r], k=25, bloom_bits=1 << 18, n_hashes=4, min_count=2)
          for n, r in (("small", small), ("big", big))]
    d = kc.KmerCounter(25, 1, 1 << 18, 4, 2, strategy="partitioned", part_bits=2, smem_table_log2=10, split_max=-1)
    for w in wf:
        d.reset()
        d.add_readset(0, w.samples[0])
        d.finalize()
        _check(d, oracle_mod.count(w))
    assert d.stats()["fallback_partitions"] > 0

"""GPU parity of hash-range ownership and of the device-budget spill.

Ownership (kc_config.own_bits): N handles over the same reads, each owning a
contiguous range of 2^own_bits hash shards, are run one after another on
one GPU.  Their results, merged by key (kc_merge_results), must equal the
oracle's result bit for bit, their filters must OR to the oracle's filter and
each must hold only its own filter slice, and their owned windows must add up
to the job's windows.

Device budget (kc_config.device_budget): a budget too small for the window
hashes makes kc_add_reads keep the packed reads, and kc_finalize extract them
again one hash range at a time, spilling each range's sorted result to pinned
host memory; the result and filter must still equal the oracle's.
"""
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
    torch.cuda.init()
    kc.lib()


def _count(w, batches=1, **kw):
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", **kw)
    for s, rs in enumerate(w.samples):
        cuts = np.linspace(0, rs.n_reads, batches + 1).astype(int)
        for a, b in zip(cuts[:-1], cuts[1:]):
            c.add_readset(s, rs.slice(a, b))
    c.finalize()
    return c


def _owners_parity(w, o, n_owners, own_bits, **kw):
    ok, oc = o.result()
    ob = o.bloom()
    n_words = w.bloom_bits // 64
    results, bloom_or, owned = [], np.zeros_like(ob), 0
    for r in range(n_owners):
        lo, hi = kc.owned_shards(r, n_owners, own_bits)
        c = _count(w, own_bits=own_bits, own_lo=lo, own_hi=hi, **kw)
        keys, counts = c.dump()
        # every key of the owner lies in its shard range
        if keys.size:
            import oracle

            shards = oracle.partitions(keys, own_bits)
            assert shards.min() >= lo and shards.max() < hi
        results.append((keys.copy(), counts.copy()))
        f = c.export_bloom()
        w0, w1 = lo * n_words >> own_bits, hi * n_words >> own_bits
        assert np.array_equal(f[w0:w1], ob[w0:w1])  # its slice is the oracle's
        assert not f[:w0].any() and not f[w1:].any()  # nothing outside it
        bloom_or |= f
        st = c.stats()
        assert st["windows"] == o.windows  # every owner scans every window
        owned += st["owned_windows"]
        c.close()
    mk, mc = kc.merge_results(results, len(w.samples))
    assert np.array_equal(mk, ok)
    assert np.array_equal(mc, oc)
    assert np.array_equal(bloom_or, ob)
    assert owned == o.windows


@pytest.mark.parametrize("n_owners", [2, 4])
def test_owners_with_library_partition_bits(oracle_mod, n_owners):
    """Owners of 2^2 shards whose partitions the library raises from 4 to 64
    at their first kc_add_reads (a 2^20-bit filter, tiny's 1.4 M windows):
    each owner's partition range follows, and the merge is the oracle's."""
    w = synth.tiny()
    w.bloom_bits = 1 << 20
    o = oracle_mod.count(w)
    c = _count(w, own_bits=2, own_lo=0, own_hi=1)
    assert c.stats()["partitions"] == 64
    c.close()
    _owners_parity(w, o, n_owners, own_bits=2)


@pytest.mark.parametrize("n_owners", [2, 4])
def test_owners_merge_to_the_oracle_tiny(oracle_mod, n_owners):
    w = synth.tiny(scale=0.5)
    o = oracle_mod.count(w)
    _owners_parity(w, o, n_owners, own_bits=6, batches=2)


@pytest.mark.parametrize("n_owners", [2, 4])
def test_owners_two_samples_two_levels(oracle_mod, n_owners):
    """Joint table of two samples; 14 partition bits (two grouping levels), so an owner's range covers
    whole first-level groups (two owners) or one group (four)."""
    w = synth.paired(scale=0.002)
    w.bloom_bits = 1 << 28
    o = oracle_mod.count(w)
    _owners_parity(w, o, n_owners, own_bits=3, part_bits=14)


@pytest.mark.parametrize("spill", [1, 2])
def test_owners_with_spill(oracle_mod, spill):
    w = synth.paired(scale=0.002)
    w.bloom_bits = 1 << 28
    o = oracle_mod.count(w)
    _owners_parity(w, o, 3, own_bits=6, part_bits=10, spill=spill)


def test_owner_of_one_shard_with_no_key_in_it(oracle_mod):
    """An owner whose range holds no window: empty result, zero filter."""
    reads = ["ACGTACGTACGTACGTACGTACGTACGTACGTACG"] * 3
    w = synth.Workload("one", [synth.ReadSet.from_strings(reads)], 31, 1 << 16, 4, 1)
    o = oracle_mod.count(w)
    ok, _ = o.result()
    import oracle

    used = set(oracle.partitions(ok, 6).tolist())
    empty = next(s for s in range(64) if s not in used)
    c = _count(w, own_bits=6, own_lo=empty, own_hi=empty + 1, part_bits=6)
    keys, _ = c.dump()
    assert keys.size == 0
    assert not c.export_bloom().any()
    assert c.stats()["owned_windows"] == 0


# ---------------------------------------------------------------- device budget


def _budget_parity(w, o, budget, batches=1, **kw):
    c = _count(w, batches=batches, device_budget=budget, **kw)
    st = c.stats()
    ok, oc = o.result()
    keys, counts = c.dump()
    assert np.array_equal(keys, ok)
    assert np.array_equal(counts, oc)
    assert np.array_equal(c.export_bloom(), o.bloom())
    assert st["windows"] == o.windows
    return c, st


@pytest.mark.parametrize("spill", [0, 2])
def test_small_budget_keeps_reads_and_groups_by_range(oracle_mod, spill):
    w = synth.tiny(scale=0.5)
    o = oracle_mod.count(w)
    budget = w.bloom_bits // 8 + (4 << 20)  # the filter and 4 MiB
    c, st = _budget_parity(w, o, budget, batches=3, spill=spill)
    assert st["deferred_batches"] == 3
    assert st["scan_groups"] > 1
    assert st["spilled_bytes"] == 16 * st["result_keys"] > 0


def test_budget_passed_midway_mixes_grouped_and_kept_batches(oracle_mod):
    """The first batches' hashes fit, the later ones are kept as reads."""
    w = synth.paired(scale=0.002)
    w.bloom_bits = 1 << 26
    o = oracle_mod.count(w)
    batch_bases = sum(rs.n_bases for rs in w.samples) // 8
    budget = w.bloom_bits // 8 + 3 * 16 * batch_bases  # linear + grouped hashes (16 B/base) of three batches
    c, st = _budget_parity(w, o, budget, batches=4, part_bits=8)
    assert 0 < st["deferred_batches"] < 8


def test_budget_with_owner(oracle_mod):
    w = synth.tiny(scale=0.5)
    o = oracle_mod.count(w)
    ok, oc = o.result()
    results, bloom_or = [], np.zeros_like(o.bloom())
    for r in range(2):
        lo, hi = kc.owned_shards(r, 2, 6)
        c = _count(w, batches=2, own_bits=6, own_lo=lo, own_hi=hi, device_budget=w.bloom_bits // 8 + (2 << 20))
        assert c.stats()["deferred_batches"] == 2
        k, cnt = c.dump()
        results.append((k.copy(), cnt.copy()))
        bloom_or |= c.export_bloom()
        c.close()
    mk, mc = kc.merge_results(results, 1)
    assert np.array_equal(mk, ok) and np.array_equal(mc, oc)
    assert np.array_equal(bloom_or, o.bloom())


def test_budget_reuse_after_reset(oracle_mod):
    w = synth.tiny(scale=0.3)
    o = oracle_mod.count(w)
    c = _count(w, device_budget=w.bloom_bits // 8 + (2 << 20))
    for _ in range(2):
        c.reset()
        for s, rs in enumerate(w.samples):
            c.add_readset(s, rs)
        c.finalize()
        ok, oc = o.result()
        keys, counts = c.dump()
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
        assert np.array_equal(c.export_bloom(), o.bloom())

"""GPU parity of the Prune chain (kc_config.prune_chain): the counting result
and the first filter bit for bit against the oracle, the second filter
between the oracle's bounds (its content depends on the order in which
concurrent windows reach the first filter)."""
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
    torch.cuda.init()
    kc.lib()


def chain_count(w, **kw):
    kw.setdefault("table_slots", w.table_slots)
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, prune_chain=True, **kw)
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    c.finalize()
    return c


def assert_chain_matches(c, o):
    gk, gc = c.dump()
    ok, oc = o.result()
    assert np.array_equal(gk, ok) and np.array_equal(gc, oc)
    bf1 = c.export_bloom()
    assert np.array_equal(bf1, o.bloom())
    bf2 = c.export_bloom2()
    lo, hi = o.bloom2_bounds()
    assert not np.any(lo & ~bf2), "a key seen twice is missing from the second filter"
    assert not np.any(bf2 & ~hi), "the second filter holds bits no insertion order can give"
    return bf2


def test_chain_tiny(oracle_mod):
    w = synth.tiny()
    o = oracle_mod.count(w)
    c = chain_count(w)
    assert c.stats()["strategy"] == 1  # direct
    bf2 = assert_chain_matches(c, o)
    assert bf2.any()


def test_chain_two_samples(oracle_mod):
    w = synth.paired(scale=0.002)
    o = oracle_mod.count(w)
    assert_chain_matches(chain_count(w, table_slots=1 << 20), o)


@pytest.mark.parametrize("k", [5, 16, 25, 31])
@pytest.mark.parametrize("min_count", [1, 2, 3])
def test_chain_ragged_reads(oracle_mod, k, min_count):
    rng = random.Random(1000 + 10 * k + min_count)
    reads = ["".join("N" if rng.random() < 0.01 else rng.choice("ACGT") for _ in range(rng.randint(0, 300)))
             for _ in range(800)]
    w = synth.Workload("ragged", [synth.ReadSet.from_strings(reads)], k, 1 << 18, 4, min_count)
    o = oracle_mod.count(w)
    assert_chain_matches(chain_count(w, table_slots=1 << 18), o)


def test_chain_small_filter_false_positives(oracle_mod):
    """A 4096-bit filter for ~135,000 distinct keys: most singletons are false
    positives of the first filter and reach the second one; the count pass
    counts them and the compaction drops them."""
    w = synth.tiny(scale=0.1)
    w.bloom_bits = 4096
    o = oracle_mod.count(w)
    c = chain_count(w, table_slots=1 << 19)
    bf2 = assert_chain_matches(c, o)
    st = c.stats()
    assert st["table_keys"] > 2 * st["result_keys"]  # false positives were counted, then dropped
    assert bin(int(np.bitwise_or.reduce(bf2))).count("1") > 0


def test_chain_reset_and_errors(oracle_mod):
    w = synth.tiny(scale=0.2)
    o = oracle_mod.count(w)
    c = chain_count(w)
    for _ in range(2):
        c.reset()
        for s, rs in enumerate(w.samples):
            c.add_readset(s, rs)
        c.finalize()
        assert_chain_matches(c, o)
    plain = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy="direct")
    with pytest.raises(kc.KcError) as e:
        plain.export_bloom2()
    assert e.value.name == "KC_ERR_STATE"


def test_chain_mid_full_size(oracle_mod):
    """mid at full size (1,000,000 reads) through the chain: four of 64 hash
    partitions against the restricted oracle, every result key's pattern in
    the second filter, the second filter inside the first."""
    w = synth.mid()
    q, parts = 6, [0, 17, 42, 63]
    o = oracle_mod.count(w, restrict=(q, parts))
    c = chain_count(w)
    gk, gc = c.dump()
    sel = np.isin(oracle_mod.partitions(gk, q), parts)
    ok, oc = o.result()
    assert np.array_equal(gk[sel], ok) and np.array_equal(gc[sel], oc)
    bf1, bf2 = c.export_bloom(), c.export_bloom2()
    assert not np.any(bf2 & ~bf1)
    for key in gk[:: max(1, gk.size // 2000)]:
        wi, p = o.bloom_word_index(int(key)), o.bloom_pattern(int(key))
        assert int(bf2[wi]) & p == p
    assert c.stats()["windows"] == o.windows

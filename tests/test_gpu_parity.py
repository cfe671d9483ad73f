"""GPU parity: libkc through its C ABI against the CPU oracle, bit for bit.

Count tables (keys and per-sample counts) and Bloom filter words must match
the oracle exactly: everything on this path is integer work.
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
    torch.cuda.init()
    kc.lib()


STRATEGIES = ["direct", "partitioned"]


@pytest.fixture(params=STRATEGIES)
def strategy(request):
    return request.param


def gpu_count(w, batches=1, **kw):
    kw.setdefault("table_slots", w.table_slots)
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, **kw)
    for s, rs in enumerate(w.samples):
        if batches == 1:
            c.add_readset(s, rs)
        else:
            cuts = np.linspace(0, rs.n_reads, batches + 1).astype(int)
            for a, b in zip(cuts[:-1], cuts[1:]):
                c.add_readset(s, rs.slice(a, b))
    c.finalize()
    return c


def assert_same_result(c, o):
    gk, gc = c.dump()
    ok, oc = o.result()
    assert gk.shape == ok.shape, (gk.shape, ok.shape)
    assert np.array_equal(gk, ok)
    assert np.array_equal(gc, oc)


def assert_same_bloom(c, o):
    assert np.array_equal(c.export_bloom(), o.bloom())


def test_tiny_full_parity(oracle_mod, strategy):
    """20,000 x 100 bp reads, k=31, 2^24-bit filter, 4 hashes, min_count 2."""
    w = synth.tiny()
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    st = c.stats()
    assert st["windows"] == o.windows
    assert st["result_keys"] == len(o.result()[0])


@pytest.mark.parametrize("k", [1, 2, 5, 8, 16, 25, 31])
@pytest.mark.parametrize("min_count", [1, 2, 3])
def test_ragged_random_reads(oracle_mod, k, min_count, strategy):
    """Read lengths 0..300 (shorter than k, exactly k, across word boundaries), 2 % N."""
    rng = random.Random(31 * k + min_count)
    g = "".join(rng.choice("ACGT") for _ in range(3000))
    reads = []
    for _ in range(700):
        L = rng.choice([0, 1, k - 1, k, k + 1, 31, 32, 33, 63, 64, 65, rng.randint(0, 300)])
        L = max(0, min(L, len(g)))
        s = rng.randint(0, len(g) - L)
        r = list(g[s : s + L])
        for i in range(L):
            if rng.random() < 0.02:
                r[i] = "N"
        reads.append("".join(r))
    w = synth.Workload("ragged", [synth.ReadSet.from_strings(reads)], k, 1 << 16, 3, min_count)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 16, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    assert c.stats()["windows"] == o.windows


def test_n_at_every_position(oracle_mod, strategy):
    k = 7
    base = "ACGTTGCAACGTAGGCTAAC"
    reads = [base[:i] + "N" + base[i + 1 :] for i in range(len(base))] + [base, "N" * 40, "NACGTACGN"]
    w = synth.Workload("nmask", [synth.ReadSet.from_strings(reads)], k, 1 << 12, 2, 1)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 12, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_empty_and_degenerate_inputs(oracle_mod, strategy):
    for reads in ([], [""], ["", "", ""], ["ACG"], ["NNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNN"]):
        w = synth.Workload("empty", [synth.ReadSet.from_strings(reads)], 5, 1 << 12, 4, 1)
        o = oracle_mod.count(w)
        c = gpu_count(w, table_slots=1 << 12, strategy=strategy)
        assert_same_result(c, o)
        assert c.result_size() == 0
        assert_same_bloom(c, o)


def test_several_batches_and_offset_base(oracle_mod, strategy):
    """Reads added in uneven batches, with offsets not starting at 0 (unaligned base)."""
    w = synth.tiny(scale=0.2)
    o = oracle_mod.count(w)
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy=strategy)
    rs = w.samples[0]
    packed, mask = kc.pack_ascii(rs.ascii)
    cuts = [0, 1, 7, 500, 1333, 2000, rs.n_reads]
    for a, b in zip(cuts[:-1], cuts[1:]):
        # the whole packed stream is passed; offsets select the batch's reads
        c.add_reads(0, packed, np.ascontiguousarray(rs.offsets[a : b + 1]), mask)
    c.finalize()
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_many_batches_full_recount(oracle_mod):
    """40 read batches per sample: a partition spans more batches than the
    consumer's window bitmap covers, so the second pass recounts every window
    instead of only the first pass's uncounted ones; same result either way."""
    w = synth.paired(scale=0.001)
    o = oracle_mod.count(w)
    c = gpu_count(w, batches=40, strategy="partitioned")
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    c = gpu_count(w, batches=7, strategy="partitioned")
    assert_same_result(c, o)


@pytest.mark.parametrize("n_hashes", [1, 7, 10])
def test_bits_per_key_extremes(oracle_mod, n_hashes, strategy):
    """One and ten filter bits per key (the smallest and largest accepted), and
    an odd count in between: the filter words and the counts."""
    w = synth.tiny(scale=0.3)
    w.n_hashes = n_hashes
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_smallest_filter_many_false_positives(oracle_mod, strategy):
    """A 4096-bit filter (the minimum) for about 136,000 windows: almost every window
    is a candidate, the exact recount still drops every singleton."""
    w = synth.tiny(scale=0.1)
    w.bloom_bits = 1 << 12
    w.table_slots = 1 << 20  # direct: every distinct key becomes a candidate
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy, part_bits=1 if strategy == "partitioned" else 0)
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    assert c.stats()["candidates"] > 0.9 * o.windows


def test_largest_partition_count(oracle_mod):
    """20 partition bits (the maximum: 2^20 partitions in two levels) over a
    2^34-bit filter (2 GiB, slices of 256 words)."""
    w = synth.tiny(scale=0.3)
    w.bloom_bits = 1 << 34
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=20)
    assert c.stats()["partitions"] == 1 << 20
    assert_same_result(c, o)
    nw = w.bloom_bits // 64
    for first in (0, nw // 3, nw - 4096):  # three stretches of the 2^28 filter words
        assert np.array_equal(c.export_bloom(first, 4096), o.bloom(first, 4096))


def test_high_min_count_keeps_nothing(oracle_mod, strategy):
    w = synth.tiny(scale=0.2)
    w.min_count = 1000
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy)
    assert c.result_size() == 0 == len(o.result()[0])
    assert_same_bloom(c, o)


def test_two_samples_joint_table(oracle_mod, strategy):
    w = synth.paired(scale=0.002)
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    gk, gc = c.dump()
    assert gc.shape[1] == 2 and gc[:, 0].sum() > 0 and gc[:, 1].sum() > 0


def test_device_resident_inputs(oracle_mod, strategy):
    torch = pytest.importorskip("torch")
    w = synth.tiny(scale=0.3)
    o = oracle_mod.count(w)
    rs = w.samples[0]
    packed, mask = kc.pack_ascii(rs.ascii)
    dp = torch.from_numpy(packed.view(np.int64)).cuda()
    dm = torch.from_numpy(mask.view(np.int64)).cuda()
    do = torch.from_numpy(rs.offsets.view(np.int64)).cuda()
    torch.cuda.synchronize()
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy=strategy)
    c.add_reads(0, dp, do, dm)
    c.finalize()
    n = c.result_size()
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    counts = torch.empty((n, 1), dtype=torch.int32, device="cuda")
    c.dump(keys, counts)
    ok, oc = o.result()
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
    bloom = torch.empty(w.bloom_bits // 64, dtype=torch.int64, device="cuda")
    c.export_bloom(out=bloom)
    assert np.array_equal(bloom.cpu().numpy().view(np.uint64), o.bloom())


def test_reset_reuses_handle(oracle_mod, strategy):
    w = synth.tiny(scale=0.25)
    o = oracle_mod.count(w)
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy=strategy)
    for _ in range(3):
        c.add_readset(0, w.samples[0])
        c.finalize()
        assert_same_result(c, o)
        assert_same_bloom(c, o)
        c.reset()


def test_errors_are_reported_not_faulted(oracle_mod):
    w = synth.tiny(scale=0.2)
    # table far too small: probes are bounded, the job reports KC_ERR_CAPACITY
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, table_slots=1024, strategy="direct")
    c.add_readset(0, w.samples[0])
    with pytest.raises(kc.KcError) as e:
        c.finalize()
    assert e.value.name == "KC_ERR_CAPACITY"
    with pytest.raises(kc.KcError) as e:
        c.finalize()
    assert e.value.name == "KC_ERR_STATE"
    c.reset()
    c.close()
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count)
    # decreasing offsets are rejected on the host
    packed, mask = kc.pack_ascii(np.frombuffer(b"ACGT" * 40, dtype=np.uint8))
    with pytest.raises(kc.KcError) as e:
        c.add_reads(0, packed, np.array([0, 100, 50, 160], dtype=np.uint64), mask)
    assert e.value.name == "KC_ERR_ARG"
    # dump before finalize, and into a buffer that is too small
    with pytest.raises(kc.KcError):
        c.dump()
    c.add_readset(0, w.samples[0])
    c.finalize()
    n = c.result_size()
    assert n > 10
    with pytest.raises(kc.KcError) as e:
        c.dump(np.empty(n - 1, dtype=np.uint64), np.empty((n - 1, 1), dtype=np.uint32))
    assert e.value.name == "KC_ERR_CAPACITY"


def library_part_bits(bloom_bits, bases, reads, k):
    """The partition bits the library picks when kc_config.part_bits is 0, as
    include/kc.h states the rule: slices of 4096 filter words, or more
    partitions, up to 2^12 and slices of at least 8 words, for at most 32768
    windows (bases - reads * (k - 1)) each."""
    lw = (bloom_bits // 64).bit_length() - 1
    base = min(20, max(1, lw - 12))
    est = max(0, bases - reads * (k - 1))
    want = 0
    while want < 12 and (est >> want) > 32768:
        want += 1
    return max(base, min(want, lw - 3))


def test_library_partition_bits_follow_the_windows(oracle_mod):
    """part_bits left to the library: a 2^20-bit filter alone gives 4
    partitions of 4096 words, but tiny's 1.4 M windows take 64 partitions of at
    most 32768 windows, which the first kc_add_reads sets; after a reset a job
    of 1,000 reads is back at 4.  Both results and filters are the oracle's."""
    w = synth.tiny()
    w.bloom_bits = 1 << 20
    rs = w.samples[0]
    o = oracle_mod.count(w)
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned")
    assert c.stats()["partitions"] == 4
    c.add_readset(0, rs)
    c.finalize()
    pb = library_part_bits(w.bloom_bits, rs.n_bases, rs.n_reads, w.k)
    assert pb == 6
    assert c.stats()["partitions"] == 1 << pb
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    small = synth.Workload("tiny_1000", [rs.slice(0, 1000)], k=w.k, bloom_bits=w.bloom_bits, n_hashes=w.n_hashes,
                           min_count=w.min_count)
    o2 = oracle_mod.count(small)
    c.reset()
    c.add_readset(0, small.samples[0])
    c.finalize()
    assert c.stats()["partitions"] == 4
    assert_same_result(c, o2)
    assert_same_bloom(c, o2)
    # the first call decides: a second one adds to the partitions already chosen
    c.reset()
    c.add_readset(0, rs.slice(0, 1000))
    c.add_readset(0, rs.slice(1000, rs.n_reads))
    c.finalize()
    assert c.stats()["partitions"] == 4
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    c.close()


def test_partition_fallback_matches(oracle_mod):
    """With splitting switched off, two partitions with 1024-slot shared-memory
    tables cannot hold tiny's candidates: every partition takes the
    global-memory fallback."""
    w = synth.tiny(scale=0.5)
    w.bloom_bits = 1 << 20  # 2 partitions of 8192 filter words
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=1, smem_table_log2=10, split_max=-1)
    st = c.stats()
    assert st["fallback_partitions"] == 2 and st["split_partitions"] == 0
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    # sixteen partitions of about 6,100 candidates each, 4096-slot tables
    c = gpu_count(w, strategy="partitioned", part_bits=4, smem_table_log2=12, split_max=-1)
    assert c.stats()["fallback_partitions"] == 16
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_overflowing_partitions_split(oracle_mod):
    """Sixteen partitions of about 6,100 candidates, 4096-slot tables: each is
    counted as sub-ranges of its filter slice in shared memory, none falls
    back, and the result and filter are the oracle's."""
    w = synth.tiny(scale=0.5)
    w.bloom_bits = 1 << 20
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=4, smem_table_log2=12)
    st = c.stats()
    assert st["fallback_partitions"] == 0
    assert st["split_partitions"] == 16 and st["split_level"] >= 1
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    # two partitions of about 49,000 candidates, 1024-slot tables: down to 64 sub-ranges
    c = gpu_count(w, strategy="partitioned", part_bits=1, smem_table_log2=10)
    st = c.stats()
    assert st["split_partitions"] + st["fallback_partitions"] == 2 and st["split_level"] >= 5
    assert_same_result(c, o)
    assert_same_bloom(c, o)


@pytest.mark.parametrize("split_max", [1, 2, 3])
def test_split_then_fallback_for_the_rest(oracle_mod, split_max):
    """Splitting capped below what the candidates need: the sub-ranges that
    fit are finished in shared memory, the rest of the partition (from its
    first unfinished sub-range on) goes to the global table; nothing is
    counted twice."""
    w = synth.tiny(scale=0.5)
    w.bloom_bits = 1 << 20
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=1, smem_table_log2=13, split_max=split_max)
    st = c.stats()
    assert st["fallback_partitions"] + st["split_partitions"] == 2
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_finished_sub_range_then_fallback(oracle_mod):
    """Keys chosen by hash: partition 0 holds 200 keys in its first half-slice
    and 10,000 in its second, more than an 8192-slot table takes.  With one
    split level the first half is finished in shared memory and only the
    second half goes to the global table."""
    rng = random.Random(77)
    lo, hi = [], []
    while len(lo) < 200 or len(hi) < 10_000:
        s = "".join(rng.choice("ACGT") for _ in range(31))
        h = oracle_mod.mixer64(oracle_mod.canonical(s))
        if h >> 63:  # partition 1 stays empty
            continue
        side, cap = (hi, 10_000) if (h >> 62) & 1 else (lo, 200)
        if len(side) < cap:
            side.append(s)
    reads = lo + hi + lo + hi  # every key twice
    w = synth.Workload("split_half", [synth.ReadSet.from_strings(reads)], k=31, bloom_bits=1 << 20, n_hashes=4,
                       min_count=2)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=0, strategy="partitioned", part_bits=1, smem_table_log2=13, split_max=1)
    st = c.stats()
    assert st["fallback_partitions"] == 1
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    assert c.result_size() == 10_200


def test_split_two_samples(oracle_mod):
    """Per-sample counts of split partitions (tumour/normal pair)."""
    w = synth.paired(scale=0.002)
    w.bloom_bits = 1 << 22
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=3, smem_table_log2=10, batches=2)  # slices of 2^13 words
    assert c.stats()["split_partitions"] > 0
    assert_same_result(c, o)
    assert_same_bloom(c, o)


@pytest.mark.parametrize("part_bits", [5, 8, 10, 14])
def test_partition_counts(oracle_mod, part_bits):
    w = synth.tiny(scale=0.3)
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=part_bits)
    assert c.stats()["partitions"] == 1 << part_bits
    assert_same_result(c, o)
    assert_same_bloom(c, o)


def test_mid_full_size_sampled_partitions(oracle_mod, strategy):
    """1,000,000 x 150 bp, 2^30-bit filter, 2^24 slots: the configuration the
    benchmark times.  The oracle counts four of 64 hash partitions in full;
    the GPU result restricted to them, and their filter words, must match."""
    w = synth.mid()
    q, parts = 6, [0, 17, 42, 63]
    o = oracle_mod.count(w, restrict=(q, parts))
    c = gpu_count(w, strategy=strategy)
    gk, gc = c.dump()
    sel = np.isin(oracle_mod.partitions(gk, q), parts)
    ok, oc = o.result()
    assert np.array_equal(gk[sel], ok)
    assert np.array_equal(gc[sel], oc)
    assert np.all(np.diff(gk.astype(np.uint64)) > 0)  # strictly ascending everywhere
    nw = w.bloom_bits // 64
    per = nw >> q
    for p in parts:
        assert np.array_equal(c.export_bloom(p * per, per), o.bloom(p * per, per))
    st = c.stats()
    assert st["windows"] == o.windows


@pytest.mark.parametrize("scatter_mode", [1, 2, 3, 4])
@pytest.mark.parametrize("ctas_per_sm", [1, 2])
def test_scatter_modes(oracle_mod, scatter_mode, ctas_per_sm):
    w = synth.tiny(scale=0.5)
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", scatter_mode=scatter_mode, ctas_per_sm=ctas_per_sm)
    assert_same_result(c, o)
    assert_same_bloom(c, o)


@pytest.mark.parametrize("n_reads", [200, 1500, 6000])
def test_skewed_key_prefixes_sort_paths(oracle_mod, n_reads, strategy):
    """Keys sharing a 20-base prefix land in one sort bucket: up to 256 keys
    are sorted by a warp, up to 2048 by a CTA, more in global memory."""
    rng = random.Random(n_reads)
    reads = ["A" * 20 + "".join(rng.choice("ACGT") for _ in range(11)) for _ in range(n_reads)]
    w = synth.Workload("skew", [synth.ReadSet.from_strings(reads)], 31, 1 << 16, 4, 1)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 16, strategy=strategy)
    assert_same_result(c, o)
    assert_same_bloom(c, o)


@pytest.mark.parametrize("part_bits", [13, 16, 18])
def test_two_level_partitions(oracle_mod, part_bits):
    """More than 12 partition bits: hashes are grouped by the top bits at
    ingest and each group re-bucketed by the next 12 bits."""
    w = synth.tiny(scale=0.5)
    w.bloom_bits = 1 << 30  # 2^24 words: slices of at most 2^11 words at 13+ bits
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=part_bits, batches=3)
    assert c.stats()["partitions"] == 1 << part_bits
    assert_same_result(c, o)
    assert_same_bloom(c, o)


@pytest.mark.parametrize("spill", [1, 2])  # dump re-sorts on the device / merges on the host
@pytest.mark.parametrize("part_bits", [10, 16])  # 2^22 filter words: slices of 2^12 and 2^6 words
def test_spill_to_host_merges_runs(oracle_mod, part_bits, spill):
    """Out-of-core finalize: 64 groups of partitions in turn, each group's
    sorted survivors copied to pinned host memory; kc_dump puts the runs back
    in key order (on the device, or merged on the host)."""
    w = synth.paired(scale=0.002)
    w.bloom_bits = 1 << 28
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy="partitioned", part_bits=part_bits, spill=spill)
    st = c.stats()
    assert st["spilled_bytes"] == 16 * st["result_keys"] > 0
    assert_same_result(c, o)
    assert_same_bloom(c, o)
    # dump into device buffers as well
    torch = pytest.importorskip("torch")
    n = c.result_size()
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    counts = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    c.dump(keys, counts)
    ok, oc = o.result()
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), ok)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
    assert c.stats()["spilled_bytes"] == st["spilled_bytes"]
    # the same handle again: the pinned runs are reused
    c.reset()
    for s_i, rs in enumerate(w.samples):
        c.add_readset(s_i, rs)
    c.finalize()
    assert_same_result(c, o)


def test_chunked_host_copies_equal_oracle(oracle_mod):
    """Host reads of at least 2 x 2^15 units (64 bases each) are copied in
    chunks, each chunk's windows extracted as soon as it lands, the offsets
    checked on the device first: the result and filter equal the oracle's
    and those of the same reads given from device memory, with several calls
    and two samples; decreasing offsets are still rejected by the call and
    leave the handle usable."""
    torch = pytest.importorskip("torch")
    g = synth.genome(61, 400_000)
    rs = synth.reads(61, g, 60_000, 100, 160, 0.01, 0.001)  # about 7.8 Mbases: 3 or 4 chunks
    rs2 = synth.reads(62, g, 45_000, 100, 160, 0.01, 0.001)
    w = synth.Workload("chunked", [rs, rs2], k=25, bloom_bits=1 << 24, n_hashes=4, min_count=2)
    o = oracle_mod.count(w)
    ok, oc = o.result()
    c = kc.KmerCounter(w.k, 2, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned")
    c.add_readset(0, rs)
    c.add_readset(1, rs2.slice(0, 20_000))  # below the chunked size: one copy
    c.add_readset(1, rs2.slice(20_000, 45_000))
    c.finalize()
    gk, gc = c.dump()
    assert np.array_equal(gk, ok) and np.array_equal(gc, oc)
    assert np.array_equal(c.export_bloom(), o.bloom())
    assert c.stats()["windows"] == o.windows
    # the same reads from device memory (one copy, no chunks)
    d = kc.KmerCounter(w.k, 2, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned")
    for s, r in enumerate((rs, rs2)):
        packed, mask = kc.pack_ascii(r.ascii)
        offs = np.ascontiguousarray(r.offsets, dtype=np.uint64)
        d.add_reads(s, *(torch.from_numpy(a.view(np.int64)).cuda() for a in (packed, offs, mask)))
    d.finalize()
    dk, dc = d.dump()
    assert np.array_equal(dk, gk) and np.array_equal(dc, gc)
    # decreasing offsets: rejected, nothing added, the handle goes on
    c.reset()
    packed, mask = kc.pack_ascii(rs.ascii)
    bad = np.ascontiguousarray(rs.offsets, dtype=np.uint64).copy()
    bad[30_000] = bad[30_001] + 5
    with pytest.raises(kc.KcError) as e:
        c.add_reads(0, packed, bad, mask)
    assert e.value.name == "KC_ERR_ARG"
    c.add_readset(0, rs)
    c.add_readset(1, rs2)
    c.finalize()
    gk2, gc2 = c.dump()
    assert np.array_equal(gk2, ok) and np.array_equal(gc2, oc)


def test_chunked_host_copies_owned_two_levels(oracle_mod):
    """Chunked host copies with k = 31 (the compile-time-k extraction), two
    grouping levels (14 partition bits) and hash-range owners (the ranged
    extraction adding to its rows chunk by chunk): the owners' merged result
    and OR-ed filters equal the oracle's."""
    g = synth.genome(71, 300_000)
    rs = synth.reads(71, g, 50_000, 120, 160, 0.01, 0.001)  # about 7 Mbases: chunked
    w = synth.Workload("chunked-owned", [rs], k=31, bloom_bits=1 << 26, n_hashes=4, min_count=2)
    o = oracle_mod.count(w)
    ok, oc = o.result()
    runs, bloom = [], np.zeros_like(o.bloom())
    for r in range(2):
        lo, hi = kc.owned_shards(r, 2, 3)
        c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", part_bits=14,
                           own_bits=3, own_lo=lo, own_hi=hi)
        c.add_readset(0, rs)
        c.finalize()
        runs.append(c.dump())
        bloom |= c.export_bloom()
        c.close()
    keys, counts = kc.merge_results(runs, 1)
    assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    assert np.array_equal(bloom, o.bloom())


def test_dump_into_pinned_host_buffers(oracle_mod):
    """kc_dump into pinned host buffers (the counts narrowed straight into
    them by a kernel while the keys are copied) gives the oracle's result;
    one sample and two."""
    torch = pytest.importorskip("torch")
    w = synth.tiny(scale=0.5)
    o = oracle_mod.count(w)
    ok, oc = o.result()
    c = gpu_count(w, strategy="partitioned")
    n = c.result_size()
    keys = torch.empty(n, dtype=torch.int64).pin_memory()
    counts = torch.empty((n, 1), dtype=torch.int32).pin_memory()
    c.dump(keys, counts)
    assert np.array_equal(keys.numpy().view(np.uint64), ok)
    assert np.array_equal(counts.numpy().view(np.uint32), oc)
    w2 = synth.paired(scale=0.002)
    o2 = oracle_mod.count(w2)
    c2 = gpu_count(w2, strategy="partitioned")
    n2 = c2.result_size()
    k2 = torch.empty(n2, dtype=torch.int64).pin_memory()
    n2c = torch.empty((n2, 2), dtype=torch.int32).pin_memory()
    c2.dump(k2, n2c)
    ok2, oc2 = o2.result()
    assert np.array_equal(k2.numpy().view(np.uint64), ok2)
    assert np.array_equal(n2c.numpy().view(np.uint32), oc2)

"""GPU parity of the downstream entry points against the CPU oracle, bit for bit:
16-byte items, joint count spectrum, Filter-unit selection and read hits."""
import random

import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc
from tests import _brute

pytestmark = pytest.mark.gpu

SPECS = [  # (tumor, min_tumor, max_normal, ratio)
    (1, 2, 0, 0),
    (1, 4, 1, 0),
    (0, 2, 0, 0),
    (1, 2, 5, 3),
    (1, 1, 1 << 31, 0),  # every result key
    (1, 1 << 30, 0, 0),  # none
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    kc.lib()


@pytest.fixture(params=["direct", "partitioned"])
def strategy(request):
    return request.param


@pytest.fixture(scope="module")
def paired_small(oracle_mod):
    w = synth.paired(scale=0.002)  # 100 kbp genomes, 2 x 20,000 reads of 150 bp
    return w, oracle_mod.count(w)


def gpu_count(w, **kw):
    kw.setdefault("table_slots", w.table_slots)
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, **kw)
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    c.finalize()
    return c


def test_items_and_spectrum_two_samples(paired_small, strategy):
    w, o = paired_small
    c = gpu_count(w, strategy=strategy)
    items = c.export_items()
    assert items.tobytes() == o.items16().tobytes()
    for cap in (1, 7, 255, 1023):
        assert np.array_equal(c.spectrum(cap), o.spectrum(cap)), cap


def test_items_and_spectrum_one_sample(oracle_mod, strategy):
    w = synth.tiny(scale=0.3)
    o = oracle_mod.count(w)
    c = gpu_count(w, strategy=strategy)
    assert c.export_items().tobytes() == o.items16().tobytes()
    for cap in (1, 50, 1023):
        assert np.array_equal(c.spectrum(cap), o.spectrum(cap))


def test_items_count_clamp(oracle_mod, strategy):
    """A key seen 69,998 times: its 16-bit item count is 65535, the uint32 count is exact."""
    normal = ["A" * 70_000, "ACGTTGCA" * 3]
    tumour = ["AAAC", "ACGTTGCA" * 3, "C" * 40]
    w = synth.Workload("clamp", [synth.ReadSet.from_strings(normal), synth.ReadSet.from_strings(tumour)],
                       3, 1 << 16, 4, 2)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 12, strategy=strategy)
    items = c.export_items()
    assert items.tobytes() == o.items16().tobytes()
    assert items[0]["key"] == 0 and list(items[0]["count"]) == [65535, 1]
    keys, counts = c.dump()
    assert keys[0] == 0 and counts[0, 0] == 69_998


def test_items_and_spectrum_into_device_buffers(paired_small):
    torch = pytest.importorskip("torch")
    w, o = paired_small
    c = gpu_count(w)
    n = c.result_size()
    out = torch.empty(2 * n, dtype=torch.int64, device="cuda")
    c.export_items(out)
    assert out.cpu().numpy().view(np.uint8).tobytes() == o.items16().tobytes()
    hist = torch.empty((64, 64), dtype=torch.int64, device="cuda")
    c.spectrum(63, out=hist)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), o.spectrum(63))
    with pytest.raises(kc.KcError) as e:  # too small a buffer
        c.export_items(out[: n])
    assert e.value.name == "KC_ERR_CAPACITY"


def _check_filter(c, o, w, spec):
    n_sel = c.filter_select(*spec)
    ok, oc = o.filter_select(*spec)
    gk, gc = c.filter_keys()
    assert n_sel == len(ok)
    assert np.array_equal(gk, ok) and np.array_equal(gc, oc)
    for rs in w.samples:
        hits, cand, n_cand = c.filter_readset(rs)
        oh, on = o.filter_reads(rs, *spec)
        assert np.array_equal(hits, oh)
        assert n_cand == on
        assert np.array_equal(cand, np.nonzero(oh)[0].astype(np.uint64))


@pytest.mark.parametrize("spec", SPECS)
def test_filter_parity(paired_small, strategy, spec):
    w, o = paired_small
    c = gpu_count(w, strategy=strategy)
    _check_filter(c, o, w, spec)
    st = c.stats()
    assert st["filter_selected"] == c.filter_keys()[0].size
    assert st["filter_windows"] == o.windows  # both samples rescanned once


def test_filter_parity_large_selection(oracle_mod):
    """Selections of more than 196,608 keys (both orientations above 2^18 x 1.5
    table entries) are probed without the shared-memory prefilter; smaller
    ones with it.  Both give the oracle's hits."""
    w = synth.paired(scale=0.006)  # 300 kbp genomes, 2 x 60,000 reads
    o = oracle_mod.count(w)
    c = gpu_count(w)
    big = (1, 1, 1 << 31, 0)  # every result key
    _check_filter(c, o, w, big)
    assert 2 * c.filter_keys()[0].size > 49152 * 32 // 4
    small = (1, 3, 0, 0)
    _check_filter(c, o, w, small)
    assert 2 * c.filter_keys()[0].size <= 49152 * 32 // 4


def test_filter_reselect_and_other_read_sets(paired_small):
    """A new selection replaces the old one; any read set may be rescanned."""
    w, o = paired_small
    c = gpu_count(w, strategy="partitioned")
    for spec in SPECS[:3]:
        _check_filter(c, o, w, spec)
    other = synth.reads(77, synth.genome(3, 100_000), 3000, 90, 220, 0.01, 0.002)
    hits, cand, n_cand = c.filter_readset(other)
    oh, on = o.filter_reads(other, *SPECS[2])
    assert np.array_equal(hits, oh) and n_cand == on


def test_filter_single_substitution_closed_form(oracle_mod, strategy):
    """One substitution in the tumour genome, reads at every start on both strands:
    the selection is the k windows over it and the hits follow the read geometry."""
    rng = random.Random(2024)
    G, L, k, p = 1200, 60, 21, 600
    normal_g = "".join(rng.choice("ACGT") for _ in range(G))
    alt = rng.choice([b for b in "ACGT" if b != normal_g[p]])
    tumour_g = normal_g[:p] + alt + normal_g[p + 1 :]

    def tiling(g):
        out = []
        for s in range(G - L + 1):
            out += [g[s : s + L], _brute.revcomp_str(g[s : s + L])]
        return out

    samples = [synth.ReadSet.from_strings(tiling(normal_g)), synth.ReadSet.from_strings(tiling(tumour_g))]
    w = synth.Workload("snv", samples, k, 1 << 18, 4, 2)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 16, strategy=strategy)
    assert c.filter_select(1, 2, 0, 0) == k
    keys, counts = c.filter_keys()
    windows = [tumour_g[j : j + k] for j in range(p - k + 1, p + 1)]
    expect = sorted((_brute.as_int(_brute.canonical_str(x)), 2 * (min(j, G - L) - max(0, j + k - L) + 1))
                    for j, x in zip(range(p - k + 1, p + 1), windows))
    assert [int(x) for x in keys] == [a for a, _ in expect]
    assert [int(x) for x in counts[:, 1]] == [b for _, b in expect] and not counts[:, 0].any()
    hits, cand, n_cand = c.filter_readset(samples[1])
    expect_hits = np.repeat([max(0, min(s + L - k, p) - max(s, p - k + 1) + 1) for s in range(G - L + 1)], 2)
    assert np.array_equal(hits, expect_hits.astype(np.uint32))
    assert np.array_equal(hits, o.filter_reads(samples[1], 1, 2, 0, 0)[0])
    hits, cand, n_cand = c.filter_readset(samples[0])
    assert n_cand == 0 and not hits.any() and cand.size == 0


def test_filter_edge_cases(oracle_mod, paired_small):
    w, o = paired_small
    c = gpu_count(w)
    with pytest.raises(kc.KcError) as e:
        c.filter_readset(w.samples[0])
    assert e.value.name == "KC_ERR_STATE"  # before any selection
    with pytest.raises(kc.KcError) as e:
        c.filter_select(2, 1, 0, 0)
    assert e.value.name == "KC_ERR_ARG"
    spec = (1, 2, 0, 0)
    c.filter_select(*spec)
    # no reads, and reads that add no window (shorter than k, all N, empty)
    empty = synth.ReadSet.from_strings([])
    hits, cand, n_cand = c.filter_readset(empty)
    assert hits.size == 0 and n_cand == 0
    short = synth.ReadSet.from_strings(["", "ACGT", "N" * 80, "A" * 30, ""])
    hits, cand, n_cand = c.filter_readset(short)
    assert hits.tolist() == [0] * 5 and n_cand == 0
    # reads whose first base is not at a word boundary, N-heavy
    rs = w.samples[1].slice(37, 3037)
    text = bytearray(rs.ascii.tobytes())
    for i in range(0, len(text), 97):
        text[i] = ord("N")
    lead = b"G" * 45
    ragged = synth.ReadSet(np.frombuffer(lead + bytes(text), dtype=np.uint8).copy(),
                           (rs.offsets + np.uint64(len(lead))).astype(np.uint64))
    hits, cand, n_cand = c.filter_readset(ragged)
    oh, on = o.filter_reads(ragged, *spec)
    assert np.array_equal(hits, oh) and n_cand == on and on > 0
    # decreasing offsets are rejected
    packed, mask = kc.pack_ascii(np.frombuffer(b"ACGT" * 40, dtype=np.uint8))
    with pytest.raises(kc.KcError) as e:
        c.filter_reads(packed, np.array([0, 100, 50, 160], dtype=np.uint64), mask)
    assert e.value.name == "KC_ERR_ARG"
    # hits only, no candidate list
    hits, cand, n_cand = c.filter_readset(w.samples[1], want_candidates=False)
    oh, on = o.filter_reads(w.samples[1], *spec)
    assert cand is None and np.array_equal(hits, oh) and n_cand == on
    # a one-sample job has no filter
    t = synth.tiny(scale=0.05)
    c1 = gpu_count(t)
    with pytest.raises(kc.KcError) as e:
        c1.filter_select(1, 2, 0, 0)
    assert e.value.name == "KC_ERR_STATE"
    # reset forgets the selection
    c.reset()
    with pytest.raises(kc.KcError) as e:
        c.filter_keys()
    assert e.value.name == "KC_ERR_STATE"


def test_filter_device_inputs_and_outputs(paired_small):
    torch = pytest.importorskip("torch")
    w, o = paired_small
    c = gpu_count(w)
    spec = (1, 2, 1, 0)
    c.filter_select(*spec)
    rs = w.samples[1]
    packed, mask = kc.pack_ascii(rs.ascii)
    dp = torch.from_numpy(packed.view(np.int64)).cuda()
    dm = torch.from_numpy(mask.view(np.int64)).cuda()
    do = torch.from_numpy(rs.offsets.view(np.int64)).cuda()
    hits = torch.empty(rs.n_reads, dtype=torch.int32, device="cuda")
    cand = torch.empty(rs.n_reads, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    _, cand_view, n_cand = c.filter_reads(dp, do, dm, hits=hits, candidates=cand)
    oh, on = o.filter_reads(rs, *spec)
    assert np.array_equal(hits.cpu().numpy().view(np.uint32), oh) and n_cand == on
    assert np.array_equal(cand_view.cpu().numpy().view(np.uint64), np.nonzero(oh)[0].astype(np.uint64))


@pytest.mark.parametrize("spill", [1, 2])
def test_filter_and_items_of_a_spilled_result(paired_small, spill):
    """A result spilled to pinned host memory is brought back to the device first."""
    w, o = paired_small
    w2 = synth.Workload(w.name, w.samples, w.k, 1 << 28, w.n_hashes, w.min_count)  # 2^10 slices of 2^12 words
    c = gpu_count(w2, strategy="partitioned", part_bits=10, spill=spill)
    assert c.stats()["spilled_bytes"] > 0
    ok, oc = o.result()  # the result does not depend on the filter size
    assert c.export_items().tobytes() == o.items16().tobytes()
    _check_filter(c, o, w, (1, 2, 0, 0))
    gk, gc = c.dump()
    assert np.array_equal(gk, ok) and np.array_equal(gc, oc)


def test_filter_bench_size_properties(oracle_mod):
    """The paired shape the benchmark's filter line times: 2 x 1,000,000 reads
    of 150 bp from 5 Mbp genomes (the tumour one with SNVs and indels), 2^32-bit
    filter, default configuration.  The selection is exactly the dump's keys
    that meet the predicate, each sample's hits add up to the selected keys'
    counts of that sample, and the oracle, counting two of 64 hash partitions
    in full, gives the same selected keys and counts in those partitions."""
    w = synth.paired(scale=0.1)
    c = gpu_count(w)
    gk, gc = c.dump()
    spec = (1, 2, 0, 0)
    n_sel = c.filter_select(*spec)
    sk, sc = c.filter_keys()
    t, n = gc[:, 1].astype(np.int64), gc[:, 0].astype(np.int64)
    want = (t >= 2) & (n <= 0)
    assert n_sel == int(want.sum()) > 1000
    assert np.array_equal(sk, gk[want]) and np.array_equal(sc, gc[want])
    for s, rs in enumerate(w.samples):
        hits, cand, n_cand = c.filter_readset(rs)
        assert int(hits.sum(dtype=np.uint64)) == int(sc[:, s].sum(dtype=np.uint64))
        assert n_cand == int((hits > 0).sum())
    q, parts = 6, [3, 40]
    o = oracle_mod.count(w, restrict=(q, parts))
    ok, oc = o.filter_select(*spec)
    mine = np.isin(oracle_mod.partitions(sk, q), parts)
    assert np.array_equal(sk[mine], ok) and np.array_equal(sc[mine], oc)


def test_stems_parity_two_samples(paired_small, strategy):
    w, o = paired_small
    c = gpu_count(w, strategy=strategy)
    got = c.export_stems()
    assert got.tobytes() == o.stems().tobytes()
    assert c.stats()["stem_items"] == got.size


@pytest.mark.parametrize("k", [3, 4, 8, 16, 31])
def test_stems_parity_ragged_even_and_odd_k(oracle_mod, k):
    """Even k: stems of even length can be their own reverse complement (two
    entries per key); odd k: never."""
    rng = random.Random(400 + k)
    alphabet = "AT" if k <= 8 else "ACGT"
    reads = ["".join("N" if rng.random() < 0.01 else rng.choice(alphabet) for _ in range(rng.randint(0, 200)))
             for _ in range(600)]
    w = synth.Workload("ragged", [synth.ReadSet.from_strings(reads)], k, 1 << 20, 3, 1)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 18)
    assert c.export_stems().tobytes() == o.stems().tobytes()


def test_stems_clamp_device_buffer_and_errors(oracle_mod):
    torch = pytest.importorskip("torch")
    normal = ["A" * 70_000, "ACGTTGCA" * 3]
    tumour = ["AAAC", "ACGTTGCA" * 3, "C" * 40]
    w = synth.Workload("clamp", [synth.ReadSet.from_strings(normal), synth.ReadSet.from_strings(tumour)],
                       3, 1 << 16, 4, 2)
    o = oracle_mod.count(w)
    c = gpu_count(w, table_slots=1 << 12)
    items = c.export_stems()
    assert items.tobytes() == o.stems().tobytes()
    assert items[0]["stem"] == 0 and items[0]["count"][0][0] == 65535
    out = torch.empty(9 * items.size, dtype=torch.int64, device="cuda")
    c.export_stems(out)
    assert out.cpu().numpy().view(np.uint8).tobytes() == o.stems().tobytes()
    with pytest.raises(kc.KcError) as e:
        c.export_stems(out[: 9 * (items.size - 1)])
    assert e.value.name == "KC_ERR_CAPACITY"
    # after a reset the table is rebuilt for the new job
    c.reset()
    c.add_readset(0, w.samples[1])
    c.finalize()
    o2 = oracle_mod.Oracle(3, 2, 1 << 16, 4, 2)
    o2.add_reads(0, w.samples[1])
    assert c.export_stems().tobytes() == o2.stems().tobytes()
    # k < 3 has no stems
    c2 = kc.KmerCounter(2, 1, 1 << 16, 4, 1)
    c2.add_readset(0, synth.ReadSet.from_strings(["ACGTACGT"]))
    c2.finalize()
    with pytest.raises(kc.KcError) as e:
        c2.export_stems()
    assert e.value.name == "KC_ERR_STATE"


@pytest.mark.parametrize("spill", [1, 2])
def test_stems_of_a_spilled_result(paired_small, spill):
    w, o = paired_small
    w2 = synth.Workload(w.name, w.samples, w.k, 1 << 28, w.n_hashes, w.min_count)
    c = gpu_count(w2, strategy="partitioned", part_bits=10, spill=spill)
    assert c.export_stems().tobytes() == o.stems().tobytes()


def test_stems_bench_size_properties():
    """Paired shape of the benchmark (2 x 1,000,000 reads, k = 31): a stem of
    29 bases is never its own reverse complement, so every result key fills
    exactly one entry: the entries add up to the dump's counts per sample,
    stems are strictly ascending and every item has an entry."""
    w = synth.paired(scale=0.1)
    c = gpu_count(w)
    keys, counts = c.dump()
    items = c.export_stems()
    cnt = items["count"].astype(np.uint64)  # [n, 2, 16]
    assert counts.max() < 65535
    for s in range(2):
        assert int(cnt[:, s, :].sum()) == int(counts[:, s].sum(dtype=np.uint64))
    assert int(((cnt[:, 0, :] + cnt[:, 1, :]) > 0).sum()) == keys.size
    assert np.all(np.diff(items["stem"].astype(np.uint64)) > 0)
    assert np.all((cnt.sum(axis=(1, 2))) > 0)

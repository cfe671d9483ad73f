"""The synthetic inputs follow their stated recipe (they stand in for the
paper's sequencing data): uniform i.i.d. genome bases, reads that start
uniformly on either strand with the stated substitution and N rates, read
lengths uniform in their range, tumour copies with the stated SNV and indel
rates, seeded and independent of the thread count."""
import ctypes

import numpy as np
import pytest

import synth

COMP = bytes.maketrans(b"ACGT", b"TGCA")


def _revcomp(b: bytes) -> bytes:
    return b.translate(COMP)[::-1]


def _chi2_uniform(counts):
    counts = np.asarray(counts, dtype=np.float64)
    e = counts.sum() / counts.size
    return float(((counts - e) ** 2 / e).sum())


def test_genome_uniform_and_seeded():
    g = synth.genome(5, 2_000_000)
    assert set(np.unique(g).tobytes()) == set(b"ACGT")
    counts = [int((g == c).sum()) for c in b"ACGT"]
    assert _chi2_uniform(counts) < 16.3  # 3 degrees of freedom, p = 0.001
    # adjacent bases independent: the 16 dinucleotides are uniform too
    pair = (np.searchsorted(np.frombuffer(b"ACGT", np.uint8), g[:-1]) * 4
            + np.searchsorted(np.frombuffer(b"ACGT", np.uint8), g[1:]))
    assert _chi2_uniform(np.bincount(pair, minlength=16)) < 37.7  # 15 d.o.f., p = 0.001
    assert np.array_equal(g, synth.genome(5, 2_000_000))
    assert not np.array_equal(g[:1000], synth.genome(6, 1000))


def test_output_does_not_depend_on_threads():
    lib = synth._load()
    G = 3_000_000
    a = np.empty(G, dtype=np.uint8)
    b = np.empty(G, dtype=np.uint8)
    assert lib.synth_genome(9, G, a.ctypes.data, 1) == 0
    assert lib.synth_genome(9, G, b.ctypes.data, 7) == 0
    assert np.array_equal(a, b)
    n = 40_000
    o1 = np.empty(n + 1, dtype=np.uint64)
    o2 = np.empty(n + 1, dtype=np.uint64)
    assert lib.synth_read_offsets(9, n, 100, 250, o1.ctypes.data, 1) == 0
    assert lib.synth_read_offsets(9, n, 100, 250, o2.ctypes.data, 5) == 0
    assert np.array_equal(o1, o2)
    r1 = np.empty(int(o1[-1]), dtype=np.uint8)
    r2 = np.empty(int(o1[-1]), dtype=np.uint8)
    assert lib.synth_reads(9, a.ctypes.data, G, n, ctypes.c_double(0.005), ctypes.c_double(0.0005),
                           o1.ctypes.data, r1.ctypes.data, 1) == 0
    assert lib.synth_reads(9, a.ctypes.data, G, n, ctypes.c_double(0.005), ctypes.c_double(0.0005),
                           o1.ctypes.data, r2.ctypes.data, 6) == 0
    assert np.array_equal(r1, r2)


def test_read_lengths_uniform_in_range():
    rs = synth.reads(3, synth.genome(3, 100_000), 200_000, 100, 250, 0.0, 0.0)
    lens = np.diff(rs.offsets.astype(np.int64))
    assert lens.min() == 100 and lens.max() == 250
    assert _chi2_uniform(np.bincount(lens - 100, minlength=151)) < 209.0  # 150 d.o.f., p = 0.001
    assert abs(lens.mean() - 175.0) < 0.5


def test_error_free_reads_are_genome_substrings_from_both_strands():
    G = 20_000
    g = synth.genome(4, G)
    gb, gr = g.tobytes(), _revcomp(g.tobytes())
    rs = synth.reads(4, g, 4000, 60, 60, 0.0, 0.0)
    plus = minus = 0
    starts = []
    for r in range(rs.n_reads):
        s = rs.ascii[rs.offsets[r]:rs.offsets[r + 1]].tobytes()
        i = gb.find(s)
        if i >= 0:
            plus += 1
            starts.append(i)
        else:
            j = gr.find(s)
            assert j >= 0, "a read is not a substring of either strand"
            minus += 1
            starts.append(G - 60 - j)  # start on the plus strand
    assert abs(plus - minus) < 4 * np.sqrt(rs.n_reads)  # fair strand coin
    hist = np.bincount(np.asarray(starts) * 10 // (G - 60 + 1), minlength=10)
    assert _chi2_uniform(hist) < 27.9  # uniform starts, 9 d.o.f., p = 0.001


def test_substitution_and_n_rates():
    """Reads of a short genome are placed back by their error-free 16-base
    anchors; mismatches (not N) and N bases match the stated rates."""
    G, L = 50_000, 150
    g = synth.genome(8, G)
    gb, gr = g.tobytes(), _revcomp(g.tobytes())
    e, n = 0.005, 0.0005
    rs = synth.reads(8, g, 6000, L, L, e, n)
    index = {}
    for strand, seq in ((0, gb), (1, gr)):
        for i in range(len(seq) - 15):
            index.setdefault(seq[i:i + 16], []).append((strand, i))
    subs = ns = bases = 0
    for r in range(rs.n_reads):
        s = rs.ascii[rs.offsets[r]:rs.offsets[r + 1]].tobytes()
        placed = None
        for a in range(0, L - 16, 16):  # the first anchor that occurs once
            hits = index.get(s[a:a + 16], [])
            if len(hits) == 1:
                strand, i = hits[0]
                if 0 <= i - a and i - a + L <= G:
                    placed = ((gb, gr)[strand], i - a)
                    break
        if placed is None:
            continue
        seq, st = placed
        ref = seq[st:st + L]
        ra = np.frombuffer(s, np.uint8)
        rb = np.frombuffer(ref, np.uint8)
        is_n = ra == ord("N")
        ns += int(is_n.sum())
        subs += int(((ra != rb) & ~is_n).sum())
        bases += L
    assert bases > 0.95 * rs.n_reads * L
    # substitutions are drawn before N, so a base that is N hides its substitution: rate e (1 - n)
    for got, p in ((subs / bases, e * (1 - n)), (ns / bases, n)):
        sd = np.sqrt(p * (1 - p) / bases)
        assert abs(got - p) < 5 * sd + 1e-9, (got, p)


def test_tumour_copy_rates():
    G = 2_000_000
    g = synth.genome(3, G)
    t = synth.mutate(6, g, 0.001, 0.0, 10)
    assert t.size == G
    diff = int((t != g).sum())
    p = 0.001
    assert abs(diff / G - p) < 5 * np.sqrt(p * (1 - p) / G)
    t2 = synth.mutate(6, g, 0.0, 1e-4, 10)
    # insertions and deletions of 1..10 bases with equal odds: the length moves by a zero-mean walk
    assert t2.size != G and abs(t2.size - G) < 2000
    assert np.array_equal(synth.mutate(6, g, 0.001, 1e-5, 10), synth.mutate(6, g, 0.001, 1e-5, 10))


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_named_workloads_match_their_shapes(name):
    w = synth.WORKLOADS[name](scale=0.01)
    rs = w.samples[0]
    lens = np.diff(rs.offsets.astype(np.int64))
    assert lens.min() == lens.max() == (100 if name == "tiny" else 150)
    assert w.k == 31 and w.n_hashes == 4 and w.min_count == 2
    assert w.bloom_bits == (1 << 24 if name == "tiny" else 1 << 30)

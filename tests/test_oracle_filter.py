"""Pins for the oracle's downstream functions: 16-byte items, joint spectrum,
Filter-unit selection and read hits, stem-grouped 72-byte items.

* brute force by string operations on tiny random inputs (tests/_brute.py);
* the item layout of Section III-D (8-byte key, two counts in 4 bytes, 4
  bytes of padding) written with struct, and the clamp of a count above
  65535;
* the paper's stem example (Section II-A: the stem of ACGGCAGC is CGGCAG)
  and the stem item layout (8-byte stem, 16 + 16 two-byte counts, Section
  III-D); stem items rebuilt from brute force by enumerating the 16
  extensions of every canonical stem;
* a closed form: a tumour genome that differs from the normal one by one
  substitution, read by reads at every start on both strands, has exactly the
  k windows over the substitution as tumour-only k-mers, with counts and read
  hits that follow from the read geometry alone.
"""
import random
import struct

import numpy as np
import pytest

import synth
from tests import _brute

SPECS = [  # (tumor, min_tumor, max_normal, ratio)
    (1, 2, 0, 0),
    (1, 1, 1, 0),
    (0, 2, 0, 0),
    (1, 2, 3, 2),
    (0, 1, 100, 1),
    (1, 1000, 0, 0),  # selects nothing
]


def _oracle(oracle_mod, samples, k, min_count, bloom_bits=1 << 16, n_hashes=4):
    o = oracle_mod.Oracle(k, len(samples), bloom_bits, n_hashes, min_count)
    for s, reads in enumerate(samples):
        o.add_reads(s, synth.ReadSet.from_strings(reads))
    return o


def _random_reads(rng, n, max_len, n_rate, alphabet="ACGT"):
    out = []
    for _ in range(n):
        L = rng.randint(0, max_len)
        out.append("".join("N" if rng.random() < n_rate else rng.choice(alphabet) for _ in range(L)))
    return out


def _paired_reads(rng, n, max_len):
    """Two samples over a small alphabet so keys repeat and counts differ."""
    normal = _random_reads(rng, n, max_len, 0.02, alphabet="ACGT")
    tumour = [r[: len(r) // 2] + "".join(rng.choice("AC") for _ in range(len(r) - len(r) // 2)) for r in normal]
    tumour += _random_reads(rng, n // 2, max_len, 0.02, alphabet="AC")
    return normal, tumour


def _item_bytes(key, counts):
    c = [min(x, 65535) for x in counts] + [0] * (2 - len(counts))
    return struct.pack("<QHHI", key, c[0], c[1], 0)


@pytest.mark.parametrize("n_samples", [1, 2])
@pytest.mark.parametrize("k", [3, 7, 13])
def test_items16_bruteforce(oracle_mod, n_samples, k):
    rng = random.Random(100 + k + n_samples)
    samples = [_random_reads(rng, 30, 60, 0.02, alphabet="ACG") for _ in range(n_samples)]
    o = _oracle(oracle_mod, samples, k, 2)
    expect = b"".join(_item_bytes(key, c) for key, c in _brute.count(samples, k, 2))
    got = o.items16()
    assert got.shape[1] == 16  # Section III-D: one k-mer item is 16 bytes
    assert got.tobytes() == expect


def test_items16_count_clamp(oracle_mod):
    """A count above 65535 is clamped in the 16-bit field; the key and the other count are intact."""
    long_read = "A" * 70_000  # k=3: key AAA (0) seen 69,998 times
    o = _oracle(oracle_mod, [[long_read, "ACGTTG"], ["AAAC", "ACGTTG"]], 3, 2)
    items = o.items16()
    expect = b"".join(_item_bytes(key, c) for key, c in _brute.count([[long_read, "ACGTTG"], ["AAAC", "ACGTTG"]], 3, 2))
    assert items.tobytes() == expect
    key, c0, c1, pad = struct.unpack("<QHHI", items[0].tobytes())
    assert (key, c0, c1, pad) == (0, 65535, 1, 0)  # AAA: 69,998 times in sample 0, once (in AAAC) in sample 1


@pytest.mark.parametrize("cap", [1, 3, 50])
@pytest.mark.parametrize("n_samples", [1, 2])
def test_spectrum_bruteforce(oracle_mod, cap, n_samples):
    rng = random.Random(7 * cap + n_samples)
    samples = [_random_reads(rng, 40, 80, 0.01, alphabet="AC") for _ in range(n_samples)]
    o = _oracle(oracle_mod, samples, 5, 1)
    expect = np.zeros((cap + 1,) * n_samples, dtype=np.uint64)
    for _, c in _brute.count(samples, 5, 1):
        expect[tuple(min(x, cap) for x in c)] += 1
    got = o.spectrum(cap)
    assert np.array_equal(got, expect)
    assert int(got.sum()) == len(o.result()[0])


def _brute_selected(samples, k, min_count, spec):
    tumor, min_tumor, max_normal, ratio = spec
    out = []
    for key, c in _brute.count(samples, k, min_count):
        t, n = c[tumor], c[1 - tumor]
        if t >= min_tumor and n <= max_normal and t >= ratio * n:
            out.append((key, c))
    return out


@pytest.mark.parametrize("spec", SPECS)
@pytest.mark.parametrize("k", [4, 9])
def test_filter_select_and_reads_bruteforce(oracle_mod, spec, k):
    rng = random.Random(31 * k + spec[1])
    normal, tumour = _paired_reads(rng, 40, 70)
    samples = [normal, tumour]
    o = _oracle(oracle_mod, samples, k, 2)
    sel = _brute_selected(samples, k, 2, spec)
    keys, counts = o.filter_select(*spec)
    assert [int(x) for x in keys] == [key for key, _ in sel]
    assert [[int(a), int(b)] for a, b in counts] == [c for _, c in sel]
    sel_keys = {key for key, _ in sel}
    for reads in samples + [_random_reads(rng, 25, 50, 0.05, alphabet="ACGT")]:
        hits, n_cand = o.filter_reads(synth.ReadSet.from_strings(reads), *spec)
        expect = [sum(1 for w in _brute.windows(r, k) if _brute.as_int(_brute.canonical_str(w)) in sel_keys)
                  for r in reads]
        assert [int(x) for x in hits] == expect
        assert n_cand == sum(1 for x in expect if x > 0)


def test_filter_hits_sum_to_selected_counts(oracle_mod):
    """Counts are exact, so a sample's hits add up to the selected keys' counts of that sample."""
    rng = random.Random(5)
    normal, tumour = _paired_reads(rng, 60, 90)
    o = _oracle(oracle_mod, [normal, tumour], 6, 2)
    for spec in SPECS:
        _, counts = o.filter_select(*spec)
        for s, reads in enumerate([normal, tumour]):
            hits, _ = o.filter_reads(synth.ReadSet.from_strings(reads), *spec)
            assert int(hits.sum()) == int(counts[:, s].sum())


def _revcomp(s):
    return _brute.revcomp_str(s)


def test_filter_single_substitution_closed_form(oracle_mod):
    """Tumour = normal genome with one substitution at p; reads of length L at every
    start on both strands.  The selected k-mers (tumour >= 2, normal 0) are the k
    windows over p, window j seen 2 * (min(j, G-L) - max(0, j+k-L) + 1) times; a
    tumour read at start s hits max(0, min(s+L-k, p) - max(s, p-k+1) + 1) of them."""
    rng = random.Random(2024)
    G, L, k, p = 1200, 60, 21, 600
    normal_g = "".join(rng.choice("ACGT") for _ in range(G))
    alt = rng.choice([b for b in "ACGT" if b != normal_g[p]])
    tumour_g = normal_g[:p] + alt + normal_g[p + 1 :]
    mutant = [tumour_g[j : j + k] for j in range(p - k + 1, p + 1)]
    # the construction relies on these windows being new and unique (true for this seed)
    both = normal_g + "|" + _revcomp(normal_g)
    for w in mutant:
        assert w not in both and _revcomp(w) not in both
        assert tumour_g.count(w) + _revcomp(tumour_g).count(w) == 1

    def tiling(g):
        reads = []
        for s in range(G - L + 1):
            reads.append(g[s : s + L])
            reads.append(_revcomp(g[s : s + L]))
        return reads

    normal_reads, tumour_reads = tiling(normal_g), tiling(tumour_g)
    o = _oracle(oracle_mod, [normal_reads, tumour_reads], k, 2, bloom_bits=1 << 18)
    keys, counts = o.filter_select(1, 2, 0, 0)
    expect = sorted((_brute.as_int(_brute.canonical_str(w)),
                     2 * (min(j, G - L) - max(0, j + k - L) + 1))
                    for j, w in zip(range(p - k + 1, p + 1), mutant))
    assert [int(x) for x in keys] == [key for key, _ in expect]
    assert [int(x) for x in counts[:, 1]] == [c for _, c in expect]
    assert not counts[:, 0].any()
    hits, n_cand = o.filter_reads(synth.ReadSet.from_strings(tumour_reads), 1, 2, 0, 0)
    expect_hits = []
    for s in range(G - L + 1):
        h = max(0, min(s + L - k, p) - max(s, p - k + 1) + 1)
        expect_hits += [h, h]
    assert [int(x) for x in hits] == expect_hits
    assert n_cand == sum(1 for h in expect_hits if h)
    n_hits, n_cand_normal = o.filter_reads(synth.ReadSet.from_strings(normal_reads), 1, 2, 0, 0)
    assert n_cand_normal == 0 and not n_hits.any()


def test_filter_needs_two_samples(oracle_mod):
    o = _oracle(oracle_mod, [["ACGTACGT"]], 3, 1)
    with pytest.raises(ValueError):
        o.filter_select(1, 2, 0, 0)


def _stem_items_brute(samples, k, min_count):
    """Stem items from brute-force counts: every canonical stem that a result
    k-mer has (in either orientation), each of its 16 one-base extensions
    looked up by its canonical string."""
    counts = {_brute.as_str(key, k): c for key, c in _brute.count(samples, k, min_count)}
    stems = set()
    for kmer in counts:
        for o in (kmer, _brute.revcomp_str(kmer)):
            st = o[1:-1]
            stems.add(min(st, _brute.revcomp_str(st)))
    out = []
    for st in sorted(stems):
        per = [[0] * 16 for _ in range(2)]
        for xi, x in enumerate("ACGT"):
            for yi, y in enumerate("ACGT"):
                c = counts.get(_brute.canonical_str(x + st + y))
                if c:
                    for s_i, v in enumerate(c):
                        per[s_i][4 * xi + yi] = min(v, 65535)
        out.append(struct.pack("<Q16H16H", _brute.as_int(st), *per[0], *per[1]))
    return b"".join(out)


def test_stem_paper_example(oracle_mod):
    """Section II-A: the stem of ACGGCAGC is CGGCAG.  Alone, the k-mer gives one
    item: stem CGGCAG (its own canonical form), count 1 at (first A, last C)."""
    o = _oracle(oracle_mod, [["ACGGCAGC"]], 8, 1)
    items = o.stems()
    assert items.shape == (1, 72)
    stem, *counts = struct.unpack("<Q16H16H", items[0].tobytes())
    assert _brute.as_str(stem, 6) == "CGGCAG"
    assert counts[: 16] == [0, 1] + [0] * 14 and counts[16:] == [0] * 16


@pytest.mark.parametrize("k", [3, 4, 5, 8])
@pytest.mark.parametrize("n_samples,min_count", [(1, 1), (2, 1), (2, 2)])
def test_stems_bruteforce(oracle_mod, k, n_samples, min_count):
    rng = random.Random(17 * k + 3 * n_samples + min_count)
    alphabet = "ACG" if k > 4 else "ACGT"  # repeats for larger k; even k also meets palindromic stems
    samples = [_random_reads(rng, 40, 40, 0.02, alphabet=alphabet) for _ in range(n_samples)]
    o = _oracle(oracle_mod, samples, k, min_count)
    got = o.stems()
    assert got.shape[1] == 72  # Section III-D: 8 bytes of stem, 2 bytes per count, 16 + 16 counts
    assert got.tobytes() == _stem_items_brute(samples, k, min_count)


def test_stems_palindromic_stems(oracle_mod):
    """k = 4: stem AT is its own reverse complement; AATG and its reverse complement
    CATT both extend it, so the item holds the count at (A, G) and at (C, T)."""
    o = _oracle(oracle_mod, [["AATG", "AATG"]], 4, 1)
    items = o.stems()
    assert items.tobytes() == _stem_items_brute([["AATG", "AATG"]], 4, 1)
    rows = {_brute.as_str(struct.unpack("<Q", it[:8].tobytes())[0], 2): it for it in items}
    c = struct.unpack("<16H", rows["AT"][8:40].tobytes())
    assert c[4 * 0 + 2] == 2 and c[4 * 1 + 3] == 2  # (A, G) and (C, T)


def test_stems_need_k3(oracle_mod):
    o = _oracle(oracle_mod, [["ACGT"]], 2, 1)
    with pytest.raises(ValueError):
        o.stems()


def test_stems_count_clamp(oracle_mod):
    """AAA seen 69,998 times: its stem item (stem A, entry (A, A)) holds 65535."""
    samples = [["A" * 70_000, "CAGT"], ["AAAC"]]
    o = _oracle(oracle_mod, samples, 3, 1)
    items = o.stems()
    assert items.tobytes() == _stem_items_brute(samples, 3, 1)
    stem, *counts = struct.unpack("<Q16H16H", items[0].tobytes())
    assert stem == 0 and counts[0] == 65535 and counts[16] == 1

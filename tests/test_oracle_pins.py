"""Pins for the CPU oracle, against facts that do not come from the oracle.

* the paper's worked example and amplification arithmetic (Section II-A);
* brute force by string operations on tiny random inputs (tests/_brute.py);
* invariants: total count = number of valid windows, strand symmetry,
  no false negatives in the Bloom filter, OR-union of filters;
* the word-blocked Bloom filter's false-positive rate against its closed form;
* the mixer against the published SplitMix64 outputs and its exact inverse.
"""
import math
import os
import random

import numpy as np
import pytest

import synth
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _reads(strings):
    return synth.ReadSet.from_strings(strings)


def _oracle_result(oracle_mod, samples, k, min_count, bloom_bits=1 << 16, n_hashes=4):
    o = oracle_mod.Oracle(k, len(samples), bloom_bits, n_hashes, min_count)
    for s, reads in enumerate(samples):
        o.add_reads(s, _reads(reads))
    keys, counts = o.result()
    return o, [(int(a), [int(x) for x in c]) for a, c in zip(keys, counts)]


def _random_reads(rng, n, max_len, n_rate):
    out = []
    for _ in range(n):
        L = rng.randint(0, max_len)
        out.append("".join("N" if rng.random() < n_rate else rng.choice("ACGT") for _ in range(L)))
    return out


def test_paper_worked_example(oracle_mod):
    """Section II-A: ACGGCAGCTG has exactly the three 8-mers the paper lists."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "paper_example_k8.txt")) if l.strip() and l[0] != "#"]
    read = lines[0][1]
    k = int(lines[1][1])
    rows = lines[2:]
    assert len(read) - k + 1 == len(rows) == 3
    assert [_brute.windows(read, k).__next__()] == [rows[0][0]]
    assert list(_brute.windows(read, k)) == [r[0] for r in rows]
    for w, rc, can in rows:
        assert _brute.revcomp_str(w) == rc
        assert oracle_mod.canonical(w) == _brute.as_int(can)
    _, res = _oracle_result(oracle_mod, [[read]], k, 1)
    assert [(_brute.as_str(key, k), c) for key, c in res] == sorted((r[2], [1]) for r in rows)


def test_paper_amplification(oracle_mod):
    """Section II-A: a 100-base read has 71 30-mers, 568 bytes at 8 bytes each (5.68x)."""
    rng = random.Random(5)
    read = "".join(rng.choice("ACGT") for _ in range(100))
    o, _ = _oracle_result(oracle_mod, [[read]], 30, 1)
    assert o.windows == 71
    assert o.windows * 8 == 568
    assert abs(o.windows * 8 / len(read) - 5.68) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 4, 5, 8, 13, 25, 31])
@pytest.mark.parametrize("min_count", [1, 2, 3])
def test_bruteforce_single_sample(oracle_mod, k, min_count):
    rng = random.Random(1000 * k + min_count)
    reads = _random_reads(rng, 40, 120, 0.02)
    # repeats make counts above 1 likely even for long k
    reads += reads[:10] + [_brute.revcomp_str(r.replace("N", "A")) for r in reads[10:15]]
    _, got = _oracle_result(oracle_mod, [reads], k, min_count)
    assert got == _brute.count([reads], k, min_count)


@pytest.mark.parametrize("k", [3, 8, 31])
def test_bruteforce_two_samples(oracle_mod, k):
    rng = random.Random(77 + k)
    a = _random_reads(rng, 30, 150, 0.01)
    b = a[:12] + _random_reads(rng, 20, 150, 0.01)
    for mc in (1, 2, 4):
        _, got = _oracle_result(oracle_mod, [a, b], k, mc)
        assert got == _brute.count([a, b], k, mc)


def test_edge_reads(oracle_mod):
    k = 5
    reads = ["", "A", "ACGT", "ACGTA", "NNNNNNNN", "ACGTN", "NACGTA", "ACGTAACGTA", "acgta", "ACGTRACGTA"]
    o, got = _oracle_result(oracle_mod, [reads], k, 1)
    assert got == _brute.count([reads], k, 1)
    assert o.windows == _brute.n_valid_windows(reads, k)


def test_empty_read_sets(oracle_mod):
    for reads in ([], [""], ["", "", ""], ["ACG"], ["N" * 40]):
        o, got = _oracle_result(oracle_mod, [reads], 5, 1)
        assert got == [] and o.windows == 0
        assert not o.bloom().any()


def test_even_k_palindrome(oracle_mod):
    # ACGT is its own reverse complement: fwd == rc, counted once per window.
    _, got = _oracle_result(oracle_mod, [["ACGT", "ACGT", "TTTT"]], 4, 1)
    assert got == [(_brute.as_int("AAAA"), [1]), (_brute.as_int("ACGT"), [2])]


def _valid_windows_numpy(rs, k):
    """Valid windows from N positions and read lengths only (no k-mers built)."""
    total = 0
    bad = ~np.isin(rs.ascii, np.frombuffer(b"ACGT", dtype=np.uint8))
    csum = np.concatenate([[0], np.cumsum(bad, dtype=np.int64)])
    for r in range(rs.n_reads):
        lo, hi = int(rs.offsets[r]), int(rs.offsets[r + 1])
        if hi - lo < k:
            continue
        starts = np.arange(lo, hi - k + 1)
        total += int(np.count_nonzero(csum[starts + k] - csum[starts] == 0))
    return total


@pytest.mark.parametrize("k", [25, 31])
def test_invariant_total_count(oracle_mod, k):
    """I1: with min_count=1 the counts sum to the number of N-free windows."""
    w = synth.tiny(scale=0.1)
    o = oracle_mod.Oracle(k, 1, 1 << 20, 4, 1)
    o.add_reads(0, w.samples[0])
    keys, counts = o.result()
    expected = _valid_windows_numpy(w.samples[0], k)
    assert o.windows == expected
    assert int(counts.sum()) == expected
    assert len(keys) == o.distinct


def _revcomp_readset(rs):
    comp = np.frombuffer(bytes.maketrans(b"ACGT", b"TGCA"), dtype=np.uint8)
    out = []
    for r in range(rs.n_reads):
        seg = rs.ascii[rs.offsets[r] : rs.offsets[r + 1]]
        out.append(comp[seg[::-1]])
    data = np.concatenate(out) if out else np.zeros(0, np.uint8)
    offs = np.concatenate([[0], np.cumsum([len(x) for x in out])]).astype(np.uint64)
    return synth.ReadSet(data, offs)


def test_invariant_strand_symmetry(oracle_mod):
    """I2: reverse-complementing every read leaves the table and the filter unchanged."""
    w = synth.tiny(scale=0.1)
    fwd = oracle_mod.count(w)
    w.samples = [_revcomp_readset(w.samples[0])]
    rev = oracle_mod.count(w)
    kf, cf = fwd.result()
    kr, cr = rev.result()
    assert np.array_equal(kf, kr) and np.array_equal(cf, cr)
    assert np.array_equal(fwd.bloom(), rev.bloom())


def test_invariant_bloom_no_false_negative(oracle_mod):
    """I3: every counted key's pattern is contained in its word."""
    w = synth.tiny(scale=0.05)
    w.min_count = 1
    o = oracle_mod.count(w)
    keys, _ = o.result()
    bloom = o.bloom()
    for key in keys[:: max(1, len(keys) // 3000)]:
        p = o.bloom_pattern(int(key))
        assert 1 <= bin(p).count("1") <= w.n_hashes
        assert int(bloom[o.bloom_word_index(int(key))]) & p == p
        assert o.bloom_query(int(key))
    total_bits = sum(bin(int(x)).count("1") for x in bloom[bloom != 0])
    assert total_bits <= len(keys) * w.n_hashes


def test_bloom_union_is_or_and_order_free(oracle_mod):
    w = synth.tiny(scale=0.05)
    rs = w.samples[0]
    half = rs.n_reads // 2
    a, b = rs.slice(0, half), rs.slice(half, rs.n_reads)

    def bloom_of(parts):
        o = oracle_mod.Oracle(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count)
        for p in parts:
            o.add_reads(0, p)
        return o.bloom()

    ab, ba = bloom_of([a, b]), bloom_of([b, a])
    assert np.array_equal(ab, ba)
    assert np.array_equal(ab, bloom_of([a]) | bloom_of([b]))


def _fpr_closed_form(n_keys, n_words, h):
    """Word-blocked filter, h uniform bit draws per key in one of n_words words.

    A query with d distinct bits is a false positive iff all d bits were drawn by
    the X keys sharing its word: inclusion-exclusion over the h*X draws.
    """
    from math import comb

    # distribution of distinct bits among h uniform draws out of 64
    pd = np.zeros(h + 1)
    pd[0] = 1.0
    for _ in range(h):
        nxt = np.zeros(h + 1)
        for d in range(h):
            if pd[d]:
                nxt[d] += pd[d] * d / 64
                nxt[d + 1] += pd[d] * (64 - d) / 64
        pd = nxt
    p = 1.0 / n_words
    fpr = 0.0
    logp, log1p_ = math.log(p), math.log1p(-p)
    for x in range(0, min(n_keys, 200) + 1):
        px = math.exp(math.lgamma(n_keys + 1) - math.lgamma(x + 1) - math.lgamma(n_keys - x + 1)
                      + x * logp + (n_keys - x) * log1p_)
        for d in range(1, h + 1):
            all_set = sum((-1) ** j * comb(d, j) * (1 - j / 64) ** (h * x) for j in range(d + 1))
            fpr += px * pd[d] * all_set
    return fpr


@pytest.mark.parametrize("h,lam", [(1, 2.0), (3, 8.0)])
def test_bloom_fpr_closed_form(oracle_mod, h, lam):
    k = 31
    bloom_bits = 1 << 18
    n_words = bloom_bits // 64
    n_target = int(lam * n_words)
    g = synth.genome(12345 + h, n_target + k - 1)
    o = oracle_mod.Oracle(k, 1, bloom_bits, h, 1)
    o.add_reads(0, synth.ReadSet(g, np.array([0, len(g)], dtype=np.uint64)))
    inserted = set(int(x) for x in o.result()[0])
    rng = np.random.default_rng(9)
    queries = rng.integers(0, 1 << 62, size=60000, dtype=np.uint64)
    hits = trials = 0
    for q in queries:
        q = int(q)
        if q in inserted:
            continue
        trials += 1
        hits += o.bloom_query(q)
    fpr = hits / trials
    expect = _fpr_closed_form(len(inserted), n_words, h)
    sigma = math.sqrt(expect * (1 - expect) / trials)
    assert abs(fpr - expect) <= 5 * sigma + 0.03 * expect, (fpr, expect)


def test_mixer_published_outputs(oracle_mod):
    """SplitMix64 from state 0: output i = mixer64(i * golden gamma)."""
    gamma = 0x9E3779B97F4A7C15
    for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")):
        if line.startswith("#") or not line.strip():
            continue
        i, out = (int(x) for x in line.split())
        assert oracle_mod.mixer64((i * gamma) & M64) == out


def _unxorshift(y, s):
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x & M64


def test_mixer_is_a_bijection(oracle_mod):
    """Invert every stage (xor-shift, odd multiply, add) and recover the input."""
    c1, c2, gamma = 0xBF58476D1CE4E5B9, 0x94D049BB133111EB, 0x9E3779B97F4A7C15
    i1, i2 = pow(c1, -1, 1 << 64), pow(c2, -1, 1 << 64)
    rng = random.Random(3)
    for x in [0, 1, M64, 1 << 63] + [rng.getrandbits(64) for _ in range(2000)]:
        z = _unxorshift(oracle_mod.mixer64(x), 31)
        z = (z * i2) & M64
        z = _unxorshift(z, 27)
        z = (z * i1) & M64
        z = _unxorshift(z, 30)
        assert (z - gamma) & M64 == x


def test_restricted_runs_partition_the_result(oracle_mod):
    w = synth.tiny(scale=0.05)
    full = oracle_mod.count(w)
    fk, fc = full.result()
    fb = full.bloom()
    q = 2
    nw = w.bloom_bits // 64
    parts_k, parts_c = [], []
    for p in range(1 << q):
        o = oracle_mod.count(w, restrict=(q, [p]))
        k, c = o.result()
        parts_k.append(k)
        parts_c.append(c)
        assert o.windows == full.windows
        lo, n = p * (nw >> q), nw >> q
        assert np.array_equal(o.bloom(lo, n), fb[lo : lo + n])
        for key in k[:50]:
            assert oracle_mod.mixer64(int(key)) >> (64 - q) == p
    allk = np.concatenate(parts_k)
    order = np.argsort(allk)
    assert np.array_equal(allk[order], fk)
    assert np.array_equal(np.concatenate(parts_c)[order], fc)


def test_min_count_is_a_filter_on_the_sum(oracle_mod):
    w = synth.tiny(scale=0.05)
    rs = w.samples[0]
    half = rs.n_reads // 2
    two = synth.Workload("t2", [rs.slice(0, half), rs.slice(half, rs.n_reads)], w.k, w.bloom_bits,
                         w.n_hashes, 1)
    k1, c1 = oracle_mod.count(two).result()
    for mc in (2, 3, 7):
        two.min_count = mc
        k, c = oracle_mod.count(two).result()
        keep = c1.sum(axis=1) >= mc
        assert np.array_equal(k, k1[keep]) and np.array_equal(c, c1[keep])


def test_invalid_parameters_rejected(oracle_mod):
    for args in [(0, 1, 1 << 16, 4, 2), (32, 1, 1 << 16, 4, 2), (31, 3, 1 << 16, 4, 2),
                 (31, 1, 3000, 4, 2), (31, 1, 1 << 16, 0, 2), (31, 1, 1 << 16, 11, 2), (31, 1, 1 << 16, 4, 0)]:
        with pytest.raises(ValueError):
            oracle_mod.Oracle(*args)

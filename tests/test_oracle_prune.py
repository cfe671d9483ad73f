"""Pins for the oracle's bounds on the Prune chain's second filter (Section
III, Prune unit: a k-mer already present in the first filter goes into the
second one).

The second filter depends on the order of the insertions.  Here every order
of a handful of windows is played out one insertion at a time, in Python, with
the first filter and the second filter as dictionaries of words; the oracle's
lower bound must lie inside every order's second filter and its upper bound
must be the union over all orders.  Words and patterns come from the
oracle's own word/pattern functions, which test_oracle_pins.py pins against
the published SplitMix64 outputs.
"""
import itertools
import random

import numpy as np
import pytest

import synth
from tests import _brute


def _chain(o, keys):
    """Second filter after inserting keys in this order (word -> bits)."""
    bf1, bf2 = {}, {}
    for key in keys:
        w, p = o.bloom_word_index(key), o.bloom_pattern(key)
        if bf1.get(w, 0) & p == p:
            bf2[w] = bf2.get(w, 0) | p
        bf1[w] = bf1.get(w, 0) | p
    return bf2


def _bounds_as_dicts(o):
    lo, hi = o.bloom2_bounds()
    return ({int(i): int(lo[i]) for i in np.nonzero(lo)[0]}, {int(i): int(hi[i]) for i in np.nonzero(hi)[0]})


def _check_all_orders(o, keys):
    lo, hi = _bounds_as_dicts(o)
    union = {}
    for order in set(itertools.permutations(keys)):
        bf2 = _chain(o, order)
        for w, bits in lo.items():
            assert bf2.get(w, 0) & bits == bits  # lower bound inside every order
        for w, bits in bf2.items():
            union[w] = union.get(w, 0) | bits
    assert union == hi  # upper bound = what some order reaches


def _oracle_of_kmers(oracle_mod, kmers, k, bloom_bits, n_hashes):
    o = oracle_mod.Oracle(k, 1, bloom_bits, n_hashes, 2)
    o.add_reads(0, synth.ReadSet.from_strings(kmers))
    return o


def test_bounds_random_small_sets(oracle_mod):
    rng = random.Random(11)
    for trial in range(12):
        k = rng.choice([3, 4])
        kmers = ["".join(rng.choice("ACGT") for _ in range(k)) for _ in range(rng.randint(3, 6))]
        kmers += rng.sample(kmers, 1)  # one key seen twice
        o = _oracle_of_kmers(oracle_mod, kmers, k, 4096, rng.choice([1, 2, 3]))
        keys = [_brute.as_int(_brute.canonical_str(x)) for x in kmers]
        _check_all_orders(o, keys)


def test_bounds_singleton_covered_by_others(oracle_mod):
    """Three singletons A, B, C in one word with C's bits inside A's | B's but in
    neither alone: C is in the second filter exactly when it comes after both."""
    rng = random.Random(3)
    k, bloom_bits, n_hashes = 7, 4096, 2
    probe = oracle_mod.Oracle(k, 1, bloom_bits, n_hashes, 2)
    by_word = {}
    for _ in range(20000):
        s = "".join(rng.choice("ACGT") for _ in range(k))
        key = _brute.as_int(_brute.canonical_str(s))
        by_word.setdefault(probe.bloom_word_index(key), {})[key] = s
    found = None
    for keys in by_word.values():
        items = list(keys.items())
        for (a, sa), (b, sb), (c, sc) in itertools.permutations(items[:40], 3):
            pa, pb, pc = (probe.bloom_pattern(x) for x in (a, b, c))
            if pc & (pa | pb) == pc and pc & pa != pc and pc & pb != pc and (pa | pc) != pa:
                found = (sa, sb, sc)
                break
        if found:
            break
    assert found, "no covered triple in the sample"
    o = _oracle_of_kmers(oracle_mod, list(found), k, bloom_bits, n_hashes)
    keys = [_brute.as_int(_brute.canonical_str(x)) for x in found]
    lo, hi = _bounds_as_dicts(o)
    assert not lo  # all singletons
    w = probe.bloom_word_index(keys[2])
    assert hi.get(w, 0) & probe.bloom_pattern(keys[2]) == probe.bloom_pattern(keys[2])
    _check_all_orders(o, keys)


def test_bounds_keys_seen_twice_are_in_both(oracle_mod):
    rng = random.Random(8)
    reads = ["".join(rng.choice("AC") for _ in range(30)) for _ in range(20)]
    o = oracle_mod.Oracle(9, 1, 1 << 16, 4, 2)
    o.add_reads(0, synth.ReadSet.from_strings(reads))
    lo, hi = o.bloom2_bounds()
    keys, counts = o.result()
    assert keys.size > 0
    for key in keys:
        w, p = o.bloom_word_index(int(key)), o.bloom_pattern(int(key))
        assert int(lo[w]) & p == p
    assert np.all(lo & ~hi == 0) and np.all(hi & ~o.bloom() == 0)  # lower <= upper <= first filter

"""Brute-force k-mer counting on tiny inputs, by string operations only.

Used to pin the oracle: every window is taken as a substring, the reverse
complement is built by reversing the string and swapping A<->T, C<->G, the
canonical form is the lexicographically smaller string, and occurrences are
counted by sorting the list of strings and measuring runs (no hash map).
Strings are turned into integers only at the end, by reading them as base-4
numbers with A<C<G<T as digits 0..3 (the 2-bit reading of Section II-A).
"""
from __future__ import annotations

_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}
_DIGIT = {"A": 0, "C": 1, "G": 2, "T": 3}


def revcomp_str(s: str) -> str:
    return "".join(_COMP[c] for c in reversed(s))


def canonical_str(s: str) -> str:
    r = revcomp_str(s)
    return s if s <= r else r


def as_int(s: str) -> int:
    v = 0
    for c in s:
        v = v * 4 + _DIGIT[c]
    return v


def as_str(v: int, k: int) -> str:
    letters = "ACGT"
    out = []
    for _ in range(k):
        out.append(letters[v % 4])
        v //= 4
    return "".join(reversed(out))


def windows(read: str, k: int):
    for j in range(len(read) - k + 1):
        w = read[j : j + k]
        if all(c in _DIGIT for c in w):
            yield w


def count(samples, k: int, min_count: int):
    """samples: list (per sample) of lists of read strings.

    Returns sorted list of (key_int, [count per sample]) with total >= min_count.
    """
    tagged = []
    for s, reads in enumerate(samples):
        for read in reads:
            for w in windows(read, k):
                tagged.append((canonical_str(w), s))
    tagged.sort()
    out = []
    i = 0
    while i < len(tagged):
        j = i
        per = [0] * len(samples)
        while j < len(tagged) and tagged[j][0] == tagged[i][0]:
            per[tagged[j][1]] += 1
            j += 1
        if sum(per) >= min_count:
            out.append((as_int(tagged[i][0]), per))
        i = j
    out.sort()
    return out


def n_valid_windows(reads, k: int) -> int:
    return sum(1 for r in reads for _ in windows(r, k))

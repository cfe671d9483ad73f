"""Writes bloom_placement.txt: the word-blocked filter of three short reads,
placed step by step from printed hash values.

The filter's definition (hash C14 of the library's readings; the paper names
no hash, Section III, Prune unit):
    h = mixer64(key), g = mixer64(h)
    word  = the top log2(words) bits of h
    bit i = the i-th 6-bit field of g, counted from the least significant end
Only the two mixer values come from the oracle (``oracle.mixer64``, itself
pinned against the published SplitMix64 outputs).  Keys are found by string
operations, and the word and the bits are cut out of the binary digit
strings of h and g, so that a reader can repeat every step with a pencil.

Run from the repository root:  python tests/golden/make_bloom_placement.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests import _brute  # noqa: E402

K = 5
BLOOM_BITS = 4096                       # 64 words of 64 bits
LOG2_WORDS = 6
READS = ["ACGTTGCAT", "GGATGCNAC", "TTTTTAAAAA"]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bloom_placement.txt")


def main():
    keys = sorted({_brute.canonical_str(w) for r in READS for w in _brute.windows(r, K)},
                  key=_brute.as_int)
    lines = [
        "# Word-blocked Bloom filter of three hand-picked reads, placed by hand.",
        "# k = 5, filter of 4096 bits = 64 words (6 word bits), one sample.",
        "# Written by make_bloom_placement.py: h = mixer64(code) and g = mixer64(h)",
        "# come from oracle.mixer64 (pinned by the published SplitMix64 outputs);",
        "# everything after them is cut out of their binary digits:",
        "#   word  = the first 6 of the 64 binary digits of h (most significant first)",
        "#   bit i = binary digits 64-6(i+1) .. 64-6i-1 of g, i.e. the i-th 6-bit",
        "#           field from the least significant end (i = 0..3)",
        "# n_hashes = 1 uses bit 0 only; n_hashes = 4 uses bits 0..3.",
        "# The read GGATGCNAC loses its three windows over the N; TTTTTAAAAA shows",
        "# a window and its reverse complement sharing one canonical key.",
        f"k {K}",
        f"bloom_bits {BLOOM_BITS}",
    ]
    lines += [f"read {r}" for r in READS]
    lines.append("# key  code  h(hex)  h top byte(bin)  word  g(hex)  g low 24 bits(bin, 4 fields)  bits")
    words1, words4 = {}, {}
    for s in keys:
        code = _brute.as_int(s)
        h = oracle.mixer64(code)
        g = oracle.mixer64(h)
        hb, gb = format(h, "064b"), format(g, "064b")
        word = int(hb[:LOG2_WORDS], 2)
        fields = [gb[64 - 6 * (i + 1): 64 - 6 * i] for i in range(4)]
        bits = [int(f, 2) for f in fields]
        low24 = "_".join(reversed(fields))  # most significant field first, as printed binary reads
        lines.append(f"key {s} {code} {h:016x} {hb[:8]} {word} {g:016x} {low24} {','.join(map(str, bits))}")
        words1[word] = words1.get(word, 0) | (1 << bits[0])
        for b in bits:
            words4[word] = words4.get(word, 0) | (1 << b)
    for nh, words in ((1, words1), (4, words4)):
        lines.append(f"# filter with n_hashes = {nh}: the non-zero words (every other word is 0)")
        lines.append(f"filter {nh}")
        for w in sorted(words):
            lines.append(f"word {w} {words[w]:016x}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

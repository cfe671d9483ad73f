"""Pin of the oracle's Bloom placement against a filter placed by hand.

tests/golden/bloom_placement.txt lists, for three short reads (k = 5, a
64-word filter), every canonical key, its two mixer values and the word and
bits cut out of their binary digits, and the filter words that result for one
and for four hash bits.  The mixer is pinned separately (the published
SplitMix64 outputs); this file pins what the oracle does with its values:
which bits of h choose the word, which hash gives the bits, and the 6-bit
stride between them.  Three mistakes planted in a copy of the oracle (bits
from h instead of g, the word from the low bits of h, an 8-bit stride) each
change the filter.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from tests import _brute

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "bloom_placement.txt")
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "kc_oracle.cpp")


def _golden():
    g = {"reads": [], "keys": [], "filters": {}}
    cur = None
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "k":
            g["k"] = int(f[1])
        elif f[0] == "bloom_bits":
            g["bloom_bits"] = int(f[1])
        elif f[0] == "read":
            g["reads"].append(f[1])
        elif f[0] == "key":
            g["keys"].append(dict(s=f[1], code=int(f[2]), h=int(f[3], 16), h_top=f[4], word=int(f[5]),
                                  g=int(f[6], 16), g_low=f[7], bits=[int(b) for b in f[8].split(",")]))
        elif f[0] == "filter":
            cur = int(f[1])
            g["filters"][cur] = {}
        elif f[0] == "word":
            g["filters"][cur][int(f[1])] = int(f[2], 16)
    return g


def _expected_words(g, nh):
    out = np.zeros(g["bloom_bits"] // 64, dtype=np.uint64)
    for w, v in g["filters"][nh].items():
        out[w] = v
    return out


def test_placement_inputs(oracle_mod):
    """The listed keys are the reads' canonical k-mers; h and g are the mixer's values."""
    g = _golden()
    k = g["k"]
    want = sorted({_brute.canonical_str(w) for r in g["reads"] for w in _brute.windows(r, k)})
    assert sorted(x["s"] for x in g["keys"]) == want
    assert len(want) == 10
    for x in g["keys"]:
        assert x["code"] == _brute.as_int(x["s"])
        assert oracle_mod.canonical(x["s"]) == x["code"]
        assert x["h"] == oracle_mod.mixer64(x["code"])
        assert x["g"] == oracle_mod.mixer64(x["h"])
        # the printed binary digits are those of the printed hex values
        assert x["h_top"] == format(x["h"] >> 56, "08b")
        assert x["g_low"].replace("_", "") == format(x["g"] & 0xFFFFFF, "024b")


def test_placement_file_is_consistent():
    """Each listed filter word is the OR of the listed bits of the keys placed in it."""
    g = _golden()
    for nh in (1, 4):
        words = {}
        for x in g["keys"]:
            for b in x["bits"][:nh]:
                words[x["word"]] = words.get(x["word"], 0) | (1 << b)
        assert words == g["filters"][nh]
    # the example exercises two keys sharing a word and a key whose bits collide
    assert len({x["word"] for x in g["keys"]}) < len(g["keys"])
    assert any(len(set(x["bits"])) < 4 for x in g["keys"])


@pytest.mark.parametrize("nh", [1, 4])
def test_oracle_filter_equals_hand_placement(oracle_mod, nh):
    g = _golden()
    o = oracle_mod.Oracle(g["k"], 1, g["bloom_bits"], nh, 1)
    o.add_reads(0, synth.ReadSet.from_strings(g["reads"]))
    assert np.array_equal(o.bloom(), _expected_words(g, nh))


def _compile_variant(src_text, path):
    with open(path + ".cpp", "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", path + ".cpp", "-o", path + ".so"])
    lib = ctypes.CDLL(path + ".so")
    u64, u32, p, i = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
    lib.orc_create.argtypes = [i, i, u64, i, u32]
    lib.orc_create.restype = p
    lib.orc_add_reads.argtypes = [p, i, p, p, u64]
    lib.orc_add_reads.restype = i
    lib.orc_bloom.argtypes = [p, p, u64, u64]
    lib.orc_bloom.restype = i
    lib.orc_destroy.argtypes = [p]
    lib.orc_destroy.restype = None
    return lib


def _variant_filter(lib, g, nh):
    rs = synth.ReadSet.from_strings(g["reads"])
    ascii = np.ascontiguousarray(rs.ascii, dtype=np.uint8)
    offs = np.ascontiguousarray(rs.offsets, dtype=np.uint64)
    h = lib.orc_create(g["k"], 1, g["bloom_bits"], nh, 1)
    assert h
    assert lib.orc_add_reads(h, 0, ascii.ctypes.data, offs.ctypes.data, len(offs) - 1) == 0
    out = np.zeros(g["bloom_bits"] // 64, dtype=np.uint64)
    assert lib.orc_bloom(h, out.ctypes.data, 0, out.size) == 0
    lib.orc_destroy(h)
    return out


# (name, text in the oracle, replacement): each a plausible misreading of the placement
PLANTED = [
    ("bits drawn from h instead of g", "uint64_t g = mixer64(mixer64(key));", "uint64_t g = mixer64(key);"),
    ("word from the low bits of h", "h >> (64 - log2_words)", "(h & ((1ull << log2_words) - 1))"),
    ("8-bit stride between the bit fields", "(g >> (6 * i))", "(g >> (8 * i))"),
]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs the host C++ compiler")
def test_planted_placement_mistakes_fail(tmp_path):
    g = _golden()
    src = open(ORACLE_SRC).read()
    # the unchanged source, compiled the same way, reproduces the hand placement
    lib = _compile_variant(src, str(tmp_path / "same"))
    for nh in (1, 4):
        assert np.array_equal(_variant_filter(lib, g, nh), _expected_words(g, nh))
    for n, (name, old, new) in enumerate(PLANTED):
        assert old in src, name
        lib = _compile_variant(src.replace(old, new), str(tmp_path / f"m{n}"))
        differs = [not np.array_equal(_variant_filter(lib, g, nh), _expected_words(g, nh)) for nh in (1, 4)]
        assert any(differs), f"planted mistake not caught: {name}"

"""CPU-side checks of the C ABI: the library builds, loads, exports every
declared symbol, validates arguments before touching the GPU, and packs reads
in the documented format."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1712_03254_gb300 as kc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(kc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = kc.build()
    declared = _declared_functions()
    assert "kc_create" in declared and "kc_add_reads" in declared and "kc_dump" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(path)
    for n in declared:
        assert getattr(L, n) is not None


def test_status_strings_and_default_config():
    L = kc.lib()
    assert L.kc_status_string(0) == b"KC_OK"
    assert L.kc_status_string(7) == b"KC_ERR_CAPACITY"
    cfg = kc.Config()
    L.kc_default_config(ctypes.byref(cfg))
    assert cfg.struct_size == ctypes.sizeof(kc.Config)
    assert cfg.table_slots == 0 and cfg.part_bits == 0


@pytest.mark.parametrize("args", [
    (0, 1, 1 << 20, 4, 2), (32, 1, 1 << 20, 4, 2), (31, 0, 1 << 20, 4, 2), (31, 3, 1 << 20, 4, 2),
    (31, 1, 3 << 20, 4, 2), (31, 1, 2048, 4, 2), (31, 1, 1 << 20, 0, 2), (31, 1, 1 << 20, 11, 2),
    (31, 1, 1 << 20, 4, 0),
])
def test_create_rejects_bad_arguments_before_cuda(args):
    L = kc.lib()
    h = ctypes.c_void_p()
    assert L.kc_create(*args, ctypes.byref(h)) == 1  # KC_ERR_ARG
    assert not h.value
    assert L.kc_last_error()


def test_null_handle_calls_fail_cleanly():
    L = kc.lib()
    n = ctypes.c_uint64()
    assert L.kc_finalize(None) == 1
    assert L.kc_dump(None, None, None, 0, ctypes.byref(n)) == 1
    assert L.kc_add_reads(None, 0, None, None, None, 0) == 1
    assert L.kc_export_items(None, None, 0, ctypes.byref(n)) == 1
    assert L.kc_spectrum(None, 4, None) == 1
    assert L.kc_export_stems(None, None, 0, ctypes.byref(n)) == 1
    assert L.kc_export_bloom2(None, None, 0, 0) == 1
    spec = kc.FilterSpec(1, 2, 0, 0)
    assert L.kc_filter_select(None, ctypes.byref(spec), ctypes.byref(n)) == 1
    assert L.kc_filter_keys(None, None, None, 0, ctypes.byref(n)) == 1
    assert L.kc_filter_reads(None, None, None, None, 0, None, None, ctypes.byref(n)) == 1
    L.kc_destroy(None)


def test_item16_layout_matches_the_header(tmp_path):
    """kc_item16 is the 16-byte item of Section III-D: key at 0, counts at 8 and 10, padding at 12."""
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "kc.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(kc_item16), offsetof(kc_item16, key),'
                   ' offsetof(kc_item16, count), offsetof(kc_item16, pad), sizeof(kc_filter_spec),'
                   ' sizeof(kc_stem_item), offsetof(kc_stem_item, count)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [16, 0, 8, 12, ctypes.sizeof(kc.FilterSpec), 72, 8]
    assert kc.STEM_ITEM.itemsize == 72 and kc.STEM_ITEM.fields["count"][1] == 8
    assert kc.ITEM16.itemsize == 16 and kc.ITEM16.fields["count"][1] == 8 and kc.ITEM16.fields["pad"][1] == 12


def test_stats_struct_matches_the_header(tmp_path):
    src = tmp_path / "stats.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "kc.h"\n'
                   'int main(void) { printf("%zu %zu\\n", sizeof(kc_stats), offsetof(kc_stats, filter_hits));'
                   ' return 0; }\n')
    exe = tmp_path / "stats"
    subprocess.run(["gcc", "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    size, off = (int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    assert size == ctypes.sizeof(kc.Stats) and off == kc.Stats.filter_hits.offset


def _pack_reference(ascii: bytes):
    """The packed format of include/kc.h, bit by bit."""
    n = len(ascii)
    packed = [0] * ((n + 31) // 32)
    mask = [0] * ((n + 63) // 64)
    code = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
    for i, c in enumerate(ascii):
        if c in code:
            packed[i // 32] |= code[c] << (63 - 2 * (i % 32) - 1)
        else:
            mask[i // 64] |= 1 << (63 - i % 64)
    return np.array(packed, dtype=np.uint64), np.array(mask, dtype=np.uint64)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 63, 64, 65, 127, 1000, 70001])
def test_pack_ascii_matches_format(n):
    rng = np.random.default_rng(n)
    ascii = rng.choice(np.frombuffer(b"ACGTNacgRY", dtype=np.uint8), size=n,
                       p=[0.22, 0.22, 0.22, 0.22, 0.04, 0.02, 0.02, 0.02, 0.02, 0.0])
    packed, mask = kc.pack_ascii(ascii)
    ref_p, ref_m = _pack_reference(ascii.tobytes())
    assert np.array_equal(packed, ref_p)
    assert np.array_equal(mask, ref_m)


@pytest.mark.parametrize("bloom_log2,part_bits,ok", [(24, 1, False), (24, 4, False), (24, 5, True), (24, 21, False),
                                                     (20, 1, True), (36, 14, False)])
def test_partitioned_slice_limit(bloom_log2, part_bits, ok):
    """The partitioned strategy keeps one partition's filter words (at most
    8192) in shared memory; larger slices are rejected before any CUDA call."""
    if ok:
        pytest.skip("valid configurations need a GPU to create")
    with pytest.raises(kc.KcError) as e:
        kc.KmerCounter(31, 1, 1 << bloom_log2, 4, 2, strategy="partitioned", part_bits=part_bits)
    assert e.value.name == "KC_ERR_ARG"


@pytest.mark.parametrize("kw", [dict(ctas_per_sm=65), dict(smem_table_log2=9), dict(smem_table_log2=14),
                                dict(split_max=14), dict(spill=3), dict(scatter_mode=5), dict(table_slots=1000),
                                dict(strategy="direct", table_slots=512), dict(prune_chain=2),
                                dict(prune_chain=True, strategy="partitioned")])
def test_config_knobs_out_of_range(kw):
    """Tuning knobs outside their documented ranges are rejected before any CUDA call."""
    with pytest.raises(kc.KcError) as e:
        kc.KmerCounter(31, 1, 1 << 24, 4, 2, **kw)
    assert e.value.name == "KC_ERR_ARG"


def test_plain_c_client_compiles_and_links(tmp_path):
    """The boundary is a C ABI: a C99 program using only include/kc.h builds and
    links against libkc.so (it runs on a GPU; here it is only built)."""
    lib = kc.build()
    exe = tmp_path / "kc_count"
    src = os.path.join(ROOT, "tests", "c_client", "kc_count.c")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INCLUDE, src, "-o", str(exe),
                    "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True, capture_output=True)
    assert exe.exists()

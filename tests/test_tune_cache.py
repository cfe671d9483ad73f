"""Tuning-cache file handling (no GPU needed: loading and saving never touch
the device).  The tuner itself is exercised in test_gpu_tune.py."""
import pytest

import paper_1712_03254_gb300 as kc

HEADER = "kc-tune-cache 1\n"
# k n_samples bloom_bits n_hashes min_gt1 bases_log2 sms | strategy part_bits table ctas scatter split ms
LINES = [
    "25 1 16777216 4 1 21 152 2 12 11 2 4 0 1.5",
    "31 1 1073741824 4 1 28 152 2 12 0 0 4 0 3.9",
    "31 2 4294967296 4 1 33 152 1 0 0 8 0 0 120.25",
]


@pytest.fixture(autouse=True)
def _clean():
    kc.tune_cache_clear()
    yield
    kc.tune_cache_clear()


def _rows(path):
    with open(path) as f:
        lines = f.read().splitlines()
    assert lines[0] == HEADER.strip()
    return sorted(tuple(float(x) for x in ln.split()) for ln in lines[1:] if ln)


def test_load_then_save_round_trip(tmp_path):
    src = tmp_path / "in.txt"
    src.write_text(HEADER + "\n".join(LINES) + "\n")
    kc.tune_cache_load(str(src))
    out = tmp_path / "out.txt"
    kc.tune_cache_save(str(out))
    assert _rows(out) == sorted(tuple(float(x) for x in ln.split()) for ln in LINES)


def test_malformed_files_change_nothing(tmp_path):
    good = tmp_path / "good.txt"
    good.write_text(HEADER + LINES[0] + "\n")
    kc.tune_cache_load(str(good))
    for bad in ["not a cache\n" + LINES[1],
                HEADER + "31 1 1073741824 4 1 28 152 2 12",              # too few fields
                HEADER + LINES[1] + " 7",                                  # trailing field
                HEADER + LINES[1].replace(" 12 0 0 4 0", " 12 9 0 4 0"),   # table log2 9: out of range
                HEADER + LINES[1].replace("1073741824", "1000000000")]:    # filter not a power of two
        p = tmp_path / "bad.txt"
        p.write_text(bad + "\n")
        with pytest.raises(kc.KcError) as e:
            kc.tune_cache_load(str(p))
        assert e.value.name == "KC_ERR_ARG"
    out = tmp_path / "out.txt"
    kc.tune_cache_save(str(out))
    assert _rows(out) == [tuple(float(x) for x in LINES[0].split())]


def test_missing_file_is_an_error(tmp_path):
    with pytest.raises(kc.KcError):
        kc.tune_cache_load(str(tmp_path / "nope.txt"))

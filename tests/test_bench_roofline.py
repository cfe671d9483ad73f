"""CPU checks of bench.py's roofline arithmetic: the committed ncu counters are
used only when their source hash matches the current kernel sources, the
"alu" form divides instructions by time by the issue peak, and the HBM forms
divide the stated algorithmic bytes by time by the measured copy bandwidth."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_counter_files_are_well_formed():
    for name, kernel, workload in (("ncu_kernels.json", "k_consume_q", "mid"),
                                   ("ncu_filter.json", "k_filter_hits", "paired-filter")):
        d = json.load(open(os.path.join(ROOT, "profiles", name)))
        assert len(d["source_hash"]) == 16
        prof = d["workloads"][workload][kernel]
        assert prof["inst_executed_per_launch"] > 0 and prof["dram_bytes_per_launch"] > 0


def test_filter_roofline_alu_form(monkeypatch):
    prof = {"inst_executed_per_launch": 348_000_000, "dram_bytes_per_launch": 78_000_000}
    monkeypatch.setattr(bench, "ncu_filter_kernel", lambda kernel, workload: prof)
    ms = 0.45
    r = bench.filter_roofline(ms, 150_000_000, 1_000_000, 16 << 19, 152, "paired-filter")
    peak, mhz = bench.issue_peak(152)
    assert r["bound"] == "alu" and r["kernel"] == "k_filter_hits"
    assert r["achieved"] == pytest.approx(prof["inst_executed_per_launch"] / (ms / 1e3) / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(prof["inst_executed_per_launch"] / (ms / 1e3) / peak, abs=1e-4)
    assert r["traffic"] == prof["dram_bytes_per_launch"]
    # algorithmic bytes: 3 bits per base, 8-byte offsets, the fingerprint words, 4 bytes of hits per read
    assert r["algorithmic_bytes"] == (150_000_000 * 3 + 7) // 8 + 8 * 1_000_001 + (16 << 19) + 4 * 1_000_000
    hbm_peak, _ = bench.measured_hbm_peak()
    assert r["hbm"]["frac"] == pytest.approx(r["algorithmic_bytes"] / (ms / 1e3) / 1e9 / hbm_peak, abs=1e-4)


def test_filter_roofline_falls_back_without_matching_counters(monkeypatch):
    monkeypatch.setattr(bench, "ncu_filter_kernel", lambda kernel, workload: None)
    r = bench.filter_roofline(0.5, 1_000_000, 10_000, 4096, 152, "paired-filter")
    assert r["bound"] == "hbm" and r["traffic"] is None and r["unit"] == "GB/s"


def test_stale_profile_hash_is_ignored(tmp_path, monkeypatch):
    """A counters file whose hash does not match the sources is not used."""
    src = os.path.join(ROOT, "profiles", "ncu_filter.json")
    d = json.load(open(src))
    d["source_hash"] = "0" * 16
    fake_root = tmp_path
    os.makedirs(fake_root / "profiles")
    json.dump(d, open(fake_root / "profiles" / "ncu_filter.json", "w"))
    os.symlink(os.path.join(ROOT, "paper_1712_03254_gb300"), fake_root / "paper_1712_03254_gb300")
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.ncu_filter_kernel("k_filter_hits", "paired-filter") is None


def test_stem_hbm():
    r = bench.stem_hbm(1_000_000, 900_000, 2.0)
    peak, _ = bench.measured_hbm_peak()
    algo = 16 * 1_000_000 + 72 * 900_000
    assert r["algorithmic_bytes"] == algo
    assert r["frac"] == pytest.approx(algo / 2e-3 / 1e9 / peak, abs=1e-4)
    assert bench.stem_hbm(10, 10, 0.0) is None


def test_algorithmic_bytes_of_the_mid_job_is_the_stated_11_7_per_window():
    """Reads 2 x 3 bits/base, filter and table 3 x their bytes, 12 B per result key: about 11.7 B per
    window on the mid job (1e6 x 150 bp reads, 118,157,762 windows, 2^30-bit filter, 2^24 slots,
    5,260,097 result keys)."""
    a = bench.algorithmic_bytes(150_000_000, 118_157_762, 1 << 30, 1 << 24, 5_260_097, 1)
    assert a["terms"]["reads"] == 2 * ((150_000_000 * 3 + 7) // 8)
    assert a["terms"]["filter"] == 3 * (1 << 27)
    assert a["terms"]["table"] == 3 * 16 * (1 << 24)
    assert a["terms"]["output"] == 12 * 5_260_097
    assert a["per_window"] == pytest.approx(11.71, abs=0.01)


def test_atomic_ceiling_combines_the_updates_of_a_window():
    rates = {"smem_or64_per_s": 2e12, "smem_add32_per_s": 6e12, "l2_or64_per_s": 1e11, "hbm_or64_per_s": 2e10}
    part = bench.atomic_ceiling(rates, 2)
    assert part["windows_per_s"] == pytest.approx(1 / (3 / 6e12 + 1 / 2e12), rel=1e-6)
    direct = bench.atomic_ceiling(rates, 1)
    assert direct["windows_per_s"] == pytest.approx(2e10, rel=1e-6)


def test_roofline_hbm_form_and_ceilings(monkeypatch):
    monkeypatch.setattr(bench, "ncu_kernel", lambda kernel, workload: None)

    class W:
        bloom_bits, table_slots, samples = 1 << 30, 1 << 24, [None]

    st = {"windows": 118_157_762, "strategy": 2, "result_keys": 5_260_097}
    phases = {"pass1": [1.2], "pass2": [1.15], "ingest": [0.05], "compact": [0.0], "sort": [0.49]}
    rates = {"smem_or64_per_s": 2e12, "smem_add32_per_s": 6e12, "l2_or64_per_s": 1e11, "hbm_or64_per_s": 2e10}
    r = bench.roofline_of(st, phases, 150_000_000, W, 152, 3.2, rates=rates)
    peak, _ = bench.measured_hbm_peak()
    algo = bench.algorithmic_bytes(150_000_000, st["windows"], W.bloom_bits, W.table_slots, st["result_keys"], 1)
    assert r["bound"] == "hbm" and r["kernel"] == "k_consume_q" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(algo["total"] / 1.15e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, abs=1e-4)
    assert r["step"]["frac"] == pytest.approx(algo["total"] / 3.2e-3 / 1e9 / peak, abs=1e-4)
    c = r["ceilings"]
    assert c["min_windows_per_s"] == min(c["hbm_windows_per_s"], c["atomic"]["windows_per_s"])
    assert c["step_frac_of_min"] == pytest.approx(st["windows"] / 3.2e-3 / c["min_windows_per_s"], abs=1e-4)
    assert r["implementation_bytes"] == 16 * st["windows"]

#!/usr/bin/env python3
"""Benchmark: canonical k-mers counted per second on one GB300 (plain path).

A step is one whole counting job on the "mid" workload: a 5 Mbp i.i.d.
uniform genome sequenced at 30x as 1,000,000 x 150 bp reads from both strands
with 0.5 % substitutions and 0.05 % N; k = 31, a 2^30-bit filter with 4 bits
per key, a 2^24-slot table, min_count 2.  The step is reset (filter and table
zeroed), ingest, pass 1 (filter + candidate claims), finalize (exact recount,
compaction, sort) and dump.  The unit of work is one valid window (an N-free
k-window inside one read).  Before the warm-up, kc_autotune picks the
strategy and its knobs on the same device-resident reads (untimed; the
choice and every trial are in the "tuning" field); --no-tune keeps the
library defaults.

  value  device-resident inputs, CUDA events on the library's stream
  e2e    the same step through the C ABI from pinned host buffers, the host to
         device copy of the reads and the device to host copy of the result
         inside the timed region (wall clock)

With N ranks (torchrun) the one job is sharded by key: the hash space is cut
into 64 shards and rank r owns a contiguous range of them (kc_config.own_bits,
own_lo, own_hi).  Every rank scans all the reads and counts only the keys it
owns, with its own filter slice and tables; no collective is on the data path,
and value = the job's windows / the slowest rank's time ("strong" scaling).
After the timed steps the ranks' results are gathered on rank 0, merged by key
(kc_merge_results) and compared with the whole job counted on one GPU.

The "served" field replays a Poisson stream of 256 jobs of mixed size (1-20
Mbp genomes, 10^4-2x10^6 reads, k 25 or 31, filters of 8 bits per expected
distinct k-mer) through one-at-a-time plain jobs and through the
continuous-batching server, at 0.7 and 0.9 of the plain capacity and all at
once; latencies count from each job's scheduled arrival.

The "paired" and "ooc" fields run this benchmark on the two-sample job
(2 x 10,000,000 reads, joint table; tuned) and on the out-of-core job
(100,000,000 reads, 64 partition groups spilled to pinned host memory), each
in a process of its own (--no-other-workloads skips them).

The "prune_chain" field times the paper's two-filter Prune chain (direct
strategy) on the mid job beside the direct strategy without it.

The "filter" field times the Filter unit downstream of the count on a
paired normal/tumour job of 2 x 1,000,000 reads: the selection of imbalanced
k-mers once, then per step both samples' reads rescanned against it (hits per
read and the candidate reads), device-resident and from pinned host memory.

--impl reference times the CPU oracle (single thread, as it stands) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib

import numpy as np
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "canonical k-mers counted/s per GB300 (plain vs batched/served); p99 job latency"
UNIT = "k-mers/s"
WORKLOADS = {
    "mid": ("mid: 5 Mbp uniform ACGT genome, 1,000,000 x 150 bp reads from both strands (30x), "
            "0.5% substitutions, 0.05% N; k=31 canonical uint64 keys, Bloom 2^30 bits with 4 hashes, "
            "2^24-slot open-addressing table, exact uint32 counts of k-mers seen >= 2 times"),
    "paired": ("paired: 50 Mbp uniform ACGT genome (normal) and a tumour copy with 0.1% SNVs and 1-10 bp indels "
               "at 1e-5/base; 10,000,000 x 150 bp reads per sample (30x), 0.5% substitutions, 0.05% N; k=31, "
               "Bloom 2^32 bits with 4 hashes, joint table of (normal, tumour) uint32 counts, count >= 2"),
    "ooc": ("ooc: 500 Mbp uniform ACGT genome, 100,000,000 x 150 bp reads (30x), 0.5% substitutions, 0.05% N; "
            "k=31, Bloom 2^34 bits with 4 hashes, count >= 2; 64 hash-prefix partition groups in turn, each "
            "group's sorted result spilled to pinned host memory on a side stream, merged by key at dump"),
}
CHUNK_READS = 20_000_000  # reads per kc_add_reads call
MID_SEED = 2
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------- distributed


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


OWN_BITS = 6  # hash shards the job is split into across ranks


def owner_knobs(rank: int, world: int) -> dict:
    """kc_config ownership of rank `rank` of `world`: a contiguous range of the 2^OWN_BITS hash shards
    (nothing with one rank: the handle owns every key)."""
    if world <= 1:
        return {}
    import paper_1712_03254_gb300 as kc

    lo, hi = kc.owned_shards(rank, world, OWN_BITS)
    return {"own_bits": OWN_BITS, "own_lo": lo, "own_hi": hi}


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- clocks


def _smi_id(local: int) -> str:
    """nvidia-smi id of CUDA device `local` (its UUID, robust to CUDA_VISIBLE_DEVICES)."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # older torch without the uuid property
        return str(local)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [l.strip().split(",") for l in self.out if l.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- roofline


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("kc_batch.cu", "kc_device.cuh", "kc_internal.h", "kc_kernels.cu", "kc_partition.cu")


def _kernel_source_hash():
    """Hash of the sources that define the counting kernels (and the structures they read):
    counters taken on other sources are not used."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1712_03254_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_kernel(kernel: str, workload: str = "mid"):
    """Per-launch ncu counters of a kernel on a workload from the committed profile, if taken on the current
    sources."""
    path = os.path.join(ROOT, "profiles", "ncu_kernels.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != _kernel_source_hash():
        return None
    return d.get("workloads", {}).get(workload, {}).get(kernel)


ISSUE_PER_SM_CYCLE = 4  # four warp schedulers per SM, one warp instruction each per cycle


def issue_peak(sm_count: int):
    """Warp instructions per second the SMs can issue at the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return sm_count * ISSUE_PER_SM_CYCLE * mhz * 1e6, mhz


def algorithmic_bytes(n_bases: int, windows: int, bloom_bits: int, table_slots: int, result_keys: int,
                      n_samples: int) -> dict:
    """Compulsory DRAM bytes of one counting job (two passes over the reads), term by term:
      reads   3 bits per base (2-bit code + N mask) read once per pass
      filter  zeroed, then read and written once: 3 x its bytes
      table   zeroed, updated, read by the compaction: 3 x its bytes (16 B slots)
      output  8 B key + 4 B count per sample per result key
    The materialised hash stream of the partitioned strategy (8 B per window
    written and read per grouping pass) is implementation traffic, never
    counted here."""
    terms = {"reads": 2 * ((n_bases * 3 + 7) // 8), "filter": 3 * (bloom_bits // 8), "table": 3 * 16 * table_slots,
             "output": (8 + 4 * n_samples) * result_keys}
    total = sum(terms.values())
    return {"total": int(total), "per_window": round(total / max(1, windows), 3), "terms": terms}


def atomic_ceiling(rates: dict, strategy: int) -> dict:
    """Windows per second the random updates allow.  Per window the partitioned
    path makes 3 random shared-memory 32-bit adds (extraction histogram,
    scatter stage fill, recount) and 1 shared-memory 64-bit OR (the filter
    slice); the direct strategy makes 1 global 64-bit OR into the filter
    (beyond L2) and its table probes."""
    if strategy == 1:
        per = {"hbm_or64": 1}
        t = 1.0 / rates["hbm_or64_per_s"]
    else:
        per = {"smem_add32": 3, "smem_or64": 1}
        t = 3.0 / rates["smem_add32_per_s"] + 1.0 / rates["smem_or64_per_s"]
    return {"windows_per_s": round(1.0 / t, 1), "updates_per_window": per,
            "rates_per_s": {k: round(v, 1) for k, v in rates.items()}}


def roofline_of(st, phases, n_bases, w, sm_count, step_ms, workload="mid", consume_launches=1, rates=None):
    """Roofline entry of the kernel that takes the most device time, against HBM.

    Partitioned strategy: the consumer k_consume_q (the largest single kernel;
    the "pass2" phase events bracket exactly its one launch).  Direct
    strategy: the larger of k_pass1 / k_pass2.  achieved = the job's
    algorithmic bytes per window (algorithmic_bytes: reads, filter, the
    configuration's table, output) x the windows one launch processes / the
    launch's mean CUDA-event time.  Beside it: the same bytes over the whole
    step, the atomic ceiling (atomic_ceiling) and HBM ceiling in windows/s,
    and, when the committed ncu counters match the current sources, the
    kernel's DRAM traffic and its fraction of the SM issue limit (a diagnosis
    of what binds it, not the headline).
    """
    import statistics as _st

    W = st["windows"]
    mean = {k: _st.mean(v) for k, v in phases.items()}
    algo = algorithmic_bytes(n_bases, W, w.bloom_bits, w.table_slots, st["result_keys"], len(w.samples))
    if st["strategy"] == 1:
        phase = "pass1" if mean["pass1"] >= mean["pass2"] else "pass2"
        kernel = "k_pass1" if phase == "pass1" else "k_pass2"
        ms = mean[phase]
    else:
        phase, kernel = "pass2", "k_consume_q"
        ms = mean[phase] / consume_launches  # with spill the consumer runs once per partition group
    per_launch = algo["total"] / (consume_launches if st["strategy"] != 1 else 1)
    peak, peak_kind = measured_hbm_peak()
    achieved = per_launch / (ms / 1e3) / 1e9
    step_achieved = algo["total"] / (step_ms / 1e3) / 1e9
    prof = ncu_kernel(kernel, workload)
    out = {"bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1), "peak": peak,
           "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
           "traffic": prof["dram_bytes_per_launch"] if prof else None,
           "algorithmic_bytes": int(per_launch), "algorithmic_bytes_per_window": algo["per_window"],
           "algorithmic_terms": algo["terms"], "ms_per_launch": round(ms, 4),
           "implementation_bytes": (16 * W if st["strategy"] != 1 else 0),
           "step": {"ms": round(step_ms, 4), "achieved": round(step_achieved, 1),
                    "frac": round(step_achieved / peak, 4)}}
    hbm_windows = peak * 1e9 / algo["per_window"]
    ceil = {"hbm_windows_per_s": round(hbm_windows, 1)}
    if rates:
        a = atomic_ceiling(rates, st["strategy"])
        ceil["atomic"] = a
        lo = min(hbm_windows, a["windows_per_s"])
        ceil["min_windows_per_s"] = round(lo, 1)
        ceil["bound_by"] = "atomic" if a["windows_per_s"] < hbm_windows else "hbm"
        ceil["step_frac_of_min"] = round(W / (step_ms / 1e3) / lo, 4)
    out["ceilings"] = ceil
    if prof is not None:
        ipk, mhz = issue_peak(sm_count)
        ach = prof["inst_executed_per_launch"] / (ms / 1e3)
        out["issue"] = {"achieved": round(ach / 1e9, 1), "peak": round(ipk / 1e9, 1), "unit": "G warp instructions/s",
                        "frac": round(ach / ipk, 4),
                        "peak_source": f"derived: {sm_count} SMs x {ISSUE_PER_SM_CYCLE} warp instructions/cycle x "
                                       f"{mhz:.0f} MHz",
                        "instructions_per_launch": prof["inst_executed_per_launch"]}
    return out


FILTER_SOURCES = ("kc_filter.cu", "kc_device.cuh", "kc_internal.h", "kc_kernels.cu")
FILTER_SPEC = (1, 4, 0, 0)  # tumour sample 1: k-mers seen >= 4 times in the tumour and never in the normal
FILTER_WORKLOAD = ("paired normal/tumour at 1/10 size: 5 Mbp uniform ACGT genome and a tumour copy with 0.1% SNVs "
                   "and 1-10 bp indels at 1e-5/base, 1,000,000 x 150 bp reads per sample (30x), 0.5% substitutions, "
                   "0.05% N; k=31, Bloom 2^32 bits, 4 hashes, count >= 2; selection count[tumour] >= 4 and "
                   "count[normal] = 0; both samples rescanned")


def ncu_filter_kernel(kernel: str, workload: str):
    """Per-launch ncu counters of a filter-unit kernel, if taken on the current filter sources."""
    path = os.path.join(ROOT, "profiles", "ncu_filter.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1712_03254_gb300", "csrc")
    for f in FILTER_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    if d.get("source_hash") != h.hexdigest()[:16]:
        return None
    return d.get("workloads", {}).get(workload, {}).get(kernel)


def filter_roofline(ms_per_launch, n_bases, n_reads, table_bytes, sm_count, workload):
    """Roofline of k_filter_hits (one launch per read set).  Algorithmic bytes:
    2 bits (packed base) + 1 bit (valid-window bit) per base, the 8-byte read
    offsets read once, the selection's fingerprint words read once, 4 bytes of
    hit count written per read."""
    algo = (n_bases * 3 + 7) // 8 + 8 * (n_reads + 1) + table_bytes + 4 * n_reads
    peak, peak_kind = measured_hbm_peak()
    hbm_achieved = algo / (ms_per_launch / 1e3) / 1e9
    hbm = {"achieved": round(hbm_achieved, 1), "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
           "frac": round(hbm_achieved / peak, 4)}
    prof = ncu_filter_kernel("k_filter_hits", workload)
    if prof is None:
        return {"bound": "hbm", "kernel": "k_filter_hits", **hbm, "traffic": None, "algorithmic_bytes": int(algo),
                "ms_per_launch": round(ms_per_launch, 4)}
    ipk, mhz = issue_peak(sm_count)
    achieved = prof["inst_executed_per_launch"] / (ms_per_launch / 1e3)
    return {"bound": "alu", "kernel": "k_filter_hits", "achieved": round(achieved / 1e9, 1),
            "peak": round(ipk / 1e9, 1),
            "peak_source": f"derived: {sm_count} SMs x {ISSUE_PER_SM_CYCLE} warp instructions/cycle x {mhz:.0f} MHz",
            "unit": "G warp instructions/s", "frac": round(achieved / ipk, 4),
            "traffic": prof["dram_bytes_per_launch"], "algorithmic_bytes": int(algo),
            "ms_per_launch": round(ms_per_launch, 4), "instructions_per_launch": prof["inst_executed_per_launch"],
            "hbm": hbm}


def run_chain_bench(w, chunks_d, stream, steps: int, warmup: int, flush):
    """The paper's two-filter Prune chain (direct strategy) on the same job,
    beside the direct strategy without it: device-resident inputs, CUDA events
    on the library's stream, the same L2 flush between steps."""
    import torch

    import paper_1712_03254_gb300 as kc

    out = {}
    for name, chain in (("direct", False), ("direct_prune_chain", True)):
        c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, table_slots=w.table_slots,
                           strategy="direct", timing=True, prune_chain=chain, stream=stream)

        def job():
            c.reset()
            for s_i, p_, o_, m_ in chunks_d:
                c.add_reads(s_i, p_, o_, m_)
            c.finalize()

        for _ in range(max(1, warmup)):
            job()
        ms, phases = [], {"pass1": [], "pass2": []}
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            job()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = c.stats()
            for k in phases:
                phases[k].append(st["ms_" + k])
        st = c.stats()
        out[name] = {"ms_per_job": round(statistics.mean(ms), 4),
                     "k_mers_per_s": round(st["windows"] / (statistics.mean(ms) / 1e3), 1),
                     "pass1_ms": round(statistics.mean(phases["pass1"]), 4),
                     "pass2_ms": round(statistics.mean(phases["pass2"]), 4),
                     "result_keys": st["result_keys"], "table_keys": st["table_keys"]}
        c.close()
    return out


def stem_hbm(n_keys: int, n_items: int, ms: float):
    """HBM roofline of the stem-table build (all its kernels): algorithmic bytes
    = the result read once (16 B per key) + the items written (72 B each)."""
    if ms <= 0:
        return None
    algo = 16 * n_keys + 72 * n_items
    peak, kind = measured_hbm_peak()
    achieved = algo / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "peak_source": kind, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "algorithmic_bytes": algo}


def run_filter_bench(dev, stream, steps: int, warmup: int, flush):
    """Filter unit on a paired job: selection once, then every timed step
    rescans both samples' device-resident reads (kc_filter_reads, hits and
    candidate list into device buffers); e2e does the same from pinned host
    reads into pinned host hits."""
    import torch

    import paper_1712_03254_gb300 as kc
    import synth

    w = synth.paired(scale=0.1)
    c = kc.KmerCounter(w.k, 2, w.bloom_bits, w.n_hashes, w.min_count, timing=True, stream=stream)
    ins_h, ins_d, outs_d, outs_h = [], [], [], []
    for s_i, rs in enumerate(w.samples):
        packed, mask = kc.pack_ascii(rs.ascii)
        offsets = np.ascontiguousarray(rs.offsets, dtype=np.uint64)
        hp = tuple(torch.from_numpy(a.view(np.int64)).pin_memory() for a in (packed, offsets, mask))
        ins_h.append(hp)
        ins_d.append(tuple(t.to(dev) for t in hp))
        outs_d.append((torch.empty(rs.n_reads, dtype=torch.int32, device=dev),
                       torch.empty(rs.n_reads, dtype=torch.int64, device=dev)))
        outs_h.append((torch.empty(rs.n_reads, dtype=torch.int32).pin_memory(),
                       torch.empty(rs.n_reads, dtype=torch.int64).pin_memory()))
    torch.cuda.synchronize()
    for s_i, (p_, o_, m_) in enumerate(ins_d):
        c.add_reads(s_i, p_, o_, m_)
    c.finalize()
    t0 = time.perf_counter()
    n_sel = c.filter_select(*FILTER_SPEC)
    select_wall_ms = (time.perf_counter() - t0) * 1e3
    st0 = c.stats()

    def step(ins, outs):
        n_c = 0
        for (p_, o_, m_), (hits, cand) in zip(ins, outs):
            n_c += c.filter_reads(p_, o_, m_, hits=hits, candidates=cand)[2]
        return n_c

    for _ in range(warmup):
        step(ins_d, outs_d)
    torch.cuda.synchronize()
    base = c.stats()
    ms, n_cand = [], 0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # cold L2: the reads and the table are below its size
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n_cand = step(ins_d, outs_d)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = c.stats()
    windows = (st["filter_windows"] - base["filter_windows"]) // steps
    kernel_ms = (st["ms_filter_reads"] - base["ms_filter_reads"]) / (steps * 2)
    launches = (st["launches"] - base["launches"]) // steps
    for _ in range(max(1, warmup)):
        step(ins_h, outs_h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step(ins_h, outs_h)
    e2e_s = (time.perf_counter() - t0) / steps
    # the host hits must be the device ones
    for (hh, _), (dh, _) in zip(outs_h, outs_d):
        assert torch.equal(hh, dh.cpu()), "filter: host and device hits differ"
    # the stem-grouped table of the same result (built once on the device, then copied out)
    b0 = c.stats()
    t0 = time.perf_counter()
    stems = c.export_stems()
    stems_wall_ms = (time.perf_counter() - t0) * 1e3
    stems_ms = c.stats()["ms_stems"] - b0["ms_stems"]
    n_reads = sum(rs.n_reads for rs in w.samples)
    lb = 8  # the selection's lookup table: 2^lb buckets of four 32-bit fingerprints, 2^lb >= 2 x selected keys
    while (1 << lb) < 2 * n_sel:
        lb += 1
    table_bytes = 16 << lb  # the fingerprint words (the 64-bit codes are read only on a fingerprint match)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {
        "workload": FILTER_WORKLOAD, "spec": dict(zip(("tumor", "min_tumor", "max_normal", "ratio"), FILTER_SPEC)),
        "selected_keys": n_sel, "result_keys": st0["result_keys"], "candidate_reads": n_cand,
        "reads": n_reads, "windows_per_step": int(windows),
        "value": round(windows / (statistics.mean(ms) / 1e3), 1), "unit": "windows rescanned/s",
        "ms_per_step": round(statistics.mean(ms), 4), "kernel_ms": round(kernel_ms, 4),
        "select_ms": round(st0["ms_filter_select"], 4), "select_wall_ms": round(select_wall_ms, 3),
        "gpu_launches_per_step": int(launches),
        "roofline": filter_roofline(kernel_ms, w.n_bases // 2, n_reads // 2, table_bytes, sm_count, "paired-filter"),
        "e2e": {"value": round(windows / e2e_s, 1), "unit": "windows rescanned/s",
                "h2d_bytes_per_step": int(sum(t.numel() * 8 for ins in ins_h for t in ins)),
                "d2h_bytes_per_step": int(sum(h.numel() * 4 for h, _ in outs_h) + n_cand * 8),
                "ms_per_step": round(e2e_s * 1e3, 4)},
        "l2": "256 MiB written between timed steps (outside the step events)",
        "stems": {"items": int(stems.size), "result_keys": st0["result_keys"], "device_ms": round(stems_ms, 4),
                  "wall_ms": round(stems_wall_ms, 3),
                  "keys_per_s": round(st0["result_keys"] / (stems_ms / 1e3), 1) if stems_ms > 0 else None,
                  "hbm": stem_hbm(st0["result_keys"], int(stems.size), stems_ms)},
    }
    c.close()
    return out


# ---------------------------------------------------------------- workloads


def make_inputs(workload: str = "mid"):
    """The workload's read sets (every rank of a sharded run holds all of them)."""
    import synth

    if workload == "mid":
        return synth.mid(seed=MID_SEED)
    return synth.WORKLOADS[workload]()


def oracle_rate(w, n_reads: int):
    """Windows/s of the oracle on the first n_reads reads (single thread)."""
    import oracle

    rs = w.samples[0].slice(0, n_reads)
    o = oracle.Oracle(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count)
    t = time.perf_counter()
    o.add_reads(0, rs)
    o.result()
    dt = time.perf_counter() - t
    return o.windows, dt


def pick_sample_reads(w, seconds: float) -> int:
    win, dt = oracle_rate(w, 5000)
    per_read = max(1.0, win / 5000.0)
    rate = win / max(dt, 1e-6)
    return int(max(5000, min(w.samples[0].n_reads, seconds * rate / per_read)))


# ---------------------------------------------------------------- kc arm


def run_kc(args):
    import numpy as np
    import torch

    import paper_1712_03254_gb300 as kc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    # the library's work and the step events share one stream (a real one:
    # the legacy default stream would give the handle a stream of its own)
    stream = torch.cuda.Stream()

    w = make_inputs(args.workload)
    rs = w.samples[0]
    n_samples = len(w.samples)
    spill = bool(w.extra.get("spill_parts"))
    # each sample in chunks of at most CHUNK_READS reads: pinned host copies
    # (e2e) and device-resident copies (value)
    chunks_h, chunks_d = [], []
    for s_i, r_s in enumerate(w.samples):
        for r0 in range(0, max(1, r_s.n_reads), CHUNK_READS):
            part = r_s if r_s.n_reads <= CHUNK_READS else r_s.slice(r0, min(r_s.n_reads, r0 + CHUNK_READS))
            packed, mask = kc.pack_ascii(part.ascii)
            offsets = np.ascontiguousarray(part.offsets, dtype=np.uint64)
            hp = (torch.from_numpy(packed.view(np.int64)).pin_memory(),
                  torch.from_numpy(offsets.view(np.int64)).pin_memory(),
                  torch.from_numpy(mask.view(np.int64)).pin_memory())
            chunks_h.append((s_i, *hp))
            chunks_d.append((s_i, *(t.to(dev) for t in hp)))
            del packed, mask
    total_bases = w.n_bases
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    # autotune on this job's own device-resident reads (outside the timed
    # region) unless knobs were given on the command line
    tuning = None
    knobs = dict(strategy=args.strategy, scatter_mode=args.scatter_mode, ctas_per_sm=args.ctas_per_sm,
                 part_bits=args.part_bits, smem_table_log2=0)
    if (not args.no_tune and not spill and args.strategy == "auto"
            and not (args.scatter_mode or args.ctas_per_sm or args.part_bits)):
        t0 = time.perf_counter()
        best, trials = kc.autotune(w.k, n_samples, w.bloom_bits, w.n_hashes, w.min_count, chunks_d, reps=3)
        knobs = dict(strategy=best["strategy"], scatter_mode=best["scatter_mode"], ctas_per_sm=best["ctas_per_sm"],
                     part_bits=best["part_bits"], smem_table_log2=best["smem_table_log2"])
        short = lambda cfg: {k: v for k, v in cfg.items() if k in ("strategy", "part_bits", "smem_table_log2",
                                                                    "ctas_per_sm")}
        tuning = {"best": short(best), "seconds": round(time.perf_counter() - t0, 2),
                  "trials": [[short(cfg), round(ms, 3)] for cfg, ms in trials]}
    if spill:
        knobs["strategy"] = "partitioned"
    knobs.update(owner_knobs(rank, world))  # N > 1: this rank's hash-shard range of the one job
    if world > 1:
        knobs["strategy"] = "partitioned"
    c = kc.KmerCounter(w.k, n_samples, w.bloom_bits, w.n_hashes, w.min_count, table_slots=w.table_slots,
                       timing=True, spill=spill, stream=stream, **knobs)

    # size result buffers with one untimed job
    for s_i, p_, o_, m_ in chunks_d:
        c.add_reads(s_i, p_, o_, m_)
    c.finalize()
    n_res = c.result_size()
    h_keys = torch.empty(n_res, dtype=torch.int64).pin_memory()
    h_counts = torch.empty((n_res, n_samples), dtype=torch.int32).pin_memory()
    if spill:  # an out-of-core result lands in host memory
        d_keys, d_counts = h_keys, h_counts
    else:
        d_keys = torch.empty(n_res, dtype=torch.int64, device=dev)
        d_counts = torch.empty((n_res, n_samples), dtype=torch.int32, device=dev)

    def job(chunks, keys, counts):
        c.reset()
        for s_i, p_, o_, m_ in chunks:
            c.add_reads(s_i, p_, o_, m_)
        c.finalize()
        c.dump(keys, counts)

    # warm-up
    for _ in range(args.warmup):
        job(chunks_d, d_keys, d_counts)
    torch.cuda.synchronize()

    clocks = ClockSampler(_smi_id(local))
    clocks.start()
    time.sleep(0.3)
    phases = {"ingest": [], "pass1": [], "pass2": [], "compact": [], "sort": []}
    launches = 0
    windows = None
    step_ms = []
    barrier(dist)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # write 256 MiB between steps: the next step starts with a cold L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        job(chunks_d, d_keys, d_counts)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = c.stats()
        for k in phases:
            phases[k].append(st["ms_" + k])
        launches += st["launches"]
        windows = st["windows"]
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()

    total_ms = sum(step_ms)
    max_total_ms = reduce_max(total_ms, dist, dev)
    # every rank scans all the job's windows (and counts the keys it owns):
    # the work is the job's windows, whatever the number of ranks
    all_windows = float(windows * args.steps)
    value = all_windows / (max_total_ms / 1e3)

    # e2e: pinned host inputs and outputs through the C ABI, wall clock
    h2d = int(sum(t.numel() * 8 for ch in chunks_h for t in ch[1:]))
    d2h = int(n_res * 8 + n_res * 4 * n_samples)
    for _ in range(max(1, args.warmup)):
        job(chunks_h, h_keys, h_counts)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        job(chunks_h, h_keys, h_counts)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist, dev)
    e2e_value = all_windows / e2e_s
    # the e2e result must be the device result
    if not spill:
        assert np.array_equal(h_keys.numpy(), d_keys.cpu().numpy()), "e2e and device dumps differ (keys)"
        assert np.array_equal(h_counts.numpy(), d_counts.cpu().numpy()), "e2e and device dumps differ (counts)"

    # N > 1: the owners' results, merged by key on rank 0, must be the whole job's
    merged_check = None
    if dist is not None:
        gathered = [None] * world
        dist.all_gather_object(gathered, (h_keys.numpy().copy(), h_counts.numpy().view(np.uint32).copy()))
        if rank == 0:
            mk, mc = kc.merge_results(gathered, n_samples)
            whole = kc.KmerCounter(w.k, n_samples, w.bloom_bits, w.n_hashes, w.min_count, table_slots=w.table_slots,
                                   spill=spill, stream=stream,
                                   **{k: v for k, v in knobs.items() if not k.startswith("own_")})
            for s_i, p_, o_, m_ in chunks_d:
                whole.add_reads(s_i, p_, o_, m_)
            whole.finalize()
            wk, wc = whole.dump()
            whole.close()
            merged_check = bool(np.array_equal(mk, wk) and np.array_equal(mc, wc))
            assert merged_check, "merged owner results differ from the whole job"

    # roofline of the dominant kernel (per-launch means over the timed steps),
    # with the measured random-atomic ceilings beside it
    st = c.stats()
    try:
        rates = kc.atomic_ceilings(stream)
    except kc.KcError:
        rates = None
    roofline = roofline_of(st, phases, total_bases, w, torch.cuda.get_device_properties(dev).multi_processor_count,
                           max_total_ms / args.steps, args.workload, min(st["partitions"], 64) if spill else 1, rates)
    strategy = {1: "direct", 2: "partitioned"}.get(st["strategy"], "?")

    # CPU baseline: the oracle on a bounded sample (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = pick_sample_reads(w, args.cpu_seconds)
        win, dt = oracle_rate(w, n_s)
        cpu = {"value": round(win / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_s:,} of {rs.n_reads:,} reads of the {args.workload} workload ({win:,} windows, "
                         f"{dt:.1f} s, single-threaded C++ oracle, {os.cpu_count()} host cores present)"}

    filt = chain = None
    if rank == 0 and world == 1 and not args.no_filter and args.workload == "mid":
        filt = run_filter_bench(dev, stream, args.steps, args.warmup, flush)
        chain = run_chain_bench(w, chunks_d, stream, min(args.steps, 5), args.warmup, flush)

    # the two-sample and out-of-core configurations, each in a process of its own
    others = {}
    if rank == 0 and world == 1 and args.workload == "mid" and not args.no_other_workloads:
        others["paired"] = run_workload_subprocess("paired", min(args.steps, 5), 3)
        others["ooc"] = run_workload_subprocess("ooc", 3, 3, ["--part-bits", "18"])

    served = None
    if rank == 0 and world == 1 and not args.no_served and args.workload == "mid":
        # the mid job's buffers are not needed any more; the stream of jobs
        # runs in a process of its own, like a server process would (in this
        # one, the host memory the oracle and the mid job touched slows the
        # plain and served jobs alike by 20-30 %)
        c.close()
        del chunks_d, d_keys, d_counts, flush
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        served = run_served_subprocess(args.served_jobs, args.served_max_reads)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(max_total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded genome and reads)",
            "config": {"workload": WORKLOADS[args.workload], "windows_per_job": windows, "result_keys": n_res,
                       "l2": "256 MiB written between timed steps (outside the step events)"
                             + ("; inputs larger than L2" if args.workload != "mid" else ""),
                       "parallelism": (f"one job sharded over {world} GPUs by hash range ({1 << OWN_BITS} shards, "
                                       "a contiguous range per rank, reads replicated, no collective on the data "
                                       "path); e2e and result_keys are rank 0's; results merged by key after the "
                                       "timed steps" if world > 1 else "1 GPU")},
            "merged_equals_whole_job": merged_check,
            "strategy": strategy,
            "tuning": tuning,
            "phase_ms": {k: round(statistics.mean(v), 4) for k, v in phases.items()},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_s * 1e3 / args.steps, 4)},
            "clocks": clk,
            "gpu_launches": int(launches),
            "served": served,
            "filter": filt,
            "prune_chain": chain,
            **others,
        }
        print(json.dumps(line), flush=True)
    c.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- served stream


def _served_jobs(n_jobs: int, max_reads: int):
    """Job shapes of the served stream with their packed reads (host memory;
    the ASCII reads are dropped once packed)."""
    import paper_1712_03254_gb300 as kc
    import synth

    jobs = []
    for spec in synth.served_specs(n_jobs, 1.0, max_reads):
        w = synth.served_job(spec)
        rs = w.samples[0]
        packed, mask = kc.pack_ascii(rs.ascii)
        jobs.append({"k": w.k, "bloom_bits": w.bloom_bits, "n_hashes": w.n_hashes, "min_count": w.min_count,
                     "packed": packed, "mask": mask, "offsets": np.ascontiguousarray(rs.offsets), "windows": None})
    return jobs


def _digest(keys, counts):
    """Size and order-sensitive checksums of a result (compared instead of keeping every result)."""
    k = np.asarray(keys, dtype=np.uint64)
    pos = np.arange(1, k.size + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return (int(k.size), int(np.bitwise_xor.reduce(k * pos)) if k.size else 0,
                int(np.asarray(counts, dtype=np.uint64).sum()))


def _plain_job(kc, j):
    c = kc.KmerCounter(j["k"], 1, j["bloom_bits"], j["n_hashes"], j["min_count"], strategy="partitioned")
    c.add_reads(0, j["packed"], j["offsets"], j["mask"])
    c.finalize()
    keys, counts = c.dump()
    win = c.stats()["windows"]
    c.close()
    return _digest(keys, counts), win


def run_served_trace(n_jobs: int, max_reads: int, loads=(0.7, 0.9), budget_bytes=64 << 30):
    """The same Poisson trace through one-at-a-time plain launches and the
    continuous-batching server, at offered loads relative to plain capacity."""
    import threading

    import paper_1712_03254_gb300 as kc

    jobs = _served_jobs(n_jobs, max_reads)
    # plain capacity: the jobs back to back, one at a time
    for j in jobs[:2]:
        _plain_job(kc, j)
    t0 = time.perf_counter()
    ref = []
    for j in jobs:
        dig, win = _plain_job(kc, j)
        j["windows"] = win
        ref.append(dig)
    plain_cap = len(jobs) / (time.perf_counter() - t0)
    windows = sum(j["windows"] for j in jobs)
    rng = np.random.default_rng(99)
    gaps = rng.exponential(1.0, size=len(jobs))
    out = {"jobs": len(jobs), "max_reads": max_reads, "windows": int(windows),
           "plain_capacity_jobs_per_s": round(plain_cap, 2), "loads": []}
    for load in loads:
        arr = np.concatenate([[0.0], np.cumsum(gaps[1:])]) / (load * plain_cap)
        # plain: one worker, FIFO, one job at a time
        lat_plain = []
        start = time.perf_counter()
        for i, j in enumerate(jobs):
            now = time.perf_counter() - start
            if now < arr[i]:
                time.sleep(arr[i] - now)
            _plain_job(kc, j)
            lat_plain.append((time.perf_counter() - start - arr[i]) * 1e3)
        span_plain = time.perf_counter() - start
        # served: the same arrivals submitted to the server
        srv = kc.KcServer(budget_bytes, max_batch=64)
        ids = [None] * len(jobs)
        start = time.perf_counter()

        late = [0.0] * len(jobs)  # submit time after the scheduled arrival
        submitted = [threading.Event() for _ in jobs]

        def feeder():
            for i, j in enumerate(jobs):
                now = time.perf_counter() - start
                if now < arr[i]:
                    time.sleep(arr[i] - now)
                late[i] = time.perf_counter() - start - arr[i]
                ids[i] = srv.submit(j["k"], j["bloom_bits"], j["n_hashes"], j["min_count"],
                                    [(j["packed"], j["offsets"], j["mask"])])
                submitted[i].set()

        same = [True]
        lat_served = [0.0] * len(jobs)

        def collector():  # takes each result as it completes, as a client would
            for i in range(len(jobs)):
                submitted[i].wait()
                _, lat = srv.wait(ids[i], timeout_s=600)
                lat_served[i] = lat + late[i] * 1e3  # from the scheduled arrival, as for plain
                keys, counts = srv.result(ids[i])
                same[0] &= _digest(keys, counts) == ref[i]

        threads = [threading.Thread(target=feeder), threading.Thread(target=collector)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        same = same[0]
        span_served = time.perf_counter() - start
        st = srv.stats()
        srv.close()
        out["loads"].append({
            "offered_load": load, "arrival_rate_jobs_per_s": round(load * plain_cap, 2),
            "plain": {"jobs_per_s": round(len(jobs) / span_plain, 2),
                      "p50_ms": round(float(np.percentile(lat_plain, 50)), 3),
                      "p99_ms": round(float(np.percentile(lat_plain, 99)), 3)},
            "served": {"jobs_per_s": round(len(jobs) / span_served, 2),
                       "p50_ms": round(float(np.percentile(lat_served, 50)), 3),
                       "p99_ms": round(float(np.percentile(lat_served, 99)), 3),
                       "mean_batch": round(st["mean_batch"], 2),
                       "k_mers_per_s": round(windows / span_served, 1),
                       "stage_ms": {x: round(st["mean_" + x + "_ms"], 3)
                                    for x in ("queue", "ingest", "batch_wait", "finalize")}},
            "results_equal_alone": same,
        })
    # saturation: every job submitted at once, each result taken into the
    # client's memory as soon as it completes by two collector threads (taking
    # a result returns its pinned block to the server's pool); one untimed
    # pass first, which also checks every result against the plain run, so
    # the timed one runs with warm pinned result blocks, captured graphs and
    # recycled handles
    sat_same = True
    for timed in (False, True):
        srv = kc.KcServer(budget_bytes, max_batch=64)
        start = time.perf_counter()
        ids = [srv.submit(j["k"], j["bloom_bits"], j["n_hashes"], j["min_count"],
                          [(j["packed"], j["offsets"], j["mask"])]) for j in jobs]
        digests = [None] * len(ids)

        def collect(part):
            for i in part:
                srv.wait(ids[i], timeout_s=600)
                keys, counts = srv.result(ids[i])
                if not timed:
                    digests[i] = _digest(keys, counts)

        threads = [threading.Thread(target=collect, args=(range(c, len(ids), 2),)) for c in range(2)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        span = time.perf_counter() - start
        st = srv.stats()
        srv.close()
        if not timed:
            sat_same = all(d == r for d, r in zip(digests, ref))
    out["saturated"] = {"served_jobs_per_s": round(len(jobs) / span, 2), "plain_jobs_per_s": round(plain_cap, 2),
                        "results_equal_alone": bool(sat_same),
                        "served_k_mers_per_s": round(windows / span, 1),
                        "plain_k_mers_per_s": round(windows * plain_cap / len(jobs), 1),
                        "p99_ms": round(st["p99_ms"], 3), "mean_batch": round(st["mean_batch"], 2),
                        "stage_ms": {x: round(st["mean_" + x + "_ms"], 3)
                                     for x in ("queue", "ingest", "batch_wait", "finalize")},
                        "per_batch_ms": {x: round(st["mean_batch_" + x + "_ms"], 3)
                                         for x in ("finalize", "copy", "release")},
                        "ingest_ms": {x: round(st["mean_ingest_" + x + "_ms"], 3) for x in ("handle", "add")},
                        "reused_handles": st["reused_handles"]}
    return out


def run_workload_subprocess(workload: str, steps: int, warmup: int, extra=()):
    """This benchmark on another workload, in a fresh Python process: its JSON line (or the error)."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", workload, "--steps", str(steps), "--warmup",
           str(warmup), "--no-cpu-baseline", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        return {"error": r.stderr[-2000:]}
    line = json.loads(r.stdout.strip().splitlines()[-1])
    keep = ("value", "unit", "ms_per_step", "config", "strategy", "tuning", "phase_ms", "roofline", "e2e", "clocks",
            "gpu_launches", "steps", "warmup")
    return {k: line.get(k) for k in keep}


def run_served_subprocess(n_jobs: int, max_reads: int):
    """run_served_trace in a fresh Python process; its result (a JSON line)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.run_served_trace(%d, %d)))" % (ROOT, n_jobs, max_reads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("served stream failed:\n" + r.stderr[-4000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------- reference arm


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = make_inputs(args.workload)
    budget_s = args.ref_seconds
    per_step = budget_s / max(1, args.steps + args.warmup)
    n_s = pick_sample_reads(w, per_step)
    for _ in range(args.warmup):
        oracle_rate(w, n_s)
    times, wins = [], 0
    for _ in range(args.steps):
        win, dt = oracle_rate(w, n_s)
        times.append(dt)
        wins = win
    total = sum(times)
    value = wins * args.steps / total
    sample = (f"first {n_s:,} of {w.samples[0].n_reads:,} reads of the {args.workload} workload per step "
              f"({wins:,} windows), "
              f"single-threaded C++ oracle, {os.cpu_count()} host cores present")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded genome and reads)", "config": {"workload": WORKLOADS[args.workload]},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["kc", "reference"], default="kc")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0, help="--impl reference: CPU seconds for the whole run")
    ap.add_argument("--strategy", choices=["auto", "direct", "partitioned"], default="auto")
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream comparison")
    ap.add_argument("--no-filter", action="store_true", help="skip the Filter-unit measurement")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the paired and ooc fields of the default (mid) line")
    ap.add_argument("--filter-only", action="store_true",
                    help="print only the Filter-unit measurement (one JSON object), for profiling it alone")
    ap.add_argument("--served-jobs", type=int, default=256)
    ap.add_argument("--served-max-reads", type=int, default=2_000_000)
    ap.add_argument("--scatter-mode", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--part-bits", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="library defaults instead of kc_autotune's choice")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mid",
                    help="mid (the default bench line), paired (two samples, joint table) or ooc (spill)")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.filter_only:
        import torch

        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        print(json.dumps(run_filter_bench(dev, torch.cuda.Stream(), args.steps, args.warmup, flush)), flush=True)
    else:
        run_kc(args)


if __name__ == "__main__":
    main()

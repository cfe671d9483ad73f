"""GB300 k-mer frequency counting: Python binding of libkc (include/kc.h).

The binding only marshals arguments: every step of the counting path runs in
the library's CUDA kernels.  There is no CPU fallback; if libkc.so is missing
and cannot be built, loading fails with an error.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); the
library detects where each pointer lives.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["KmerCounter", "KcBatch", "KcServer", "KcError", "pack_ascii", "lib", "build", "Config", "Stats",
           "merge_results", "owned_shards", "atomic_ceilings",
           "FilterSpec", "ITEM16", "STEM_ITEM", "autotune", "tune_lookup", "tune_cache_save", "tune_cache_load", "tune_cache_clear"]

_lock = threading.Lock()
_lib = None

STATUS = ["KC_OK", "KC_ERR_ARG", "KC_ERR_STATE", "KC_ERR_OOM_DEVICE", "KC_ERR_OOM_HOST", "KC_ERR_CUDA",
          "KC_ERR_TIMEOUT", "KC_ERR_CAPACITY", "KC_ERR_INTERNAL"]


class KcError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{where}: {self.name}: {message}")


class Config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("part_bits", ctypes.c_uint32),
                ("table_slots", ctypes.c_uint64), ("spill", ctypes.c_uint32), ("timing", ctypes.c_uint32),
                ("strategy", ctypes.c_uint32), ("smem_table_log2", ctypes.c_uint32),
                ("scatter_mode", ctypes.c_uint32), ("split_max", ctypes.c_uint32), ("prune_chain", ctypes.c_uint32),
                ("own_bits", ctypes.c_uint32), ("own_lo", ctypes.c_uint32), ("own_hi", ctypes.c_uint32),
                ("device_budget", ctypes.c_uint64), ("batched_ingest", ctypes.c_uint32),
                ("reserved32", ctypes.c_uint32)]


assert ctypes.sizeof(Config) == 80


class Stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_uint64), ("bases", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("table_keys", ctypes.c_uint64), ("result_keys", ctypes.c_uint64),
                ("spilled_bytes", ctypes.c_uint64), ("partitions", ctypes.c_uint32),
                ("table_log2", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("ms_ingest", ctypes.c_double), ("ms_pass1", ctypes.c_double), ("ms_pass2", ctypes.c_double),
                ("ms_compact", ctypes.c_double), ("ms_sort", ctypes.c_double), ("strategy", ctypes.c_uint32),
                ("fallback_partitions", ctypes.c_uint32), ("split_partitions", ctypes.c_uint32),
                ("split_level", ctypes.c_uint32), ("ms_filter_select", ctypes.c_double),
                ("ms_filter_reads", ctypes.c_double), ("filter_selected", ctypes.c_uint64),
                ("filter_windows", ctypes.c_uint64), ("filter_hits", ctypes.c_uint64),
                ("ms_stems", ctypes.c_double), ("stem_items", ctypes.c_uint64),
                ("owned_windows", ctypes.c_uint64), ("deferred_batches", ctypes.c_uint32),
                ("scan_groups", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class AtomicRates(ctypes.Structure):
    _fields_ = [("smem_or64_per_s", ctypes.c_double), ("smem_add32_per_s", ctypes.c_double),
                ("l2_or64_per_s", ctypes.c_double), ("hbm_or64_per_s", ctypes.c_double)]


class FilterSpec(ctypes.Structure):
    _fields_ = [("tumor", ctypes.c_int), ("min_tumor", ctypes.c_uint32), ("max_normal", ctypes.c_uint32),
                ("ratio", ctypes.c_uint32)]


# kc_item16: the 16-byte k-mer item of the joint table
ITEM16 = np.dtype([("key", "<u8"), ("count", "<u2", (2,)), ("pad", "<u4")])
assert ITEM16.itemsize == 16
# kc_stem_item: stem code, then 16 counts per sample (entry 4 * first base + last base)
STEM_ITEM = np.dtype([("stem", "<u8"), ("count", "<u2", (2, 16))])
assert STEM_ITEM.itemsize == 72


class TuneInput(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_int), ("packed_reads", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("n_mask", ctypes.c_void_p), ("n_reads", ctypes.c_uint64)]


class TuneTrial(ctypes.Structure):
    _fields_ = [("config", Config), ("ms", ctypes.c_double)]


class JobSpec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_samples", ctypes.c_int), ("n_hashes", ctypes.c_int),
                ("min_count", ctypes.c_uint32), ("bloom_bits", ctypes.c_uint64),
                ("packed", ctypes.c_void_p * 2), ("offsets", ctypes.c_void_p * 2), ("n_mask", ctypes.c_void_p * 2),
                ("n_reads", ctypes.c_uint64 * 2)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("jobs_per_s", ctypes.c_double),
                ("peak_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("mean_queue_ms", ctypes.c_double), ("mean_ingest_ms", ctypes.c_double),
                ("mean_batch_wait_ms", ctypes.c_double), ("mean_finalize_ms", ctypes.c_double),
                ("mean_batch_finalize_ms", ctypes.c_double), ("mean_batch_copy_ms", ctypes.c_double),
                ("mean_batch_release_ms", ctypes.c_double), ("reused_handles", ctypes.c_uint64),
                ("mean_ingest_handle_ms", ctypes.c_double), ("mean_ingest_add_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    return _build.build(force=force)


def lib():
    """Load libkc.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            p, u64, u32, i, st = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int
            L.kc_default_config.argtypes = [ctypes.POINTER(Config)]
            L.kc_default_config.restype = None
            L.kc_create.argtypes = [i, i, u64, i, u32, ctypes.POINTER(p)]
            L.kc_create.restype = st
            L.kc_create_ex.argtypes = [i, i, u64, i, u32, ctypes.POINTER(Config), p, ctypes.POINTER(p)]
            L.kc_create_ex.restype = st
            L.kc_add_reads.argtypes = [p, i, p, p, p, u64]
            L.kc_add_reads.restype = st
            L.kc_finalize.argtypes = [p]
            L.kc_finalize.restype = st
            L.kc_dump.argtypes = [p, p, p, u64, ctypes.POINTER(u64)]
            L.kc_dump.restype = st
            L.kc_export_bloom.argtypes = [p, p, u64, u64]
            L.kc_export_bloom.restype = st
            L.kc_export_bloom2.argtypes = [p, p, u64, u64]
            L.kc_export_bloom2.restype = st
            L.kc_stats_get.argtypes = [p, ctypes.POINTER(Stats)]
            L.kc_stats_get.restype = st
            L.kc_reset.argtypes = [p]
            L.kc_reset.restype = st
            L.kc_destroy.argtypes = [p]
            L.kc_destroy.restype = None
            L.kc_last_error.argtypes = []
            L.kc_last_error.restype = ctypes.c_char_p
            L.kc_status_string.argtypes = [st]
            L.kc_status_string.restype = ctypes.c_char_p
            L.kc_pack_ascii.argtypes = [p, u64, p, p]
            L.kc_pack_ascii.restype = st
            L.kc_batch_create.argtypes = [p, ctypes.POINTER(p)]
            L.kc_batch_create.restype = st
            L.kc_batch_finalize.argtypes = [p, ctypes.POINTER(p), i]
            L.kc_batch_finalize.restype = st
            L.kc_batch_ingest.argtypes = [p, ctypes.POINTER(p), i]
            L.kc_batch_ingest.restype = st
            L.kc_batch_destroy.argtypes = [p]
            L.kc_batch_destroy.restype = None
            L.kc_server_create.argtypes = [u64, i, ctypes.POINTER(p)]
            L.kc_server_create.restype = st
            L.kc_server_submit.argtypes = [p, ctypes.POINTER(JobSpec), ctypes.POINTER(u64)]
            L.kc_server_submit.restype = st
            L.kc_server_wait.argtypes = [p, u64, ctypes.c_double, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double)]
            L.kc_server_wait.restype = st
            L.kc_server_result.argtypes = [p, u64, p, p, u64, ctypes.POINTER(u64)]
            L.kc_server_result.restype = st
            L.kc_server_stats_get.argtypes = [p, ctypes.POINTER(ServerStats)]
            L.kc_server_stats_get.restype = st
            L.kc_server_destroy.argtypes = [p]
            L.kc_server_destroy.restype = None
            L.kc_server_create_ex.argtypes = [u64, i, u32, ctypes.POINTER(p)]
            L.kc_server_create_ex.restype = st
            L.kc_autotune.argtypes = [i, i, u64, i, u32, ctypes.POINTER(TuneInput), i, i, ctypes.POINTER(Config),
                                      ctypes.POINTER(TuneTrial), i, ctypes.POINTER(i)]
            L.kc_autotune.restype = st
            L.kc_tune_lookup.argtypes = [i, i, u64, i, u32, u64, ctypes.POINTER(Config), ctypes.POINTER(i)]
            L.kc_tune_lookup.restype = st
            L.kc_tune_cache_save.argtypes = [ctypes.c_char_p]
            L.kc_tune_cache_save.restype = st
            L.kc_tune_cache_load.argtypes = [ctypes.c_char_p]
            L.kc_tune_cache_load.restype = st
            L.kc_tune_cache_clear.argtypes = []
            L.kc_tune_cache_clear.restype = None
            L.kc_export_items.argtypes = [p, p, u64, ctypes.POINTER(u64)]
            L.kc_export_items.restype = st
            L.kc_export_stems.argtypes = [p, p, u64, ctypes.POINTER(u64)]
            L.kc_export_stems.restype = st
            L.kc_spectrum.argtypes = [p, u32, p]
            L.kc_spectrum.restype = st
            L.kc_filter_select.argtypes = [p, ctypes.POINTER(FilterSpec), ctypes.POINTER(u64)]
            L.kc_filter_select.restype = st
            L.kc_filter_keys.argtypes = [p, p, p, u64, ctypes.POINTER(u64)]
            L.kc_filter_keys.restype = st
            L.kc_filter_reads.argtypes = [p, p, p, p, u64, p, p, ctypes.POINTER(u64)]
            L.kc_filter_reads.restype = st
            L.kc_merge_results.argtypes = [i, ctypes.POINTER(p), ctypes.POINTER(p), ctypes.POINTER(u64), i, p, p]
            L.kc_merge_results.restype = st
            L.kc_atomic_ceilings.argtypes = [ctypes.POINTER(AtomicRates), p]
            L.kc_atomic_ceilings.restype = st
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise KcError(status, where, lib().kc_last_error().decode(errors="replace"))


def _ptr(a) -> int | None:
    """Raw pointer of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def pack_ascii(ascii: np.ndarray):
    """Pack ASCII bases into (packed words, N-mask words) on the host."""
    ascii = np.ascontiguousarray(ascii, dtype=np.uint8)
    n = ascii.size
    packed = np.zeros((n + 31) // 32, dtype=np.uint64)
    mask = np.zeros((n + 63) // 64, dtype=np.uint64)
    if n:
        _check(lib().kc_pack_ascii(ascii.ctypes.data, n, packed.ctypes.data, mask.ctypes.data), "kc_pack_ascii")
    return packed, mask


def merge_results(results, n_samples: int):
    """Merge per-owner results [(keys uint64[n], counts uint32[n, n_samples]), ...] (each ascending, keys
    disjoint across them) into one ascending result (kc_merge_results, host memory)."""
    runs = [(np.ascontiguousarray(k, dtype=np.uint64), np.ascontiguousarray(c, dtype=np.uint32)) for k, c in results]
    n_total = sum(k.size for k, _ in runs)
    keys = np.empty(n_total, dtype=np.uint64)
    counts = np.empty((n_total, n_samples), dtype=np.uint32)
    m = len(runs)
    kp = (ctypes.c_void_p * max(1, m))(*[k.ctypes.data if k.size else None for k, _ in runs])
    cp = (ctypes.c_void_p * max(1, m))(*[c.ctypes.data if c.size else None for _, c in runs])
    ns = (ctypes.c_uint64 * max(1, m))(*[k.size for k, _ in runs])
    _check(lib().kc_merge_results(m, kp, cp, ns, n_samples, keys.ctypes.data if n_total else None,
                                  counts.ctypes.data if n_total else None), "kc_merge_results")
    return keys, counts


def atomic_ceilings(stream=None) -> dict:
    """Measured random-atomic update rates (kc_atomic_ceilings), updates per second."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    r = AtomicRates()
    _check(lib().kc_atomic_ceilings(ctypes.byref(r), stream), "kc_atomic_ceilings")
    return {name: getattr(r, name) for name, _ in r._fields_}


def owned_shards(rank: int, world: int, own_bits: int):
    """[lo, hi) of the 2^own_bits hash shards that rank `rank` of `world` owns: contiguous, as even as possible."""
    n = 1 << own_bits
    if not 0 <= rank < world <= n:
        raise ValueError("need 0 <= rank < world <= 2^own_bits")
    return rank * n // world, (rank + 1) * n // world


SPLIT_NONE = 0xFFFFFFFF  # kc_config.split_max: overflowing partitions go straight to the global table
STRATEGY_NAMES = {0: "auto", 1: "direct", 2: "partitioned"}
SERVER_TUNED = 1  # kc_server_create_ex flag


class KmerCounter:
    """One counting job: add reads per sample, finalize, dump sorted counts."""

    def __init__(self, k: int, n_samples: int, bloom_bits: int, n_hashes: int = 4, min_count: int = 2,
                 table_slots: int = 0, part_bits: int = 0, spill: bool = False, ctas_per_sm: int = 0,
                 timing: bool = False, strategy: str = "auto", smem_table_log2: int = 0, scatter_mode: int = 0,
                 split_max: int = 0, tune_bases: int = 0, prune_chain: bool = False, own_bits: int = 0,
                 own_lo: int = 0, own_hi: int = 0, device_budget: int = 0, batched_ingest: bool = False,
                 stream=None):
        L = lib()
        cfg = Config()
        L.kc_default_config(ctypes.byref(cfg))
        if tune_bases:  # the tuning cache's knobs for this job class, when it has an entry
            found = ctypes.c_int()
            _check(L.kc_tune_lookup(k, n_samples, bloom_bits, n_hashes, min_count, tune_bases, ctypes.byref(cfg),
                                    ctypes.byref(found)), "kc_tune_lookup")
            if found.value:
                table_slots = table_slots or cfg.table_slots
                part_bits = part_bits or cfg.part_bits
                ctas_per_sm = ctas_per_sm or cfg.ctas_per_sm
                strategy = strategy if strategy != "auto" else STRATEGY_NAMES[cfg.strategy]
                smem_table_log2 = smem_table_log2 or cfg.smem_table_log2
                scatter_mode = scatter_mode or cfg.scatter_mode
                split_max = split_max or (-1 if cfg.split_max == SPLIT_NONE else cfg.split_max)
        cfg.table_slots = table_slots
        cfg.part_bits = part_bits
        cfg.spill = int(spill)  # 1 or True: dump re-sorts on the device when it has room; 2: merges on the host
        cfg.ctas_per_sm = ctas_per_sm
        cfg.timing = 1 if timing else 0
        cfg.strategy = {"auto": 0, "direct": 1, "partitioned": 2}[strategy]
        cfg.smem_table_log2 = smem_table_log2
        cfg.scatter_mode = scatter_mode
        cfg.split_max = SPLIT_NONE if split_max < 0 else split_max  # -1: never split an overflowing partition
        cfg.prune_chain = int(prune_chain)  # the paper's two-filter chain (direct strategy)
        cfg.own_bits, cfg.own_lo, cfg.own_hi = own_bits, own_lo, own_hi  # hash shards [own_lo, own_hi) of 2^own_bits
        cfg.device_budget = device_budget  # bytes; 0: the device's free memory
        cfg.batched_ingest = 1 if batched_ingest else 0  # extraction and grouping at finalize, batch-wide
        h = ctypes.c_void_p()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(L.kc_create_ex(k, n_samples, bloom_bits, n_hashes, min_count, ctypes.byref(cfg), stream,
                              ctypes.byref(h)), "kc_create_ex")
        self._h = h
        self._L = L
        self.k, self.n_samples, self.bloom_bits = k, n_samples, bloom_bits

    def close(self):
        if getattr(self, "_h", None):
            self._L.kc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_reads(self, sample: int, packed, offsets, n_mask):
        n_reads = (offsets.numel() if hasattr(offsets, "numel") else len(offsets)) - 1
        _check(self._L.kc_add_reads(self._h, sample, _ptr(packed), _ptr(offsets), _ptr(n_mask), max(0, n_reads)),
               "kc_add_reads")

    def add_readset(self, sample: int, readset):
        """Pack a synth.ReadSet-like object (ascii + offsets) on the host and add it."""
        packed, mask = pack_ascii(readset.ascii)
        self.add_reads(sample, packed, np.ascontiguousarray(readset.offsets, dtype=np.uint64), mask)

    def finalize(self):
        _check(self._L.kc_finalize(self._h), "kc_finalize")

    def result_size(self) -> int:
        n = ctypes.c_uint64()
        _check(self._L.kc_dump(self._h, None, None, 0, ctypes.byref(n)), "kc_dump")
        return n.value

    def dump(self, keys=None, counts=None):
        """Return (keys uint64[n], counts uint32[n, n_samples]) as numpy, or fill given buffers."""
        n = self.result_size()
        if keys is None:
            keys = np.empty(n, dtype=np.uint64)
            counts = np.empty((n, self.n_samples), dtype=np.uint32)
        got = ctypes.c_uint64()
        cap = keys.numel() if hasattr(keys, "numel") else len(keys)
        _check(self._L.kc_dump(self._h, _ptr(keys), _ptr(counts), cap, ctypes.byref(got)), "kc_dump")
        return keys[: got.value], counts[: got.value]

    def export_bloom(self, first: int = 0, n: int | None = None, out=None):
        nw = self.bloom_bits // 64
        if n is None:
            n = nw - first
        if out is None:
            out = np.empty(n, dtype=np.uint64)
        _check(self._L.kc_export_bloom(self._h, _ptr(out), first, n), "kc_export_bloom")
        return out

    def export_bloom2(self, first: int = 0, n: int | None = None, out=None):
        """Words of the Prune chain's second filter (prune_chain=True handles)."""
        nw = self.bloom_bits // 64
        if n is None:
            n = nw - first
        if out is None:
            out = np.empty(n, dtype=np.uint64)
        _check(self._L.kc_export_bloom2(self._h, _ptr(out), first, n), "kc_export_bloom2")
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(self._L.kc_stats_get(self._h, ctypes.byref(s)), "kc_stats_get")
        return s.as_dict()

    def export_items(self, out=None):
        """The result as 16-byte items (numpy ITEM16 records), or written into out
        (a device tensor of n * 16 bytes, 16-byte aligned)."""
        n = ctypes.c_uint64()
        _check(self._L.kc_export_items(self._h, None, 0, ctypes.byref(n)), "kc_export_items")
        if out is None:
            out = np.empty(n.value, dtype=ITEM16)
            cap = n.value
        else:
            cap = (out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes) // 16
        _check(self._L.kc_export_items(self._h, _ptr(out), cap, ctypes.byref(n)), "kc_export_items")
        return out

    def export_stems(self, out=None):
        """The stem-grouped table (numpy STEM_ITEM records), or written into out (72 bytes per item)."""
        n = ctypes.c_uint64()
        _check(self._L.kc_export_stems(self._h, None, 0, ctypes.byref(n)), "kc_export_stems")
        if out is None:
            out = np.empty(n.value, dtype=STEM_ITEM)
            cap = n.value
        else:
            cap = (out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes) // 72
        _check(self._L.kc_export_stems(self._h, _ptr(out), cap, ctypes.byref(n)), "kc_export_stems")
        return out

    def spectrum(self, cap: int, out=None):
        """Joint count spectrum: uint64[cap+1] (one sample) or uint64[cap+1, cap+1] (two)."""
        if out is None:
            out = np.empty((cap + 1,) * self.n_samples, dtype=np.uint64)
        _check(self._L.kc_spectrum(self._h, cap, _ptr(out)), "kc_spectrum")
        return out

    def filter_select(self, tumor: int = 1, min_tumor: int = 2, max_normal: int = 0, ratio: int = 0) -> int:
        """Filter unit: select the imbalanced result keys; returns how many."""
        spec = FilterSpec(tumor, min_tumor, max_normal, ratio)
        n = ctypes.c_uint64()
        _check(self._L.kc_filter_select(self._h, ctypes.byref(spec), ctypes.byref(n)), "kc_filter_select")
        return n.value

    def filter_keys(self):
        """(keys uint64[n], counts uint32[n, 2]) of the selection, ascending keys."""
        n = ctypes.c_uint64()
        _check(self._L.kc_filter_keys(self._h, None, None, 0, ctypes.byref(n)), "kc_filter_keys")
        keys = np.empty(n.value, dtype=np.uint64)
        counts = np.empty((n.value, 2), dtype=np.uint32)
        _check(self._L.kc_filter_keys(self._h, _ptr(keys), _ptr(counts), n.value, ctypes.byref(n)), "kc_filter_keys")
        return keys, counts

    def filter_reads(self, packed, offsets, n_mask, hits=None, candidates=None, want_candidates: bool = True):
        """Rescan reads against the selection: (hits uint32[n_reads], candidate read indices or None,
        number of candidates).  hits / candidates may be given (numpy or torch, host or device)."""
        if isinstance(offsets, np.ndarray):
            offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        n_reads = max(0, (offsets.numel() if hasattr(offsets, "numel") else len(offsets)) - 1)
        if hits is None:
            hits = np.empty(n_reads, dtype=np.uint32)
        if candidates is None and want_candidates:
            candidates = np.empty(max(1, n_reads), dtype=np.uint64)
        n = ctypes.c_uint64()
        _check(self._L.kc_filter_reads(self._h, _ptr(packed), _ptr(offsets), _ptr(n_mask), n_reads, _ptr(hits),
                                       _ptr(candidates), ctypes.byref(n)), "kc_filter_reads")
        return hits, (candidates[: n.value] if candidates is not None else None), n.value

    def filter_readset(self, readset, **kw):
        """filter_reads on a synth.ReadSet-like object (ascii + offsets), packed on the host."""
        packed, mask = pack_ascii(readset.ascii)
        return self.filter_reads(packed, np.ascontiguousarray(readset.offsets, dtype=np.uint64), mask, **kw)

    def reset(self):
        _check(self._L.kc_reset(self._h), "kc_reset")


class KcBatch:
    """Finalizes several partitioned KmerCounter jobs together (kc_batch_*)."""

    def __init__(self, stream=None):
        L = lib()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        b = ctypes.c_void_p()
        _check(L.kc_batch_create(stream, ctypes.byref(b)), "kc_batch_create")
        self._b = b
        self._L = L

    def finalize(self, counters):
        arr = (ctypes.c_void_p * len(counters))(*[c._h for c in counters])
        _check(self._L.kc_batch_finalize(self._b, arr, len(counters)), "kc_batch_finalize")

    def ingest(self, counters):
        """Extract and group the reads the counters kept (batched_ingest), all together (kc_batch_ingest)."""
        arr = (ctypes.c_void_p * len(counters))(*[c._h for c in counters])
        _check(self._L.kc_batch_ingest(self._b, arr, len(counters)), "kc_batch_ingest")

    def close(self):
        if getattr(self, "_b", None):
            self._L.kc_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        self.close()


def config_dict(cfg: Config) -> dict:
    return {"strategy": STRATEGY_NAMES[cfg.strategy], "part_bits": cfg.part_bits,
            "smem_table_log2": cfg.smem_table_log2, "ctas_per_sm": cfg.ctas_per_sm,
            "scatter_mode": cfg.scatter_mode, "split_max": cfg.split_max}


def autotune(k: int, n_samples: int, bloom_bits: int, n_hashes: int, min_count: int, inputs, reps: int = 3,
             max_trials: int = 64):
    """kc_autotune: inputs = [(sample, packed, offsets, n_mask), ...] (numpy or torch, host or device).

    Returns (best config dict, [(config dict, ms), ...] in the order tried); the best
    configuration also goes into the process-wide tuning cache."""
    L = lib()
    arr = (TuneInput * max(1, len(inputs)))()
    keep = []
    for t, (sample, packed, offsets, mask) in enumerate(inputs):
        if isinstance(offsets, np.ndarray):
            offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        keep.append(offsets)
        n = (offsets.numel() if hasattr(offsets, "numel") else len(offsets)) - 1
        arr[t] = TuneInput(sample, _ptr(packed), _ptr(offsets), _ptr(mask), max(0, n))
    best = Config()
    trials = (TuneTrial * max_trials)()
    n = ctypes.c_int()
    _check(L.kc_autotune(k, n_samples, bloom_bits, n_hashes, min_count, arr, len(inputs), reps, ctypes.byref(best),
                         trials, max_trials, ctypes.byref(n)), "kc_autotune")
    return config_dict(best), [(config_dict(trials[i].config), trials[i].ms) for i in range(n.value)]


def tune_lookup(k: int, n_samples: int, bloom_bits: int, n_hashes: int, min_count: int, n_bases: int):
    """The tuning cache's configuration for this job class (dict), or None."""
    cfg = Config()
    found = ctypes.c_int()
    _check(lib().kc_tune_lookup(k, n_samples, bloom_bits, n_hashes, min_count, n_bases, ctypes.byref(cfg),
                                ctypes.byref(found)), "kc_tune_lookup")
    return config_dict(cfg) if found.value else None


def tune_cache_save(path: str):
    _check(lib().kc_tune_cache_save(os.fsencode(path)), "kc_tune_cache_save")


def tune_cache_load(path: str):
    _check(lib().kc_tune_cache_load(os.fsencode(path)), "kc_tune_cache_load")


def tune_cache_clear():
    lib().kc_tune_cache_clear()


class KcServer:
    """Continuous-batching job server (kc_server_*); inputs are packed host arrays."""

    def __init__(self, device_budget_bytes: int, max_batch: int = 64, tuned: bool = False):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.kc_server_create_ex(device_budget_bytes, max_batch, SERVER_TUNED if tuned else 0, ctypes.byref(h)),
               "kc_server_create_ex")
        self._s = h
        self._L = L
        self._keep = {}  # job id -> host arrays that must outlive the job
        self._samples = {}

    def submit(self, k, bloom_bits, n_hashes, min_count, samples) -> int:
        """samples: list of (packed, offsets, n_mask) numpy arrays, one per sample."""
        spec = JobSpec()
        spec.k, spec.n_samples, spec.n_hashes, spec.min_count, spec.bloom_bits = (
            k, len(samples), n_hashes, min_count, bloom_bits)
        keep = []
        for i, (packed, offsets, mask) in enumerate(samples):
            offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
            keep += [packed, offsets, mask]
            spec.packed[i] = _ptr(packed)
            spec.offsets[i] = _ptr(offsets)
            spec.n_mask[i] = _ptr(mask)
            spec.n_reads[i] = len(offsets) - 1
        jid = ctypes.c_uint64()
        _check(self._L.kc_server_submit(self._s, ctypes.byref(spec), ctypes.byref(jid)), "kc_server_submit")
        self._keep[jid.value] = keep
        self._samples[jid.value] = len(samples)
        return jid.value

    def submit_workload(self, w) -> int:
        samples = []
        for rs in w.samples:
            packed, mask = pack_ascii(rs.ascii)
            samples.append((packed, rs.offsets, mask))
        return self.submit(w.k, w.bloom_bits, w.n_hashes, w.min_count, samples)

    def wait(self, job_id: int, timeout_s: float = -1.0):
        n = ctypes.c_uint64()
        lat = ctypes.c_double()
        st = self._L.kc_server_wait(self._s, job_id, timeout_s, ctypes.byref(n), ctypes.byref(lat))
        if STATUS[st] != "KC_ERR_TIMEOUT":  # the job is done: the server no longer reads its inputs
            self._keep.pop(job_id, None)
        _check(st, "kc_server_wait")
        return n.value, lat.value

    def result(self, job_id: int):
        n = ctypes.c_uint64()
        _check(self._L.kc_server_result(self._s, job_id, None, None, 0, ctypes.byref(n)), "kc_server_result")
        keys = np.empty(n.value, dtype=np.uint64)
        counts = np.empty((n.value, self._samples.get(job_id, 1)), dtype=np.uint32)
        _check(self._L.kc_server_result(self._s, job_id, keys.ctypes.data, counts.ctypes.data, n.value,
                                        ctypes.byref(n)), "kc_server_result")
        self._samples.pop(job_id, None)
        return keys, counts

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._L.kc_server_stats_get(self._s, ctypes.byref(st)), "kc_server_stats_get")
        return st.as_dict()

    def close(self):
        if getattr(self, "_s", None):
            self._L.kc_server_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()

"""CPU oracle for k-mer counting: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never does, and this
package imports nothing from it.

``kc_oracle.cpp`` is a plain single-threaded C++ statement of the counting
result (see its header for the definition and the paper passages it follows);
this module compiles it with the host compiler on first use and wraps it with
ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain -O2, no vectorisation flags, any CPU arch)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, p, i = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
        lib.orc_create.argtypes = [i, i, u64, i, u32]
        lib.orc_create.restype = p
        lib.orc_restrict.argtypes = [p, i, p]
        lib.orc_restrict.restype = i
        lib.orc_add_reads.argtypes = [p, i, p, p, u64]
        lib.orc_add_reads.restype = i
        for name in ("orc_windows", "orc_counted", "orc_distinct", "orc_result_size"):
            getattr(lib, name).argtypes = [p]
            getattr(lib, name).restype = u64
        lib.orc_result.argtypes = [p, p, p, u64]
        lib.orc_result.restype = ctypes.c_int64
        lib.orc_bloom.argtypes = [p, p, u64, u64]
        lib.orc_bloom.restype = i
        lib.orc_bloom_query.argtypes = [p, u64]
        lib.orc_bloom_query.restype = i
        lib.orc_bloom_word_index.argtypes = [p, u64]
        lib.orc_bloom_word_index.restype = u64
        lib.orc_bloom_pattern.argtypes = [p, u64]
        lib.orc_bloom_pattern.restype = u64
        lib.orc_mixer64.argtypes = [u64]
        lib.orc_mixer64.restype = u64
        lib.orc_partitions.argtypes = [p, u64, i, p]
        lib.orc_partitions.restype = i
        lib.orc_canonical.argtypes = [ctypes.c_char_p, i]
        lib.orc_canonical.restype = u64
        lib.orc_items16.argtypes = [p, p, u64]
        lib.orc_items16.restype = ctypes.c_int64
        lib.orc_spectrum.argtypes = [p, u32, p]
        lib.orc_spectrum.restype = i
        lib.orc_filter_select.argtypes = [p, i, u32, u32, u32, p, p, u64]
        lib.orc_filter_select.restype = ctypes.c_int64
        lib.orc_filter_reads.argtypes = [p, i, u32, u32, u32, p, p, u64, p]
        lib.orc_filter_reads.restype = ctypes.c_int64
        lib.orc_stems.argtypes = [p, p, u64]
        lib.orc_stems.restype = ctypes.c_int64
        lib.orc_bloom2_bounds.argtypes = [p, p, p, u64, u64]
        lib.orc_bloom2_bounds.restype = i
        lib.orc_destroy.argtypes = [p]
        lib.orc_destroy.restype = None
        _lib = lib
    return _lib


def mixer64(x: int) -> int:
    return int(_load().orc_mixer64(x))


def partitions(keys: np.ndarray, q: int) -> np.ndarray:
    """Top q bits of mixer64(key) for every key (which partition a key is in)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(keys.size, dtype=np.uint32)
    if _load().orc_partitions(keys.ctypes.data if keys.size else None, keys.size, q,
                              out.ctypes.data if keys.size else None) != 0:
        raise ValueError("oracle: partitions")
    return out


def canonical(s: str) -> int | None:
    """Canonical 2-bit key of the string s (len <= 31), None if it has a non-ACGT."""
    v = int(_load().orc_canonical(s.encode(), len(s)))
    return None if v == (1 << 64) - 1 else v


class Oracle:
    """Counts one job: create, add reads per sample, then read the result."""

    def __init__(self, k: int, n_samples: int, bloom_bits: int, n_hashes: int, min_count: int):
        self._lib = _load()
        self.k, self.n_samples = k, n_samples
        self.bloom_bits = bloom_bits
        self._h = self._lib.orc_create(k, n_samples, bloom_bits, n_hashes, min_count)
        if not self._h:
            raise ValueError("oracle: invalid parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def restrict(self, q: int, keep_parts) -> None:
        keep = np.zeros(1 << q, dtype=np.uint8)
        keep[np.asarray(list(keep_parts), dtype=np.int64)] = 1
        if self._lib.orc_restrict(self._h, q, keep.ctypes.data) != 0:
            raise ValueError("oracle: restrict failed")

    def add_reads(self, sample: int, reads) -> None:
        ascii = np.ascontiguousarray(reads.ascii, dtype=np.uint8)
        offs = np.ascontiguousarray(reads.offsets, dtype=np.uint64)
        rc = self._lib.orc_add_reads(self._h, sample, ascii.ctypes.data if ascii.size else None,
                                     offs.ctypes.data, len(offs) - 1)
        if rc != 0:
            raise ValueError(f"oracle: add_reads failed ({rc})")

    @property
    def windows(self) -> int:
        return int(self._lib.orc_windows(self._h))

    @property
    def counted(self) -> int:
        return int(self._lib.orc_counted(self._h))

    @property
    def distinct(self) -> int:
        return int(self._lib.orc_distinct(self._h))

    def result(self):
        """(keys uint64[n], counts uint32[n, n_samples]) in ascending key order."""
        n = int(self._lib.orc_result_size(self._h))
        keys = np.zeros(n, dtype=np.uint64)
        counts = np.zeros((n, self.n_samples), dtype=np.uint32)
        got = self._lib.orc_result(self._h, keys.ctypes.data, counts.ctypes.data, n)
        if got != n:
            raise RuntimeError("oracle: result size changed")
        return keys, counts

    def bloom(self, first: int = 0, n: int | None = None) -> np.ndarray:
        nw = self.bloom_bits // 64
        if n is None:
            n = nw - first
        out = np.zeros(n, dtype=np.uint64)
        if self._lib.orc_bloom(self._h, out.ctypes.data, first, n) != 0:
            raise ValueError("oracle: bloom range")
        return out

    def bloom2_bounds(self, first: int = 0, n: int | None = None):
        """(lower, upper) word arrays that bound the Prune chain's second filter for any insertion order."""
        nw = self.bloom_bits // 64
        if n is None:
            n = nw - first
        lo = np.zeros(n, dtype=np.uint64)
        hi = np.zeros(n, dtype=np.uint64)
        if self._lib.orc_bloom2_bounds(self._h, lo.ctypes.data, hi.ctypes.data, first, n) != 0:
            raise ValueError("oracle: bloom2 bounds")
        return lo, hi

    def bloom_query(self, key: int) -> bool:
        return bool(self._lib.orc_bloom_query(self._h, key))

    def bloom_word_index(self, key: int) -> int:
        return int(self._lib.orc_bloom_word_index(self._h, key))

    def bloom_pattern(self, key: int) -> int:
        return int(self._lib.orc_bloom_pattern(self._h, key))


    def items16(self) -> np.ndarray:
        """The result as 16-byte items (uint8[n, 16]): key, two clamped 16-bit counts, padding."""
        n = int(self._lib.orc_result_size(self._h))
        out = np.zeros((n, 16), dtype=np.uint8)
        if self._lib.orc_items16(self._h, out.ctypes.data, n) != n:
            raise RuntimeError("oracle: items16")
        return out

    def spectrum(self, cap: int) -> np.ndarray:
        """Joint count spectrum, uint64[(cap+1)] or uint64[cap+1, cap+1] (clamped counts)."""
        shape = (cap + 1,) if self.n_samples == 1 else (cap + 1, cap + 1)
        out = np.zeros(shape, dtype=np.uint64)
        if self._lib.orc_spectrum(self._h, cap, out.ctypes.data) != 0:
            raise ValueError("oracle: spectrum")
        return out

    def stems(self) -> np.ndarray:
        """Stem-grouped items (uint8[n, 72]): stem code, 16 counts per sample (uint16, clamped)."""
        n = self._lib.orc_stems(self._h, None, 0)
        if n < 0:
            raise ValueError("oracle: stems need k >= 3")
        out = np.zeros((n, 72), dtype=np.uint8)
        if self._lib.orc_stems(self._h, out.ctypes.data, n) != n:
            raise RuntimeError("oracle: stems")
        return out

    def filter_select(self, tumor: int = 1, min_tumor: int = 2, max_normal: int = 0, ratio: int = 0):
        """(keys uint64[n], counts uint32[n, 2]) of the selected result keys, ascending."""
        n = self._lib.orc_filter_select(self._h, tumor, min_tumor, max_normal, ratio, None, None, 0)
        if n < 0:
            raise ValueError("oracle: filter_select")
        keys = np.zeros(n, dtype=np.uint64)
        counts = np.zeros((n, 2), dtype=np.uint32)
        got = self._lib.orc_filter_select(self._h, tumor, min_tumor, max_normal, ratio, keys.ctypes.data,
                                          counts.ctypes.data, n)
        if got != n:
            raise RuntimeError("oracle: filter_select size changed")
        return keys, counts

    def filter_reads(self, reads, tumor: int = 1, min_tumor: int = 2, max_normal: int = 0, ratio: int = 0):
        """(hits uint32[n_reads], number of candidate reads) for a read set."""
        ascii = np.ascontiguousarray(reads.ascii, dtype=np.uint8)
        offs = np.ascontiguousarray(reads.offsets, dtype=np.uint64)
        n_reads = len(offs) - 1
        hits = np.zeros(max(1, n_reads), dtype=np.uint32)
        got = self._lib.orc_filter_reads(self._h, tumor, min_tumor, max_normal, ratio,
                                         ascii.ctypes.data if ascii.size else None, offs.ctypes.data, n_reads,
                                         hits.ctypes.data)
        if got < 0:
            raise ValueError("oracle: filter_reads")
        return hits[:n_reads], int(got)


def count(workload, restrict=None):
    """Run the oracle over a synth.Workload; restrict=(q, parts) limits the keys."""
    o = Oracle(workload.k, len(workload.samples), workload.bloom_bits, workload.n_hashes, workload.min_count)
    if restrict is not None:
        o.restrict(*restrict)
    for s, rs in enumerate(workload.samples):
        o.add_reads(s, rs)
    return o

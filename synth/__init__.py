"""Seeded synthetic sequencing workloads (genomes, tumour copies, reads).

The generator is shared by the CPU oracle and the GPU library's tests and
benchmarks.  It draws random inputs only and holds none of the counting
method's arithmetic.  The native part lives in ``gen.cpp`` and is compiled on
first use with the host C++ compiler.

The five workload shapes stand in for the paper's evaluation data (an
Hg19-based personalised genome sequenced in silico with ART Illumina, 312 GB
of gzip FASTQ; Section IV-A), which is not available here:

* ``tiny``   100 kbp genome, 20,000 x 100 bp reads, 1 % substitutions, 0.1 % N
* ``mid``    5 Mbp genome, 1,000,000 x 150 bp reads (30x), 0.5 % / 0.05 %
* ``paired`` 50 Mbp genome; tumour copy with 0.1 % SNVs and 1-10 bp indels at
             1e-5 per base; 10,000,000 x 150 bp reads per sample
* ``ooc``    500 Mbp genome, 100,000,000 x 150 bp reads
* ``served`` 256 jobs: genome U{1..20} Mbp, reads log-uniform in [1e4, 2e6],
             read length U[100, 250], k in {25, 31}, Poisson arrivals
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_LIB = os.path.join(_HERE, "libkcsynth.so")
_lock = threading.Lock()
_lib = None

_THREADS = max(1, min(32, os.cpu_count() or 1))


def build(force: bool = False) -> str:
    """Compile ``gen.cpp`` into ``libkcsynth.so`` (host code, any CPU arch)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.synth_genome.argtypes = [u64, u64, p, ctypes.c_int]
        lib.synth_genome.restype = ctypes.c_int
        lib.synth_mutate.argtypes = [u64, p, u64, ctypes.c_double, ctypes.c_double, ctypes.c_int, p, u64]
        lib.synth_mutate.restype = ctypes.c_int64
        lib.synth_read_offsets.argtypes = [u64, u64, u32, u32, p, ctypes.c_int]
        lib.synth_read_offsets.restype = ctypes.c_int
        lib.synth_reads.argtypes = [u64, p, u64, u64, ctypes.c_double, ctypes.c_double, p, p, ctypes.c_int]
        lib.synth_reads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class ReadSet:
    """Concatenated ASCII reads; read r is ascii[offsets[r]:offsets[r+1]]."""

    ascii: np.ndarray  # uint8
    offsets: np.ndarray  # uint64, n_reads + 1

    @property
    def n_reads(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1] - self.offsets[0])

    def read(self, r: int) -> str:
        return self.ascii[self.offsets[r] : self.offsets[r + 1]].tobytes().decode()

    def slice(self, r0: int, r1: int) -> "ReadSet":
        """Reads r0..r1-1 as a new set with offsets starting at 0."""
        lo, hi = int(self.offsets[r0]), int(self.offsets[r1])
        return ReadSet(self.ascii[lo:hi].copy(), (self.offsets[r0 : r1 + 1] - np.uint64(lo)).astype(np.uint64))

    @staticmethod
    def from_strings(reads) -> "ReadSet":
        data = "".join(reads).encode()
        offs = np.zeros(len(reads) + 1, dtype=np.uint64)
        offs[1:] = np.cumsum([len(r) for r in reads], dtype=np.uint64)
        return ReadSet(np.frombuffer(data, dtype=np.uint8).copy(), offs)


def genome(seed: int, G: int) -> np.ndarray:
    out = np.empty(G, dtype=np.uint8)
    if _load().synth_genome(seed, G, _ptr(out), _THREADS) != 0:
        raise RuntimeError("synth_genome failed")
    return out


def mutate(seed: int, g: np.ndarray, snv_rate: float, indel_rate: float, indel_max: int = 10) -> np.ndarray:
    cap = len(g) + len(g) // 50 + 1024
    out = np.empty(cap, dtype=np.uint8)
    n = _load().synth_mutate(seed, _ptr(g), len(g), snv_rate, indel_rate, indel_max, _ptr(out), cap)
    if n < 0:
        raise RuntimeError("synth_mutate: output capacity exceeded")
    return out[:n].copy()


def reads(seed: int, g: np.ndarray, n_reads: int, len_min: int, len_max: int, sub_rate: float,
          n_rate: float) -> ReadSet:
    lib = _load()
    offs = np.empty(n_reads + 1, dtype=np.uint64)
    if lib.synth_read_offsets(seed, n_reads, len_min, len_max, _ptr(offs), _THREADS) != 0:
        raise RuntimeError("synth_read_offsets failed")
    out = np.empty(int(offs[-1]), dtype=np.uint8)
    rc = lib.synth_reads(seed, _ptr(g), len(g), n_reads, sub_rate, n_rate, _ptr(offs), _ptr(out), _THREADS)
    if rc != 0:
        raise RuntimeError(f"synth_reads failed ({rc})")
    return ReadSet(out, offs)


@dataclass
class Workload:
    """One counting job: read sets per sample plus the counting parameters."""

    name: str
    samples: list  # list[ReadSet]
    k: int
    bloom_bits: int
    n_hashes: int
    min_count: int
    table_slots: int = 0  # 0 = library default
    extra: dict = field(default_factory=dict)

    @property
    def n_bases(self) -> int:
        return sum(s.n_bases for s in self.samples)


def _scaled(n: int, scale: float) -> int:
    return max(1, int(round(n * scale)))


def tiny(scale: float = 1.0) -> Workload:
    g = genome(1, 100_000)
    rs = reads(1, g, _scaled(20_000, scale), 100, 100, 0.01, 0.001)
    return Workload("tiny", [rs], k=31, bloom_bits=1 << 24, n_hashes=4, min_count=2)


def mid(scale: float = 1.0, seed: int = 2) -> Workload:
    g = genome(seed, 5_000_000)
    rs = reads(seed, g, _scaled(1_000_000, scale), 150, 150, 0.005, 0.0005)
    return Workload("mid", [rs], k=31, bloom_bits=1 << 30, n_hashes=4, min_count=2, table_slots=1 << 24)


def paired(scale: float = 1.0) -> Workload:
    G = _scaled(50_000_000, scale)
    normal_g = genome(3, G)
    tumour_g = mutate(6, normal_g, 0.001, 1e-5, 10)
    n = _scaled(10_000_000, scale)
    normal = reads(4, normal_g, n, 150, 150, 0.005, 0.0005)
    tumour = reads(5, tumour_g, n, 150, 150, 0.005, 0.0005)
    return Workload("paired", [normal, tumour], k=31, bloom_bits=1 << 32, n_hashes=4, min_count=2)


def ooc(scale: float = 1.0) -> Workload:
    G = _scaled(500_000_000, scale)
    g = genome(7, G)
    rs = reads(7, g, _scaled(100_000_000, scale), 150, 150, 0.005, 0.0005)
    return Workload("ooc", [rs], k=31, bloom_bits=1 << 34, n_hashes=4, min_count=2, extra={"spill_parts": 64})


def served_bloom_bits(G: int, n_windows: int, k: int, sub_rate: float) -> int:
    """8 bits per expected distinct k-mer: genome k-mers plus erroneous windows."""
    expected = G + n_windows * (1.0 - (1.0 - sub_rate) ** k)
    bits = 1 << max(12, math.ceil(math.log2(max(1.0, 8.0 * expected))))
    return bits


@dataclass
class JobSpec:
    job_id: int
    seed: int
    G: int
    n_reads: int
    k: int
    arrival_s: float = 0.0


def served_specs(n_jobs: int = 256, rate_per_s: float = 1.0, max_reads: int = 2_000_000) -> list:
    """Job shapes of the served stream (seed 1000+i per job, arrivals seed 99)."""
    specs = []
    arr = np.random.default_rng(99).exponential(1.0 / rate_per_s, size=n_jobs).cumsum()
    for i in range(n_jobs):
        rng = np.random.default_rng(1000 + i)
        G = int(rng.integers(1, 21)) * 1_000_000
        R = int(round(math.exp(rng.uniform(math.log(1e4), math.log(max_reads)))))
        k = int(rng.choice([25, 31]))
        specs.append(JobSpec(i, 1000 + i, G, R, k, float(arr[i] - arr[0])))
    return specs


def served_job(spec: JobSpec) -> Workload:
    g = genome(spec.seed, spec.G)
    rs = reads(spec.seed, g, spec.n_reads, 100, 250, 0.005, 0.0005)
    approx_windows = rs.n_bases - spec.n_reads * (spec.k - 1)
    bb = served_bloom_bits(spec.G, approx_windows, spec.k, 0.005)
    return Workload(f"served{spec.job_id}", [rs], k=spec.k, bloom_bits=bb, n_hashes=4, min_count=2)


WORKLOADS = {"tiny": tiny, "mid": mid, "paired": paired, "ooc": ooc}

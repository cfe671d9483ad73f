"""The oracle over a large read set, restricted to a few hash partitions, on
several host processes.

Counts are sums over windows and the filter is an OR over windows, so the
oracle can count disjoint pieces of the reads on its own and the pieces be
combined afterwards: each piece is counted with min_count 1 (every key it
sees), the per-key counts of all pieces are added, and min_count is applied
to the sums; the filter words are OR-ed.  The workers are started with
"spawn" (the parent may already hold a CUDA context) and read the ASCII reads
from .npy files mapped into memory.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np


def _piece(args):
    path, sample, r0, r1, k, n_samples, bloom_bits, n_hashes, q, parts = args
    import oracle
    import synth

    ascii = np.load(os.path.join(path, f"ascii{sample}.npy"), mmap_mode="r")
    offs = np.load(os.path.join(path, f"offs{sample}.npy"), mmap_mode="r")
    lo, hi = int(offs[r0]), int(offs[r1])
    rs = synth.ReadSet(np.ascontiguousarray(ascii[lo:hi]), (np.asarray(offs[r0:r1 + 1]) - np.uint64(lo)).astype(np.uint64))
    o = oracle.Oracle(k, n_samples, bloom_bits, n_hashes, 1)
    o.restrict(q, parts)
    o.add_reads(sample, rs)
    keys, counts = o.result()
    per = (bloom_bits // 64) >> q
    words = {p: o.bloom(p * per, per) for p in parts}
    return keys, counts, words, o.windows


class Restricted:
    """Result of the restricted oracle over a workload: keys, counts (sum >= min_count), filter slices, windows."""

    def __init__(self, keys, counts, words, windows):
        self.keys, self.counts, self.words, self.windows = keys, counts, words, windows


def count_restricted(w, q: int, parts, n_proc: int | None = None, piece_reads: int = 500_000) -> Restricted:
    parts = list(parts)
    n_proc = n_proc or max(1, min(16, os.cpu_count() or 1))
    n_samples = len(w.samples)
    with tempfile.TemporaryDirectory() as path:
        jobs = []
        for s, rs in enumerate(w.samples):
            np.save(os.path.join(path, f"ascii{s}.npy"), rs.ascii)
            np.save(os.path.join(path, f"offs{s}.npy"), np.ascontiguousarray(rs.offsets, dtype=np.uint64))
            for r0 in range(0, rs.n_reads, piece_reads):
                jobs.append((path, s, r0, min(rs.n_reads, r0 + piece_reads), w.k, n_samples, w.bloom_bits,
                             w.n_hashes, q, parts))
        with mp.get_context("spawn").Pool(n_proc) as pool:
            pieces = pool.map(_piece, jobs, chunksize=1)
    keys = np.concatenate([p[0] for p in pieces]) if pieces else np.zeros(0, np.uint64)
    counts = np.concatenate([p[1] for p in pieces]).astype(np.uint64) if pieces else np.zeros((0, n_samples), np.uint64)
    uk, inv = np.unique(keys, return_inverse=True)
    sums = np.zeros((uk.size, n_samples), dtype=np.uint64)
    np.add.at(sums, inv, counts)
    keep = sums.sum(axis=1) >= w.min_count
    words = {}
    for p in parts:
        acc = None
        for piece in pieces:
            acc = piece[2][p].copy() if acc is None else acc | piece[2][p]
        words[p] = acc
    return Restricted(uk[keep], sums[keep].astype(np.uint32), words, sum(p[3] for p in pieces))

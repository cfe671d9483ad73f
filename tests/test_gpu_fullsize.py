"""Parity at the real shapes of the two-sample and out-of-core configurations.

* paired: 2 x 10,000,000 x 150 bp reads (a 50 Mbp genome and its tumour copy),
  a 2^32-bit filter, the joint table of two samples, 17 partition bits (two
  grouping levels), the launch configuration the benchmark tunes to;
* out-of-core shaped: a 500 Mbp genome, a 2^34-bit filter, 18 partition bits,
  the 64 partition groups spilled to pinned host memory and brought back by
  kc_dump on the device (spill 1) or merged on the host (spill 2), with
  20,000,000 of the configuration's 100,000,000 reads (as many as the oracle
  counts here in about a minute).

The oracle counts two of 64 hash partitions in full (tests/_oracle_par.py, on
host processes); the GPU result restricted to them, their filter words and
the number of windows must match bit for bit, and the whole dump must be
strictly ascending.
"""
import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc
from tests import _oracle_par

pytestmark = pytest.mark.gpu

Q, PARTS = 6, [5, 50]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    kc.lib()


def _check(c, w, ref, oracle_mod):
    gk, gc = c.dump()
    assert np.all(np.diff(gk) > 0)
    sel = np.isin(oracle_mod.partitions(gk, Q), PARTS)
    assert np.array_equal(gk[sel], ref.keys)
    assert np.array_equal(gc[sel], ref.counts)
    per = (w.bloom_bits // 64) >> Q
    for p in PARTS:
        assert np.array_equal(c.export_bloom(p * per, per), ref.words[p])
    assert c.stats()["windows"] == ref.windows
    return gk.size


def test_paired_full_size(oracle_mod):
    w = synth.paired()
    assert sum(rs.n_reads for rs in w.samples) == 20_000_000
    ref = _oracle_par.count_restricted(w, Q, PARTS)
    c = kc.KmerCounter(w.k, 2, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", part_bits=17)
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    c.finalize()
    n = _check(c, w, ref, oracle_mod)
    assert c.stats()["partitions"] == 1 << 17
    assert 30 * ref.keys.size < n < 34 * ref.keys.size  # two partitions of 64 hold about 1/32 of the keys
    c.close()


@pytest.fixture(scope="module")
def ooc_shaped():
    g = synth.genome(7, 500_000_000)
    rs = synth.reads(7, g, 20_000_000, 150, 150, 0.005, 0.0005)
    del g
    w = synth.Workload("ooc-shaped", [rs], k=31, bloom_bits=1 << 34, n_hashes=4, min_count=2)
    return w, _oracle_par.count_restricted(w, Q, PARTS)


@pytest.mark.parametrize("spill", [1, 2])
def test_ooc_shaped_spilled(oracle_mod, ooc_shaped, spill):
    w, ref = ooc_shaped
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned", part_bits=18,
                       spill=spill)
    cuts = np.linspace(0, w.samples[0].n_reads, 3).astype(int)  # two kc_add_reads calls
    for a, b in zip(cuts[:-1], cuts[1:]):
        c.add_readset(0, w.samples[0].slice(a, b))
    c.finalize()
    st = c.stats()
    assert st["spilled_bytes"] == 16 * st["result_keys"] > 0
    _check(c, w, ref, oracle_mod)
    c.close()

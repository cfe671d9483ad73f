"""Autotuner: it times candidate configurations of the caller's job, every
candidate it reports as working gives the oracle's result, and the cached
best configuration is what kc_tune_lookup, KmerCounter(tune_bases=...) and the
tuned server then use."""
import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kc.lib()
    return torch


def _device_inputs(torch, w):
    out = []
    for s, rs in enumerate(w.samples):
        packed, mask = kc.pack_ascii(rs.ascii)
        out.append((s, torch.from_numpy(packed.view(np.int64)).cuda(), torch.from_numpy(
            np.ascontiguousarray(rs.offsets, dtype=np.uint64).view(np.int64)).cuda(),
                    torch.from_numpy(mask.view(np.int64)).cuda()))
    return out


def _count(w, **kw):
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, **kw)
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    c.finalize()
    return c


def test_autotune_reports_trials_and_caches_best(torch_cuda, oracle_mod):
    kc.tune_cache_clear()
    w = synth.tiny(scale=0.5)
    best, trials = kc.autotune(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, _device_inputs(torch_cuda, w), reps=2)
    ok = [(c, ms) for c, ms in trials if ms >= 0]
    assert len(trials) >= 8 and len(ok) >= 6
    assert {c["strategy"] for c, _ in ok} == {"partitioned", "direct"}
    assert best in [c for c, _ in ok]
    assert min(ms for _, ms in ok) == [ms for c, ms in ok if c == best][0]
    # the cache holds it for this job class, not for another size class
    assert kc.tune_lookup(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, w.n_bases) == best
    assert kc.tune_lookup(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, w.n_bases * 4) is None
    o = oracle_mod.count(w)
    ok_k, ok_c = o.result()
    c = _count(w, tune_bases=w.n_bases)
    assert c.stats()["strategy"] == {"direct": 1, "partitioned": 2}[best["strategy"]]
    gk, gc = c.dump()
    assert np.array_equal(gk, ok_k) and np.array_equal(gc, ok_c)
    # every tried partitioned configuration is exact too
    for cfg, ms in ok[:4]:
        c = _count(w, strategy=cfg["strategy"], part_bits=cfg["part_bits"], smem_table_log2=cfg["smem_table_log2"],
                   ctas_per_sm=cfg["ctas_per_sm"])
        gk, gc = c.dump()
        assert np.array_equal(gk, ok_k) and np.array_equal(gc, ok_c)


def test_tuned_server_uses_cache(torch_cuda, oracle_mod, tmp_path):
    kc.tune_cache_clear()
    w = synth.tiny(scale=0.3)
    kc.autotune(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, _device_inputs(torch_cuda, w), reps=1)
    path = str(tmp_path / "tune.txt")
    kc.tune_cache_save(path)
    kc.tune_cache_clear()
    kc.tune_cache_load(path)
    assert kc.tune_lookup(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count, w.n_bases) is not None
    srv = kc.KcServer(4 << 30, max_batch=4, tuned=True)
    ids = [srv.submit_workload(w) for _ in range(3)]
    ok, oc = oracle_mod.count(w).result()
    for i in ids:
        srv.wait(i, timeout_s=120)
        keys, counts = srv.result(i)
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    srv.close()
    kc.tune_cache_clear()

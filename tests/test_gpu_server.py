"""The continuous-batching server: every job's result is the same in the mix
as alone (tolerance 0: the same keys, counts and filter-derived results), for
jobs that arrive while others run and under a memory budget that forces
admission to wait."""
import random
import threading
import time

import numpy as np
import pytest

import synth
import paper_1712_03254_gb300 as kc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kc.lib()


def _jobs(seed, n):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        G = rng.choice([30_000, 100_000, 300_000])
        g = synth.genome(seed * 1000 + i, G)
        n_reads = int(round(np.exp(rng.uniform(np.log(300), np.log(30_000)))))
        rs = synth.reads(seed * 1000 + i, g, n_reads, 100, 250, 0.005, 0.0005)
        k = rng.choice([25, 31])
        samples = [rs] if rng.random() < 0.7 else [rs.slice(0, n_reads // 2), rs.slice(n_reads // 2, n_reads)]
        bb = synth.served_bloom_bits(G, max(1, rs.n_bases - n_reads * (k - 1)), k, 0.005)
        out.append(synth.Workload(f"s{i}", samples, k, bb, 4, 2))
    return out


def _alone(w):
    c = kc.KmerCounter(w.k, len(w.samples), w.bloom_bits, w.n_hashes, w.min_count, strategy="partitioned")
    for s, rs in enumerate(w.samples):
        c.add_readset(s, rs)
    c.finalize()
    return c.dump()


def test_mix_equals_alone_with_staggered_arrivals(oracle_mod):
    jobs = _jobs(3, 14)
    srv = kc.KcServer(device_budget_bytes=8 << 30, max_batch=8)
    ids = [None] * len(jobs)

    def feeder():
        rng = random.Random(5)
        for i, w in enumerate(jobs):
            ids[i] = srv.submit_workload(w)
            time.sleep(rng.uniform(0.0, 0.01))

    t = threading.Thread(target=feeder)
    t.start()
    t.join()
    for i, w in enumerate(jobs):
        n, lat = srv.wait(ids[i], timeout_s=120)
        assert lat > 0
        keys, counts = srv.result(ids[i])
        assert len(keys) == n
        ak, ac = _alone(w)
        assert np.array_equal(keys, ak) and np.array_equal(counts, ac)
        ok, oc = oracle_mod.count(w).result()
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["batches"] >= 1
    srv.close()


def test_budget_admission_still_exact(oracle_mod):
    jobs = _jobs(4, 8)
    # a budget of about two average jobs: admission has to wait for memory
    # the server's footprint bound: filter + 50 B per base + 8 B per read + 8 MiB
    est = [w.bloom_bits // 8 + 50 * w.n_bases + 8 * sum(rs.n_reads for rs in w.samples) + (8 << 20) for w in jobs]
    budget = int(2 * np.mean(est))
    srv = kc.KcServer(device_budget_bytes=budget, max_batch=4)
    ids = [srv.submit_workload(w) for w in jobs]
    for i, w in enumerate(jobs):
        srv.wait(ids[i], timeout_s=120)
        keys, counts = srv.result(ids[i])
        ok, oc = oracle_mod.count(w).result()
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    st = srv.stats()
    assert st["completed"] == len(jobs)
    assert st["peak_bytes"] <= max(budget, max(est))
    srv.close()


def test_wait_timeout_and_unknown_job():
    srv = kc.KcServer(device_budget_bytes=1 << 30, max_batch=2)
    with pytest.raises(kc.KcError) as e:
        srv.wait(12345, timeout_s=0.01)
    assert e.value.name == "KC_ERR_ARG"
    srv.close()


def test_failed_job_reports_its_error_and_others_complete(oracle_mod):
    """A job the library rejects (k = 40) fails with its own status and
    message; the jobs around it complete with their exact results."""
    good = _jobs(9, 2)
    srv = kc.KcServer(device_budget_bytes=4 << 30, max_batch=4)
    packed, mask = kc.pack_ascii(good[0].samples[0].ascii)
    bad_id = srv.submit(40, good[0].bloom_bits, 4, 2, [(packed, good[0].samples[0].offsets, mask)])
    ids = [srv.submit_workload(w) for w in good]
    with pytest.raises(kc.KcError) as e:
        srv.wait(bad_id, timeout_s=120)
    assert e.value.name == "KC_ERR_ARG" and "k must be" in str(e.value)
    for i, w in zip(ids, good):
        srv.wait(i, timeout_s=120)
        keys, counts = srv.result(i)
        ok, oc = oracle_mod.count(w).result()
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == len(good)
    srv.close()


def test_reused_handles_give_exact_results(oracle_mod):
    """Jobs with the same parameters one after another run on the finished
    jobs' handles (reset and kept by the server); every result still equals
    the oracle's, whatever the previous job on the handle counted."""
    base = _jobs(11, 1)[0]
    jobs = []
    for i in range(6):  # same k, filter size, hashes and min_count; different reads
        g = synth.genome(500 + i, 50_000)
        rs = synth.reads(500 + i, g, 2_000 + 700 * i, 100, 250, 0.005, 0.0005)
        jobs.append(synth.Workload(f"r{i}", [rs], base.k, 1 << 20, 4, 2))
    srv = kc.KcServer(device_budget_bytes=8 << 30, max_batch=4)
    for w in jobs:  # one at a time: each job finds the previous job's handle idle
        time.sleep(0.05)  # the reaper thread parks the previous job's handle meanwhile
        jid = srv.submit_workload(w)
        srv.wait(jid, timeout_s=120)
        keys, counts = srv.result(jid)
        o = oracle_mod.count(w)
        ok, oc = o.result()
        assert np.array_equal(keys, ok) and np.array_equal(counts, oc)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs)
    assert st["reused_handles"] >= 1

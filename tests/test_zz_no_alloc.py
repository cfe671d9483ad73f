"""kc_bloom_build_noalloc against the regular counting path and the oracle.

The no-allocation entry point serves callers that cannot allocate device
memory when they need a read set's filter (their allocator owns the device,
or their loop must not wait on cudaMalloc).  It must give the same filter
words as counting the reads with kc_create / kc_add_reads / kc_finalize and
reading kc_export_bloom, and as the oracle's filter, on calls in a row
through the same fixed scratch array -- including a read range that starts
inside a 64-base unit of the caller's arrays.  This file is collected last
on purpose.
"""
import ctypes

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
    return torch


def _noalloc_fn():
    L = kc.lib()
    f = L.kc_bloom_build_noalloc
    u64, p, i = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
    f.argtypes = [i, u64, i, p, p, p, u64, p, p]
    f.restype = ctypes.c_int
    return f


def _device_inputs(torch, rs):
    packed, mask = kc.pack_ascii(rs.ascii)
    dp = torch.from_numpy(packed.view(np.int64)).cuda()
    dm = torch.from_numpy(mask.view(np.int64)).cuda()
    do = torch.from_numpy(np.ascontiguousarray(rs.offsets, dtype=np.uint64).view(np.int64)).cuda()
    return dp, dm, do


def _regular_filter(w, rs):
    c = kc.KmerCounter(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count)
    c.add_readset(0, rs)
    c.finalize()
    out = c.export_bloom()
    c.close()
    return out


def _oracle_filter(oracle_mod, w, rs):
    o = oracle_mod.Oracle(w.k, 1, w.bloom_bits, w.n_hashes, w.min_count)
    o.add_reads(0, rs)
    return o.bloom()


def test_noalloc_filter_equals_counting_path_two_calls(torch_cuda, oracle_mod):
    torch = torch_cuda
    f = _noalloc_fn()
    w = synth.tiny(scale=0.5)
    rs_all = w.samples[0]
    sets = [rs_all.slice(0, 6000), rs_all.slice(4000, rs_all.n_reads)]  # two different read sets
    bloom = torch.full((w.bloom_bits // 64,), -1, dtype=torch.int64, device="cuda")  # garbage in the output
    for rs in sets:
        expect = _regular_filter(w, rs)
        dp, dm, do = _device_inputs(torch, rs)
        torch.cuda.synchronize()
        st = f(w.k, w.bloom_bits, w.n_hashes, dp.data_ptr(), do.data_ptr(), dm.data_ptr(), rs.n_reads,
               bloom.data_ptr(), None)
        assert st == 0, kc.lib().kc_last_error()
        got = bloom.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, expect)  # bit for bit, the tolerance of every parity test here
        assert np.array_equal(got, _oracle_filter(oracle_mod, w, rs))


def test_noalloc_unaligned_range_of_full_arrays(torch_cuda, oracle_mod):
    """Reads r0..r1 of the whole packed arrays: offsets[r0] is not a multiple of 64."""
    torch = torch_cuda
    f = _noalloc_fn()
    w = synth.tiny(scale=0.5)
    rs_all = w.samples[0]
    r0 = next(r for r in range(1, rs_all.n_reads) if int(rs_all.offsets[r]) % 64 not in (0, 32))
    r1 = rs_all.n_reads - 3
    assert int(rs_all.offsets[r0]) % 64 != 0
    dp, dm, do_all = _device_inputs(torch, rs_all)
    do = do_all[r0 : r1 + 1].contiguous()
    bloom = torch.full((w.bloom_bits // 64,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        st = f(w.k, w.bloom_bits, w.n_hashes, dp.data_ptr(), do.data_ptr(), dm.data_ptr(), r1 - r0,
               bloom.data_ptr(), None)
        assert st == 0, kc.lib().kc_last_error()
        got = bloom.cpu().numpy().view(np.uint64)
        sub = rs_all.slice(r0, r1)
        assert np.array_equal(got, _oracle_filter(oracle_mod, w, sub))
        assert np.array_equal(got, _regular_filter(w, sub))


def test_noalloc_rejects_oversized_and_host_inputs(torch_cuda):
    torch = torch_cuda
    f = _noalloc_fn()
    n = (1 << 23) + 64
    packed = torch.zeros((n + 31) // 32, dtype=torch.int64, device="cuda")
    mask = torch.zeros((n + 63) // 64, dtype=torch.int64, device="cuda")
    offs = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    bloom = torch.zeros(1 << 10, dtype=torch.int64, device="cuda")
    st = f(31, 1 << 16, 4, packed.data_ptr(), offs.data_ptr(), mask.data_ptr(), 1, bloom.data_ptr(), None)
    assert kc.STATUS[st] == "KC_ERR_CAPACITY"
    host_offs = np.array([0, 100], dtype=np.uint64)
    st = f(31, 1 << 16, 4, packed.data_ptr(), host_offs.ctypes.data, mask.data_ptr(), 1, bloom.data_ptr(), None)
    assert kc.STATUS[st] == "KC_ERR_ARG"
    # pinned host memory is reachable by the GPU but is not device memory: refused too
    pinned = torch.zeros(1 << 10, dtype=torch.int64).pin_memory()
    st = f(31, 1 << 16, 4, packed.data_ptr(), offs.data_ptr(), mask.data_ptr(), 1, pinned.data_ptr(), None)
    assert kc.STATUS[st] == "KC_ERR_ARG"

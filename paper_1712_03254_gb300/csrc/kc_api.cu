// C ABI of libkc: handle lifecycle, ingest, finalize, dump (see include/kc.h).
//
// Device memory of one job:
//   filter       bloom_bits / 8 bytes, 64-bit words
//   table        table_slots x 16-byte items (key + 1, two uint32 counts), the
//                Count unit's k-mer layout of Section III-D without its padding
//   read store   per kc_add_reads call: 2-bit packed words (padded to whole
//                64-base units) and one valid-window-start bit per base, kept
//                for the exact recount of kc_finalize
//   result       sorted keys and per-sample counts after kc_finalize
// Transient buffers (N mask, read starts, offsets, sort buckets) come from the
// stream-ordered pool (cudaMallocAsync) and are released on the same stream.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <memory>
#include <thread>
#include <cstring>
#include <string>
#include <vector>

#include "kc_ctx.h"

namespace kcapi {

thread_local std::string g_last_error;

kc_status fail(kc_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

kc_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KC_ERR_OOM_DEVICE : KC_ERR_CUDA;
}


int log2_exact(uint64_t x) {
    int r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Pinned host memory the device can write (its device-side address in *dev):
// a kernel writes such memory directly, over the host link.
bool host_mapped(const void* p, void** dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

// Memory the handle's kernels may read in place: device memory of its own
// device, or managed memory (another GPU's memory is copied instead).
bool is_local_device_ptr(const void* p, int device) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}



}  // namespace kcapi

namespace kc {
void set_last_error(const std::string& msg) { kcapi::g_last_error = msg; }

std::mutex& sync_api_mutex() {
    static std::mutex m;
    return m;
}
}  // namespace kc


namespace kcapi {

cudaEvent_t phase_begin(kc_handle h, cudaStream_t st) {
    if (!h->cfg.timing) return nullptr;
    cudaEvent_t e = nullptr;
    if (!h->ev_pool.empty()) {
        e = h->ev_pool.back();
        h->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaEventRecord(e, st ? st : h->stream);
    return e;
}

void phase_end(kc_handle h, int phase, cudaEvent_t a, cudaStream_t st) {
    if (!a) return;
    cudaEvent_t b = phase_begin(h, st);
    if (!b) {
        h->ev_pool.push_back(a);
        return;
    }
    h->marks.push_back({phase, a, b});
}

// Call after the stream has been synchronised.
void phase_collect(kc_handle h) {
    for (const auto& m : h->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) h->ms[m.phase] += t;
        else cudaGetLastError();
        h->ev_pool.push_back(m.a);
        h->ev_pool.push_back(m.b);
    }
    h->marks.clear();
}

kc_status check_open(kc_handle h) {
    if (!h) return fail(KC_ERR_ARG, "null handle");
    if (h->state == State::Poisoned) return fail(KC_ERR_STATE, "handle poisoned by an earlier error; call kc_reset");
    return KC_OK;
}

void free_batches(kc_handle h) {
    for (auto& b : h->batches) {
        if (b.pw) cudaFreeAsync(b.pw, h->stream);
        if (b.vw) cudaFreeAsync(b.vw, h->stream);
        if (b.hdata) cudaFreeAsync(b.hdata, h->stream);
        if (b.hstarts) cudaFreeAsync(b.hstarts, h->stream);
    }
    h->batches.clear();
}

// Forget the spilled runs; their pinned chunks stay for the next job.
void release_spill(kc_handle h) {
    for (auto& c : h->spill_chunks) c.used = 0;
    h->spill_dir.clear();
    h->spilled = false;
    h->spilled_bytes = 0;
}

void free_spill_chunks(kc_handle h) {
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    for (auto& c : h->spill_chunks) cudaFreeHost(c.p);
    h->spill_chunks.clear();
}

// Room for `words` 64-bit words in the pinned chunks: the first chunk with
// space left, else a new chunk of at least 256 MiB.
uint64_t* spill_alloc(kc_handle h, uint64_t words) {
    for (auto& c : h->spill_chunks)
        if (c.words - c.used >= words) {
            uint64_t* p = c.p + c.used;
            c.used += words;
            return p;
        }
    PinnedChunk c;
    c.words = std::max<uint64_t>(words, 32ull << 20);
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    if (cudaMallocHost(&c.p, c.words * 8) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c.used = words;
    h->spill_chunks.push_back(c);
    return c.p;
}

// Merge the spilled sorted runs into keys[] and counts[] (host; counts may be
// null), in key ranges split among threads: each range is cut out of every run
// by binary search and merged with a small heap.
void merge_runs(const std::vector<SpillRun>& runs, uint64_t* keys, uint32_t* counts, int n_samples) {
    std::vector<uint64_t> sample;
    for (const auto& r : runs)
        for (uint64_t i = 0; i < r.n_items; i += std::max<uint64_t>(1, r.n_items / 256)) sample.push_back(r.host[i]);
    std::sort(sample.begin(), sample.end());
    unsigned T = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<uint64_t> split;  // T-1 splitters
    for (unsigned t = 1; t < T && !sample.empty(); ++t) split.push_back(sample[sample.size() * t / T]);
    T = (unsigned)split.size() + 1;
    // per thread and run: [lo, hi) of the run inside the thread's key range
    std::vector<std::vector<std::pair<uint64_t, uint64_t>>> cut(T, std::vector<std::pair<uint64_t, uint64_t>>(runs.size()));
    std::vector<uint64_t> out_off(T + 1, 0);
    for (size_t r = 0; r < runs.size(); ++r) {
        const uint64_t* k = runs[r].host;
        uint64_t prev = 0;
        for (unsigned t = 0; t < T; ++t) {
            uint64_t hi = t + 1 < T ? (uint64_t)(std::lower_bound(k, k + runs[r].n_items, split[t]) - k) : runs[r].n_items;
            hi = std::max(hi, prev);
            cut[t][r] = {prev, hi};
            out_off[t + 1] += hi - prev;
            prev = hi;
        }
    }
    for (unsigned t = 0; t < T; ++t) out_off[t + 1] += out_off[t];
    auto work = [&](unsigned t) {
        using Item = std::pair<uint64_t, size_t>;  // key, run
        std::vector<Item> heap;
        std::vector<uint64_t> pos(runs.size());
        for (size_t r = 0; r < runs.size(); ++r) {
            pos[r] = cut[t][r].first;
            if (pos[r] < cut[t][r].second) heap.push_back({runs[r].host[pos[r]], r});
        }
        auto greater = [](const Item& a, const Item& b) { return a.first > b.first; };
        std::make_heap(heap.begin(), heap.end(), greater);
        uint64_t o = out_off[t];
        while (!heap.empty()) {
            std::pop_heap(heap.begin(), heap.end(), greater);
            const size_t r = heap.back().second;
            heap.pop_back();
            keys[o] = runs[r].host[pos[r]];
            if (counts) {
                const uint64_t v = runs[r].host[runs[r].n_items + pos[r]];
                if (n_samples == 2) {
                    counts[2 * o] = (uint32_t)v;
                    counts[2 * o + 1] = (uint32_t)(v >> 32);
                } else {
                    counts[o] = (uint32_t)v;
                }
            }
            ++o;
            if (++pos[r] < cut[t][r].second) {
                heap.push_back({runs[r].host[pos[r]], r});
                std::push_heap(heap.begin(), heap.end(), greater);
            }
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < T; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
}

void free_result(kc_handle h) {
    if (h->res_keys) cudaFreeAsync(h->res_keys, h->stream);
    if (h->res_vals) cudaFreeAsync(h->res_vals, h->stream);
    h->res_keys = h->res_vals = nullptr;
    h->n_result = h->res_cap = 0;
}

kc_status read_counters(kc_handle h) {
    KC_CUDA(cudaMemcpyAsync(&h->host_ctr, h->ctr, sizeof(kc::DevCounters), cudaMemcpyDeviceToHost, h->stream));
    KC_CUDA(cudaStreamSynchronize(h->stream));
    return KC_OK;
}

kc_status device_errors(kc_handle h) {
    const unsigned e = h->host_ctr.err;
    if (e & kc::DERR_OFFSETS) {
        h->state = State::Poisoned;
        return fail(KC_ERR_ARG, "read offsets decrease");
    }
    if (e & kc::DERR_TABLE_FULL) {
        h->state = State::Poisoned;
        return fail(KC_ERR_CAPACITY, "counting table full: raise kc_config.table_slots");
    }
    if (e & kc::DERR_COUNT_OVERFLOW) {
        h->state = State::Poisoned;
        return fail(KC_ERR_CAPACITY, "a per-sample count exceeded 2^32-1");
    }
    return KC_OK;
}

// Second partitioning level: every level-1 group of the batch is split into
// segments (several CTAs per group), each segment re-bucketed by the next a2
// bits of h with the same staged whole-sector scatter.  The batch then holds
// 2^(l1_bits + a2) partitions, exactly as a single level would give them.
kc_status regroup_batch(kc_handle h, Batch& b, cudaStream_t st) {
    const int a1 = h->l1_bits, a2 = h->part_bits - h->l1_bits;
    const uint64_t P1 = 1ull << a1, P2 = 1ull << a2, P = P1 * P2;
    std::vector<uint64_t> st1(P1 + 1);
    KC_CUDA(cudaMemcpyAsync(st1.data(), b.hstarts, (P1 + 1) * 8, cudaMemcpyDeviceToHost, st));
    KC_CUDA(cudaStreamSynchronize(st));
    const uint64_t total_in = st1[P1];
    const uint64_t chunk = std::max<uint64_t>(1ull << 16, total_in / ((uint64_t)h->grid.sm_count * 4) + 1);
    std::vector<kc::SegDesc> segs;
    std::vector<uint32_t> vlo(P1 + 1);
    for (uint64_t g = 0; g < P1; ++g) {
        vlo[g] = (uint32_t)segs.size();
        for (uint64_t o = st1[g]; o < st1[g + 1]; o += chunk)
            segs.push_back(kc::SegDesc{o, std::min(chunk, st1[g + 1] - o), g, 0});
    }
    vlo[P1] = (uint32_t)segs.size();
    const uint64_t nv = std::max<size_t>(1, segs.size());
    if (segs.empty()) segs.push_back(kc::SegDesc{0, 0, 0, 0});
    uint32_t *counts = nullptr, *total = nullptr, *dvlo = nullptr;
    uint64_t *rel = nullptr, *starts = nullptr, *cursor = nullptr, *out = nullptr;
    kc::SegDesc* dsegs = nullptr;
    const uint64_t cap = total_in + 3 * nv * P2;
    cudaError_t e;
    auto bail = [&](cudaError_t err) {
        for (void* q : {(void*)counts, (void*)total, (void*)dvlo, (void*)rel, (void*)starts, (void*)cursor,
                        (void*)out, (void*)dsegs})
            if (q) cudaFreeAsync(q, st);
        return cuda_fail(err, "cudaMallocAsync(second partitioning level)");
    };
    if ((e = cudaMallocAsync(&counts, nv * P2 * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&rel, nv * P2 * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&total, P * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&starts, (P + 1) * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&cursor, P * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&out, std::max<uint64_t>(1, cap) * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&dsegs, nv * sizeof(kc::SegDesc), st)) != cudaSuccess ||
        (e = cudaMallocAsync(&dvlo, (P1 + 1) * 4, st)) != cudaSuccess)
        return bail(e);
    KC_CUDA(cudaMemcpyAsync(dsegs, segs.data(), nv * sizeof(kc::SegDesc), cudaMemcpyHostToDevice, st));
    KC_CUDA(cudaMemcpyAsync(dvlo, vlo.data(), (P1 + 1) * 4, cudaMemcpyHostToDevice, st));
    kc::launch_count_seg(b.hdata, dsegs, (int)nv, a1, a2, counts, st);
    kc::launch_regroup_offsets(counts, dvlo, a1, a2, rel, total, st);
    if ((e = kc::launch_scan(total, P, starts, cursor, st)) != cudaSuccess) return bail(e);
    kc::launch_regroup_base(rel, starts, dsegs, nv, a2, st);
    kc::launch_scatter_staged_seg(b.hdata, dsegs, (int)nv, 1, a1, a2, rel, out, st);
    h->launches += 5;
    KC_LAUNCHED("second-level bucketing launches");
    for (void* q : {(void*)counts, (void*)total, (void*)dvlo, (void*)rel, (void*)cursor, (void*)dsegs})
        cudaFreeAsync(q, st);
    cudaFreeAsync(b.hdata, st);
    cudaFreeAsync(b.hstarts, st);
    b.hdata = out;
    b.hstarts = starts;
    b.hcap = cap;
    return KC_OK;
}

// Partitioned strategy, ingest: group the batch's window hashes by partition
// (count pass, per-partition prefix over CTAs, scan, scatter pass).  With more
// than 12 partition bits the hashes are first grouped by the top l1_bits, then
// every group is re-bucketed by the next 12 bits (regroup_batch).  Only
// windows whose hash lies in [p.h_lo, p.h_hi] are kept.  exact: the grouped
// hashes get exactly the room they need, read back after the scan (one
// synchronisation), instead of one slot per base of the batch.
int scatter_mode_of(kc_handle h) {
    int mode = h->cfg.scatter_mode ? (int)h->cfg.scatter_mode : 4;
    if (h->l1_bits != h->part_bits) mode = 4;  // two levels: staged scatter only
    int max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    const int a = h->l1_bits;
    if (mode >= 3 && std::max(kc::staged_scatter_smem(a), kc::staged_seg_smem(a)) > (size_t)max_optin) mode = 2;
    return mode;
}

kc_status bucket_batch(kc_handle h, Batch& b, uint64_t n_local, cudaStream_t st, const kc::PassParams& p,
                       bool exact, const ChunkedReads* chunks) {
    const int a = h->l1_bits;
    const uint64_t P = 1ull << a;
    const int mode = scatter_mode_of(h);
    if (chunks && mode != 4) {  // the other modes extract the whole batch at once: wait for every chunk
        for (int c = 0; c < chunks->n; ++c) KC_CUDA(cudaStreamWaitEvent(st, chunks->ev[c], 0));
        kc::launch_build_valid(chunks->nm, chunks->bd, b.n_units, chunks->start_local, chunks->n_local, h->k, b.vw,
                               h->ctr, h->grid, st);
        chunks = nullptr;
    }
    const int max_ctas = h->grid.sm_count * (h->cfg.ctas_per_sm ? (int)h->cfg.ctas_per_sm : 1);
    const uint64_t upc = std::max<uint64_t>(1, (b.n_units + max_ctas - 1) / max_ctas);
    // extraction CTAs: at most max_ctas over the batch; with chunks, the same
    // CTAs take a share of every chunk (segment c = its pieces in all chunks)
    const int n_ctas = (int)((b.n_units + upc - 1) / upc);
    const int n_pieces = chunks ? chunks->n : 1;
    uint32_t *counts = nullptr, *total = nullptr;
    uint64_t *rel = nullptr, *cursor = nullptr, *lin = nullptr, *g_cursor = nullptr;
    kc::SegDesc* seg = nullptr;
    // at most one window per base, plus run padding of up to 3 per (CTA, partition)
    b.hcap = n_local + (mode >= 3 ? 3ull * (uint64_t)n_ctas * P : 0ull);
    cudaError_t e = cudaSuccess;
    auto bail = [&](cudaError_t err) {
        if (counts) cudaFreeAsync(counts, st);
        if (rel) cudaFreeAsync(rel, st);
        if (total) cudaFreeAsync(total, st);
        if (cursor) cudaFreeAsync(cursor, st);
        if (lin) cudaFreeAsync(lin, st);
        if (seg) cudaFreeAsync(seg, st);
        if (g_cursor) cudaFreeAsync(g_cursor, st);
        if (b.hstarts) cudaFreeAsync(b.hstarts, st);
        if (b.hdata) cudaFreeAsync(b.hdata, st);
        b.hstarts = b.hdata = nullptr;
        return cuda_fail(err, "cudaMallocAsync(partition buckets)");
    };
    if ((e = cudaMallocAsync(&counts, (size_t)n_ctas * P * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&rel, (size_t)n_ctas * P * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&total, P * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&cursor, P * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&b.hstarts, (P + 1) * 8, st)) != cudaSuccess ||
        (!exact && (e = cudaMallocAsync(&b.hdata, std::max<uint64_t>(1, b.hcap) * 8, st)) != cudaSuccess))
        return bail(e);
    if (mode == 4 && ((e = cudaMallocAsync(&lin, std::max<uint64_t>(1, n_local) * 8, st)) != cudaSuccess ||
                      (e = cudaMallocAsync(&seg, (size_t)n_ctas * n_pieces * sizeof(kc::SegDesc), st)) != cudaSuccess ||
                      (e = cudaMallocAsync(&g_cursor, 8, st)) != cudaSuccess))
        return bail(e);
    if (mode == 4 && chunks) {
        KC_CUDA(cudaMemsetAsync(g_cursor, 0, 8, st));
        for (int c = 0; c < chunks->n; ++c) {
            const uint64_t u0 = chunks->u[c], nu = chunks->u[c + 1] - u0;
            const uint64_t upc_c = std::max<uint64_t>(1, (nu + n_ctas - 1) / n_ctas);
            KC_CUDA(cudaStreamWaitEvent(st, chunks->ev[c], 0));
            kc::launch_build_valid_range(chunks->nm, chunks->bd, b.n_units, u0, u0 + nu, chunks->start_local,
                                         chunks->n_local, h->k, b.vw, h->ctr, h->grid, st);
            kc::launch_extract_count(b.pw + 2 * u0, b.vw + u0, nu, upc_c, n_ctas, p, a, counts, g_cursor,
                                     seg + (size_t)c * n_ctas, lin, h->ctr, st, c > 0);
        }
        h->launches += 2 * (chunks->n - 1);
    } else if (mode == 4) {
        KC_CUDA(cudaMemsetAsync(g_cursor, 0, 8, st));
        kc::launch_extract_count(b.pw, b.vw, b.n_units, upc, n_ctas, p, a, counts, g_cursor, seg, lin, h->ctr, st);
    } else {
        kc::launch_bucket_count(b.pw, b.vw, b.n_units, upc, n_ctas, p, a, counts, st);
    }
    kc::launch_bucket_offsets(counts, n_ctas, a, mode >= 3 ? 1 : 0, rel, total, st);
    if ((e = kc::launch_scan(total, P, b.hstarts, cursor, st)) != cudaSuccess) return bail(e);
    if (exact) {  // the grouped hashes need exactly hstarts[P] slots
        uint64_t need = 0;
        KC_CUDA(cudaMemcpyAsync(&need, b.hstarts + P, 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        b.hcap = need;
        if ((e = cudaMallocAsync(&b.hdata, std::max<uint64_t>(1, need) * 8, st)) != cudaSuccess) return bail(e);
    }
    if (mode != 1) kc::launch_bucket_base(rel, b.hstarts, n_ctas, a, st);
    if (mode == 4) kc::launch_scatter_staged_seg(lin, seg, n_ctas, n_pieces, 0, a, rel, b.hdata, st);
    else kc::launch_bucket_scatter(b.pw, b.vw, b.n_units, upc, n_ctas, p, a, mode, rel, cursor, b.hdata, st);
    h->launches += mode != 1 ? 5 : 4;
    cudaFreeAsync(counts, st);
    cudaFreeAsync(rel, st);
    cudaFreeAsync(total, st);
    cudaFreeAsync(cursor, st);
    if (lin) cudaFreeAsync(lin, st);
    if (seg) cudaFreeAsync(seg, st);
    if (g_cursor) cudaFreeAsync(g_cursor, st);
    if (h->l1_bits != h->part_bits) return regroup_batch(h, b, st);
    return KC_OK;
}

// Batched ingest: every pending batch of the handles, extracted and grouped
// together on stream st (which the caller has ordered after each handle's
// stream).  Items of upi units (at least 2^12, about one per SM over all
// batches); per batch the histogram rows, segments, linear hashes and run
// bases live in one scratch block freed after the scatter, the grouped
// hashes (at most one per base plus run padding of 3 per (item, partition))
// and partition starts stay with the batch.  Batches of handles with two
// grouping levels are re-bucketed afterwards (regroup_batch).
kc_status ingest_pending(kc_handle* hs, int n, cudaStream_t st, int sm_count) {
    struct Ref {
        kc_handle h;
        size_t t;
    };
    std::vector<Ref> refs;
    uint64_t total_units = 0;
    for (int j = 0; j < n; ++j)
        for (size_t t = 0; t < hs[j]->batches.size(); ++t)
            if (hs[j]->batches[t].pending) {
                refs.push_back({hs[j], t});
                total_units += hs[j]->batches[t].n_units;
            }
    if (refs.empty()) return KC_OK;
    const uint64_t upi = std::max<uint64_t>(1ull << 12, (total_units + sm_count - 1) / sm_count);
    std::vector<kc::IngestBatch> ib(refs.size());
    std::vector<uint32_t> item_batch;
    std::vector<void*> scratch(refs.size(), nullptr);
    kc::IngestPlan plan{};
    bool ranged = false, all_k31 = true;
    auto bail = [&](cudaError_t e) {
        for (size_t i = 0; i < refs.size(); ++i) {
            if (scratch[i]) cudaFreeAsync(scratch[i], st);
            Batch& b = refs[i].h->batches[refs[i].t];
            if (b.hdata) cudaFreeAsync(b.hdata, st);
            if (b.hstarts) cudaFreeAsync(b.hstarts, st);
            b.hdata = b.hstarts = nullptr;
        }
        return cuda_fail(e, "cudaMallocAsync(batched ingest)");
    };
    for (size_t i = 0; i < refs.size(); ++i) {
        kc_handle h = refs[i].h;
        Batch& b = h->batches[refs[i].t];
        kc::IngestBatch& B = ib[i];
        const uint64_t P = 1ull << h->l1_bits;
        B.pw = b.pw;
        B.vw = b.vw;
        B.n_units = b.n_units;
        B.p = h->params(b.sample);  // keeps the handle's own hash range
        ranged |= B.p.h_lo != 0ull || B.p.h_hi != ~0ull;
        all_k31 &= h->k == 31;
        B.a = h->l1_bits;
        B.item0 = (uint32_t)item_batch.size();
        B.n_items = (uint32_t)((b.n_units + upi - 1) / upi);
        B.upi = upi;
        B.ctr = h->ctr;
        B.bucket_off = plan.n_buckets;
        B.rel_off = plan.n_rel;
        plan.n_buckets += P;
        plan.n_rel += (uint64_t)B.n_items * P;
        plan.max_a = std::max(plan.max_a, B.a);
        item_batch.insert(item_batch.end(), B.n_items, (uint32_t)i);
        // scratch: counts, relative bases, segments, totals, cursor, linear hashes
        const uint64_t cells = (uint64_t)B.n_items * P;
        const uint64_t bytes = cells * 4 + cells * 8 + B.n_items * sizeof(kc::SegDesc) + P * 4 + 8 + b.n_local * 8 + 64;
        cudaError_t e;
        if ((e = cudaMallocAsync(&scratch[i], bytes, st)) != cudaSuccess) return bail(e);
        char* q = static_cast<char*>(scratch[i]);
        B.rel = reinterpret_cast<uint64_t*>(q);
        q += cells * 8;
        B.seg = reinterpret_cast<kc::SegDesc*>(q);
        q += B.n_items * sizeof(kc::SegDesc);
        B.lin = reinterpret_cast<uint64_t*>(q);
        q += b.n_local * 8;
        B.g_cursor = reinterpret_cast<unsigned long long*>(q);
        q += 8;
        B.counts = reinterpret_cast<uint32_t*>(q);
        q += cells * 4;
        B.total = reinterpret_cast<uint32_t*>(q);
        b.hcap = b.n_local + 3 * cells;
        if ((e = cudaMallocAsync(&b.hstarts, (P + 1) * 8, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&b.hdata, std::max<uint64_t>(1, b.hcap) * 8, st)) != cudaSuccess)
            return bail(e);
        B.starts = b.hstarts;
        B.out = b.hdata;
        KC_CUDA(cudaMemsetAsync(B.g_cursor, 0, 8, st));
    }
    plan.n_batches = (uint32_t)refs.size();
    plan.n_items = (uint32_t)item_batch.size();
    // the plan, its batches, item map and queue heads in one device block
    const size_t bytes = sizeof(kc::IngestPlan) + ib.size() * sizeof(kc::IngestBatch) + item_batch.size() * 4 + 16;
    char* blk = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&blk), bytes, st)) != cudaSuccess) return bail(e);
    kc::IngestPlan* dplan = reinterpret_cast<kc::IngestPlan*>(blk);
    kc::IngestBatch* dbat = reinterpret_cast<kc::IngestBatch*>(blk + sizeof(kc::IngestPlan));
    unsigned* dhead = reinterpret_cast<unsigned*>(blk + sizeof(kc::IngestPlan) + ib.size() * sizeof(kc::IngestBatch));
    uint32_t* ditems = dhead + 4;
    plan.batches = dbat;
    plan.item_batch = ditems;
    plan.head = dhead;
    KC_CUDA(cudaMemcpyAsync(dbat, ib.data(), ib.size() * sizeof(kc::IngestBatch), cudaMemcpyHostToDevice, st));
    KC_CUDA(cudaMemcpyAsync(ditems, item_batch.data(), item_batch.size() * 4, cudaMemcpyHostToDevice, st));
    KC_CUDA(cudaMemsetAsync(dhead, 0, 16, st));
    KC_CUDA(cudaMemcpyAsync(dplan, &plan, sizeof(plan), cudaMemcpyHostToDevice, st));
    const bool timed = n == 1;
    cudaEvent_t t0 = timed ? phase_begin(hs[0], st) : nullptr;
    kc::launch_ingest(dplan, plan, ranged, all_k31, sm_count, st);
    KC_LAUNCHED("batched ingest launches");
    if (timed) phase_end(hs[0], kPass1, t0, st);
    cudaFreeAsync(blk, st);
    for (size_t i = 0; i < refs.size(); ++i) {
        cudaFreeAsync(scratch[i], st);
        Batch& b = refs[i].h->batches[refs[i].t];
        cudaFreeAsync(b.pw, st);  // the hashes replace the reads
        cudaFreeAsync(b.vw, st);
        b.pw = b.vw = nullptr;
        b.pending = false;
    }
    for (int j = 0; j < n; ++j) hs[j]->launches += 5;
    for (const Ref& r : refs) {
        kc_handle h = r.h;
        if (h->l1_bits != h->part_bits) {
            kc_status s = regroup_batch(h, h->batches[r.t], st);
            if (s != KC_OK) return s;
        }
    }
    return KC_OK;
}

uint64_t bucket_bytes(kc_handle h, uint64_t n_local);

// Device bytes the handle holds now: filter, table and counters, resident
// batches (reads and grouped hashes) and its result.
uint64_t held_bytes(kc_handle h) {
    uint64_t bytes = h->fixed_bytes + h->res_cap * 16;
    for (const auto& b : h->batches) {
        if (b.pw) bytes += (2 * b.n_units + 2) * 8 + b.n_units * 8;
        if (b.hdata) bytes += b.hcap * 8 + ((1ull << h->part_bits) + 1) * 8;
        if (b.pending) bytes += bucket_bytes(h, b.n_local);  // the grouping still to come
    }
    return bytes;
}

// Bytes the handle may still allocate: kc_config.device_budget minus what it
// holds, or (no budget) the device's free memory plus what the stream-ordered
// pool has cached and not handed out, less a 1 GiB margin.
uint64_t room_bytes(kc_handle h) {
    const uint64_t held = held_bytes(h);
    if (h->cfg.device_budget) return h->cfg.device_budget > held ? h->cfg.device_budget - held : 0;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return ~0ull;  // unknown: do not defer
    }
    uint64_t cached = 0;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            cached = reserved - used;
        else
            cudaGetLastError();
    }
    const uint64_t avail = (uint64_t)free_b + cached, margin = 1ull << 30;
    return avail > margin ? avail - margin : 0;
}

// Device bytes bucket_batch needs for a batch of n_local bases: the linear
// hashes and the grouped hashes (8 bytes per window each, at most one window
// per base), and the run padding of up to 3 per (CTA, partition).
uint64_t bucket_bytes(kc_handle h, uint64_t n_local) {
    const int max_ctas = h->grid.sm_count * (h->cfg.ctas_per_sm ? (int)h->cfg.ctas_per_sm : 1);
    return 16 * n_local + 24ull * (uint64_t)max_ctas * (1ull << h->l1_bits) +
           (uint64_t)max_ctas * (1ull << h->l1_bits) * 12;
}

// Sort n (key, value) pairs held in tk/tv, keys below 2^key_bits, into
// out_k/out_v (n entries each): bucket by the top key bits (at most about 32
// keys a bucket), then sort every bucket: one warp per bucket in registers,
// larger buckets in shared memory or, rarely, global memory.  ctr->survivors
// must hold n on the device; ctr->err collects the kernels' flags (and is
// cleared of the sort flags again).  Synchronises the stream.  Device time
// goes to `phase`.
kc_status sort_pairs(kc_handle h, const uint64_t* tk, const uint64_t* tv, uint64_t n, int key_bits,
                     kc::DevCounters* ctr, uint64_t* out_k, uint64_t* out_v, int phase) {
    cudaStream_t st = h->stream;
    const uint64_t cap = std::max<uint64_t>(1, n);
    int bits = 0;
    while (bits < 24 && bits < key_bits && (cap >> bits) > 32) ++bits;
    const uint64_t n_buckets = 1ull << bits;
    const int prefix_shift = key_bits - bits;
    uint64_t *starts = nullptr, *cursor = nullptr;
    uint32_t* hist = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(&hist, n_buckets * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&starts, (n_buckets + 1) * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&cursor, n_buckets * 8, st)) != cudaSuccess) {
        if (hist) cudaFreeAsync(hist, st);
        if (starts) cudaFreeAsync(starts, st);
        return cuda_fail(e, "cudaMallocAsync(sort buffers)");
    }
    auto release = [&]() {
        cudaFreeAsync(hist, st);
        cudaFreeAsync(starts, st);
        cudaFreeAsync(cursor, st);
    };
    cudaEvent_t t0 = phase_begin(h);
    KC_CUDA(cudaMemsetAsync(hist, 0, n_buckets * 4, st));
    kc::launch_prefix_hist(tk, ctr, n, prefix_shift, n_buckets, hist, h->grid, st);
    KC_CUDA(kc::launch_scan(hist, n_buckets, starts, cursor, st));
    kc::launch_scatter(tk, tv, ctr, n, prefix_shift, n_buckets, cursor, out_k, out_v, h->grid, st);
    kc::launch_bucket_sort_warp(out_k, out_v, starts, n_buckets, prefix_shift, ctr, h->grid, st);
    phase_end(h, phase, t0);
    h->launches += 4;
    KC_LAUNCHED("sort launches");
    unsigned err = 0;
    KC_CUDA(cudaMemcpyAsync(&err, &ctr->err, 4, cudaMemcpyDeviceToHost, st));
    KC_CUDA(cudaStreamSynchronize(st));
    if (err & kc::DERR_INTERNAL) {
        release();
        h->state = State::Poisoned;
        return fail(KC_ERR_INTERNAL, "sort: key outside its bucket range");
    }
    if (err & kc::DERR_SORT_MEDIUM) {
        kc::launch_bucket_sort(out_k, out_v, starts, n_buckets, ctr, st);
        h->launches += 1;
        KC_LAUNCHED("medium sort launch");
        KC_CUDA(cudaMemcpyAsync(&err, &ctr->err, 4, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
    }
    if (err & kc::DERR_SORT_BUCKET) {
        // Rare: a bucket larger than the shared-memory tile; sort it in global memory.
        std::vector<uint64_t> hs(n_buckets + 1);
        KC_CUDA(cudaMemcpyAsync(hs.data(), starts, (n_buckets + 1) * 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        const uint64_t capb = (uint64_t)kc::bucket_sort_capacity();
        for (uint64_t i = 0; i < n_buckets; ++i)
            if (hs[i + 1] - hs[i] > capb) {
                uint64_t m = hs[i + 1] - hs[i], m2 = 1, steps = 0;
                while (m2 < m) m2 <<= 1;
                for (uint64_t size = 2; size <= m2; size <<= 1)
                    for (uint64_t stride = size >> 1; stride > 0; stride >>= 1) ++steps;
                kc::launch_bitonic_global(out_k + hs[i], out_v + hs[i], m, st);
                h->launches += steps;
            }
        KC_LAUNCHED("global sort launches");
    }
    if (err & (kc::DERR_SORT_MEDIUM | kc::DERR_SORT_BUCKET)) {
        const unsigned keep = err & ~(kc::DERR_SORT_MEDIUM | kc::DERR_SORT_BUCKET);
        KC_CUDA(cudaMemcpyAsync(&ctr->err, &keep, 4, cudaMemcpyHostToDevice, st));
    }
    release();
    KC_CUDA(cudaStreamSynchronize(st));
    return KC_OK;
}

// Sort the survivors held in tk/tv (count in host_ctr.survivors, already
// read back and on the device in ctr->survivors) into res_keys/res_vals.
kc_status sort_result(kc_handle h, uint64_t* tk, uint64_t* tv) {
    cudaStream_t st = h->stream;
    const uint64_t n = h->host_ctr.survivors;
    const uint64_t cap = std::max<uint64_t>(1, n);
    free_result(h);
    cudaError_t e;
    if ((e = cudaMallocAsync(&h->res_keys, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&h->res_vals, cap * 8, st)) != cudaSuccess) {
        free_result(h);
        return cuda_fail(e, "cudaMallocAsync(result)");
    }
    h->res_cap = cap;
    kc_status s = sort_pairs(h, tk, tv, n, 2 * h->k, h->ctr, h->res_keys, h->res_vals, kSort);
    if (s != KC_OK) return s;
    if ((s = read_counters(h)) != KC_OK) return s;
    phase_collect(h);
    h->n_result = n;
    return KC_OK;
}

kc_status finalize_direct(kc_handle h) {
    cudaStream_t st = h->stream;
    cudaEvent_t t0 = phase_begin(h);
    for (const auto& b : h->batches) {
        if (h->bloom2)
            kc::launch_count_chain(b.pw, b.vw, b.n_units, h->params(b.sample), h->bloom2, h->table, h->ctr, h->grid,
                                   st);
        else
            kc::launch_pass2(b.pw, b.vw, b.n_units, h->params(b.sample), h->table, h->ctr, h->grid, st);
    }
    phase_end(h, kPass2, t0);
    h->launches += h->batches.size();
    KC_LAUNCHED("direct recount launch");
    kc_status s = read_counters(h);
    if (s != KC_OK) return s;
    if ((s = device_errors(h)) != KC_OK) return s;
    const uint64_t cap = std::max<uint64_t>(1, h->host_ctr.claimed);
    uint64_t *tk = nullptr, *tv = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(&tk, cap * 8, st)) != cudaSuccess || (e = cudaMallocAsync(&tv, cap * 8, st)) != cudaSuccess) {
        if (tk) cudaFreeAsync(tk, st);
        return cuda_fail(e, "cudaMallocAsync(compaction)");
    }
    KC_CUDA(cudaMemsetAsync(&h->ctr->survivors, 0, 8, st));
    t0 = phase_begin(h);
    kc::launch_compact(h->table, h->n_slots, h->n_samples, h->min_count, tk, tv, h->ctr, nullptr, 0, h->grid, st);
    phase_end(h, kCompact, t0);
    h->launches += 1;
    KC_LAUNCHED("direct compaction launches");
    if ((s = read_counters(h)) != KC_OK) return s;
    s = sort_result(h, tk, tv);
    cudaFreeAsync(tk, st);
    cudaFreeAsync(tv, st);
    return s;
}

// One finalize engine per device, shared by every handle (its buffers and
// captured sort graph are reused); calls on it are serialised.
std::mutex g_engine_mutex;
kc_batch_ctx* g_engines[64] = {};

kc_status finalize_partitioned(kc_handle h) {
    if (h->device < 0 || h->device >= 64) return fail(KC_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_engine_mutex);
    if (!g_engines[h->device]) {
        kc_status s = kc_batch_create_internal(nullptr, &g_engines[h->device]);
        if (s != KC_OK) return s;
    }
    return kc_batch_finalize_internal(g_engines[h->device], &h, 1);
}

// A spilled result back on the device: the runs are copied into one device
// array and sorted there as one survivor set (sort_result), after which the
// handle holds its result on the device like an unspilled one.
// KC_ERR_OOM_DEVICE (nothing changed, no error recorded) when the device has
// no room for it.
kc_status resort_spilled(kc_handle h) {
    const uint64_t n = h->n_result;
    cudaStream_t st = h->stream;
    uint64_t *tk = nullptr, *tv = nullptr;
    if (cudaMallocAsync(&tk, n * 8, st) != cudaSuccess || cudaMallocAsync(&tv, n * 8, st) != cudaSuccess) {
        cudaGetLastError();
        if (tk) cudaFreeAsync(tk, st);
        return KC_ERR_OOM_DEVICE;
    }
    uint64_t off = 0;
    for (const auto& r : h->spill_dir) {
        if (!r.n_items) continue;
        KC_CUDA(cudaMemcpyAsync(tk + off, r.host, r.n_items * 8, cudaMemcpyHostToDevice, st));
        KC_CUDA(cudaMemcpyAsync(tv + off, r.host + r.n_items, r.n_items * 8, cudaMemcpyHostToDevice, st));
        off += r.n_items;
    }
    h->host_ctr.survivors = n;
    KC_CUDA(cudaMemcpyAsync(&h->ctr->survivors, &h->host_ctr.survivors, 8, cudaMemcpyHostToDevice, st));
    const uint64_t spilled_bytes = h->spilled_bytes;
    kc_status s = sort_result(h, tk, tv);  // synchronises the stream (reads the counters)
    cudaFreeAsync(tk, st);
    cudaFreeAsync(tv, st);
    if (s != KC_OK) return s;
    release_spill(h);  // the pinned chunks stay for the next job
    h->spilled_bytes = spilled_bytes;
    h->n_result = n;
    return KC_OK;
}

// 2^pb partitions: the grouping levels, the filter slice of a partition and
// an owner's partition range follow.
void set_partitions(kc_handle h, int pb) {
    h->part_bits = pb;
    h->l1_bits = pb <= 12 ? pb : pb - 12;
    h->slice_log2 = h->log2_words - pb;
    h->own_plo = 0;
    h->own_phi = h->strategy == KC_STRATEGY_PARTITIONED ? (1u << pb) : 0u;
    if (h->owner) {
        const int ob = (int)h->cfg.own_bits;
        const uint64_t hi = h->cfg.own_hi ? h->cfg.own_hi : (1ull << ob);
        h->own_plo = h->cfg.own_lo << (pb - ob);
        h->own_phi = (uint32_t)(hi << (pb - ob));
    }
}

// Partition bits chosen by the library (kc_config.part_bits = 0): at the
// first kc_add_reads after create / reset, enough partitions, up to 2^12 (one
// grouping level) and filter slices of at least 8 words, for at most
// kWindowsPerPartition windows each, estimated as bases - reads * (k - 1) of
// this call; never fewer than the filter's own (slices of 4096 words).  The
// consumer counts a partition's windows in one pass over its hashes while
// they number at most its threads * 64, and a partition of fewer windows
// holds fewer keys in its shared-memory table.
void choose_partitions(kc_handle h, uint64_t bases, uint64_t n_reads) {
    if (!h->auto_part || !h->batches.empty()) return;
    const uint64_t edge = n_reads * (uint64_t)(h->k - 1);
    const uint64_t est = bases > edge ? bases - edge : 0;
    int want = 0;
    while (want < 12 && (est >> want) > kWindowsPerPartition) ++want;
    const int pb = std::max(h->base_part_bits, std::min(want, h->log2_words - 3));
    if (pb != h->part_bits) set_partitions(h, pb);
}

}  // namespace kcapi

using namespace kcapi;

extern "C" {

void kc_default_config(kc_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(kc_config);
}

const char* kc_last_error(void) { return g_last_error.c_str(); }

const char* kc_status_string(kc_status s) {
    switch (s) {
        case KC_OK: return "KC_OK";
        case KC_ERR_ARG: return "KC_ERR_ARG";
        case KC_ERR_STATE: return "KC_ERR_STATE";
        case KC_ERR_OOM_DEVICE: return "KC_ERR_OOM_DEVICE";
        case KC_ERR_OOM_HOST: return "KC_ERR_OOM_HOST";
        case KC_ERR_CUDA: return "KC_ERR_CUDA";
        case KC_ERR_TIMEOUT: return "KC_ERR_TIMEOUT";
        case KC_ERR_CAPACITY: return "KC_ERR_CAPACITY";
        case KC_ERR_INTERNAL: return "KC_ERR_INTERNAL";
    }
    return "KC_ERR_UNKNOWN";
}

kc_status kc_create(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count, kc_handle* out) {
    return kc_create_ex(k, n_samples, bloom_bits, n_hashes, min_count, nullptr, nullptr, out);
}

kc_status kc_create_ex(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                       const kc_config* cfg, void* stream, kc_handle* out) {
    g_last_error.clear();
    if (!out) return fail(KC_ERR_ARG, "out is null");
    *out = nullptr;
    if (k < 1 || k > 31) return fail(KC_ERR_ARG, "k must be in 1..31");
    if (n_samples < 1 || n_samples > 2) return fail(KC_ERR_ARG, "n_samples must be 1 or 2");
    if (!is_pow2(bloom_bits) || bloom_bits < 4096) return fail(KC_ERR_ARG, "bloom_bits must be a power of two >= 4096");
    if (n_hashes < 1 || n_hashes > 10) return fail(KC_ERR_ARG, "n_hashes must be in 1..10");
    if (min_count < 1) return fail(KC_ERR_ARG, "min_count must be >= 1");
    kc_config c;
    kc_default_config(&c);
    if (cfg) {
        if (cfg->struct_size < offsetof(kc_config, timing)) return fail(KC_ERR_ARG, "kc_config.struct_size");
        std::memcpy(&c, cfg, std::min<size_t>(cfg->struct_size, sizeof(c)));
        c.struct_size = sizeof(c);
    }
    uint64_t slots = c.table_slots ? c.table_slots : std::max<uint64_t>(1ull << 12, bloom_bits / 32);
    if (!is_pow2(slots) || slots < 1024) return fail(KC_ERR_ARG, "table_slots must be a power of two >= 1024");
    if (c.block_threads && c.block_threads != 256) return fail(KC_ERR_ARG, "block_threads must be 256");
    if (c.strategy > KC_STRATEGY_PARTITIONED) return fail(KC_ERR_ARG, "unknown strategy");
    if (c.part_bits > 20) return fail(KC_ERR_ARG, "part_bits must be <= 20");
    if (c.scatter_mode > 4) return fail(KC_ERR_ARG, "scatter_mode must be in 0..4");
    if (c.smem_table_log2 && (c.smem_table_log2 < 10 || c.smem_table_log2 > 13))
        return fail(KC_ERR_ARG, "smem_table_log2 must be in 10..13");
    if (c.split_max != KC_SPLIT_NONE && c.split_max > 13) return fail(KC_ERR_ARG, "split_max must be in 0..13");
    if (c.spill > 2) return fail(KC_ERR_ARG, "spill must be 0, 1 or 2");
    if (c.ctas_per_sm > 64) return fail(KC_ERR_ARG, "ctas_per_sm must be in 0..64");
    if (c.prune_chain > 1) return fail(KC_ERR_ARG, "prune_chain must be 0 or 1");
    if (c.prune_chain && c.strategy == KC_STRATEGY_PARTITIONED)
        return fail(KC_ERR_ARG, "prune_chain runs on the direct strategy");
    // Partitions: filter slices of 4096 words (32 KiB) unless set; the
    // partitioned strategy needs a slice of at most 8192 words in shared memory.
    const int lw = log2_exact(bloom_bits / 64);
    int pb = c.part_bits ? (int)c.part_bits : std::min(20, std::max(1, lw - 12));
    pb = std::min(pb, lw);
    const bool part_ok = lw - pb <= 13 && pb >= 1;
    int strategy = (int)c.strategy;
    if (strategy == KC_STRATEGY_AUTO)
        strategy = part_ok && !c.prune_chain ? KC_STRATEGY_PARTITIONED : KC_STRATEGY_DIRECT;
    if (strategy == KC_STRATEGY_PARTITIONED && !part_ok)
        return fail(KC_ERR_ARG, "partitioned strategy: filter slice per partition exceeds 8192 words");

    if (c.own_bits) {
        if (strategy != KC_STRATEGY_PARTITIONED)
            return fail(KC_ERR_ARG, "own_bits needs the partitioned strategy");
        if ((int)c.own_bits > pb) return fail(KC_ERR_ARG, "own_bits must not exceed the partition bits");
        const uint64_t n_shards = 1ull << c.own_bits, hi = c.own_hi ? c.own_hi : n_shards;
        if (c.own_lo >= hi || hi > n_shards) return fail(KC_ERR_ARG, "owned shards must satisfy own_lo < own_hi <= 2^own_bits");
    } else if (c.own_lo || c.own_hi) {
        return fail(KC_ERR_ARG, "own_lo / own_hi need own_bits");
    }

    kc_ctx* h = new (std::nothrow) kc_ctx();
    if (!h) return fail(KC_ERR_OOM_HOST, "host allocation");
    h->k = k;
    h->n_samples = n_samples;
    h->bloom_bits = bloom_bits;
    h->n_hashes = n_hashes;
    h->min_count = min_count;
    h->cfg = c;
    h->log2_words = log2_exact(bloom_bits / 64);
    h->strategy = strategy;
    if (strategy == KC_STRATEGY_PARTITIONED) slots = 0;
    if (c.own_bits) {
        const int ob = (int)c.own_bits;
        const uint64_t hi = c.own_hi ? c.own_hi : (1ull << ob);
        h->owner = true;
        h->own_h_lo = (uint64_t)c.own_lo << (64 - ob);
        h->own_h_hi = (hi << (64 - ob)) - 1ull;  // hi = 2^ob wraps to 0, giving ~0
    }
    set_partitions(h, pb);
    h->auto_part = strategy == KC_STRATEGY_PARTITIONED && c.part_bits == 0;
    h->base_part_bits = pb;
    h->n_slots = slots;
    h->log2_slots = slots ? log2_exact(slots) : 0;

    auto bail = [&](kc_status s) {
        kc_destroy(h);
        return s;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->grid.sm_count = sms > 0 ? sms : 152;
    h->grid.ctas_per_sm = c.ctas_per_sm ? (int)c.ctas_per_sm : 8;
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
        h->own_stream = true;
    }
    if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_copy, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_main, cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "stream/event create"));
    // Keep freed stream-ordered allocations cached for the next job.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    const size_t bloom_bytes = bloom_bits / 8, table_bytes = slots * sizeof(kc::Slot);
    // stream-ordered pool allocations: no device-wide synchronisation
    if ((e = cudaMallocAsync(&h->bloom, bloom_bytes, h->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocAsync(filter)"));
    if (table_bytes && (e = cudaMallocAsync(&h->table, table_bytes, h->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocAsync(table)"));
    if (c.prune_chain && (e = cudaMallocAsync(&h->bloom2, bloom_bytes, h->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocAsync(second filter)"));
    if ((e = cudaMallocAsync(&h->ctr, sizeof(kc::DevCounters), h->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocAsync(counters)"));
    h->fixed_bytes = bloom_bytes * (c.prune_chain ? 2 : 1) + table_bytes + sizeof(kc::DevCounters);
    kc_status s = kc_reset(h);
    if (s != KC_OK) return bail(s);
    *out = h;
    return KC_OK;
}

kc_status kc_reset(kc_handle h) {
    if (!h) return fail(KC_ERR_ARG, "null handle");
    free_batches(h);
    h->n_result = 0;  // the result arrays stay allocated for the next job (finalize reuses them)
    free_selection(h);
    free_stems(h);
    h->filter_windows = h->filter_hits = 0;
    if (!h->spill_dir.empty()) {
        cudaStreamSynchronize(h->copy_stream);
        release_spill(h);
    }
    // The partition consumer writes back every word of every partition's
    // filter slice (fallback partitions clear theirs first), so a partitioned
    // handle that owns every key needs no cleared filter; an owner of a hash
    // range keeps the other slices at zero.
    if (h->strategy != KC_STRATEGY_PARTITIONED || h->owner)
        KC_CUDA(cudaMemsetAsync(h->bloom, 0, h->bloom_bits / 8, h->stream));
    if (h->bloom2) KC_CUDA(cudaMemsetAsync(h->bloom2, 0, h->bloom_bits / 8, h->stream));
    if (h->table) KC_CUDA(cudaMemsetAsync(h->table, 0, h->n_slots * sizeof(kc::Slot), h->stream));
    KC_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(kc::DevCounters), h->stream));
    h->bases = 0;
    h->reads = 0;
    std::memset(&h->host_ctr, 0, sizeof(h->host_ctr));
    for (const auto& m : h->marks) {
        h->ev_pool.push_back(m.a);
        h->ev_pool.push_back(m.b);
    }
    h->marks.clear();
    for (double& x : h->ms) x = 0.0;
    h->launches = 0;
    h->fallback_partitions = 0;
    h->deferred = h->scan_groups = 0;
    h->state = State::Open;
    return KC_OK;
}

void kc_destroy(kc_handle h) {
    if (!h) return;
    if (h->stream) {
        free_batches(h);
        free_result(h);
        free_selection(h);
        free_stems(h);
        if (!h->spill_dir.empty()) cudaStreamSynchronize(h->copy_stream);
        release_spill(h);
        free_spill_chunks(h);
        if (h->bloom) cudaFreeAsync(h->bloom, h->stream);
        if (h->bloom2) cudaFreeAsync(h->bloom2, h->stream);
        if (h->table) cudaFreeAsync(h->table, h->stream);
        if (h->ctr) cudaFreeAsync(h->ctr, h->stream);
        if (h->chk_ctr) cudaFreeAsync(h->chk_ctr, h->copy_stream);
    }
    for (const auto& m : h->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->ev_copy) cudaEventDestroy(h->ev_copy);
    if (h->ev_main) cudaEventDestroy(h->ev_main);
    for (cudaEvent_t e : h->ev_chunk)
        if (e) cudaEventDestroy(e);
    if (h->pinned) {
        std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
        cudaFreeHost(h->pinned);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"

namespace kcapi {

// The handle's pinned readback words (8), allocated at first use.
cudaError_t pinned_words(kc_handle h) {
    if (h->pinned) return cudaSuccess;
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());  // pinning may synchronise the device
    return cudaMallocHost(&h->pinned, 8 * sizeof(uint64_t));
}

// kc_add_reads of host reads in n_chunks chunks (the read store b.pw / b.vw
// and the scratch nm, bd, doff are allocated on the copy stream; all are
// freed here, the grouped hashes replacing the reads).  On the copy stream: the offsets,
// their check (read starts marked into bd, error bits into chk_ctr), then
// each chunk's packed and N-mask words.  On the handle's stream, after the
// check: per chunk its valid-window bits and extraction, then the grouping.
kc_status add_reads_chunked(kc_handle h, Batch& b, int sample, const uint64_t* packed_reads, const uint64_t* offsets,
                            const uint64_t* n_mask, uint64_t n_reads, uint64_t b0, uint64_t b1, int n_chunks,
                            uint64_t* nm, uint64_t* bd, uint64_t* doff) {
    cudaStream_t st = h->stream, cs = h->copy_stream;
    const uint64_t B = (b0 / 64) * 64;
    const uint64_t n_local = b1 - B;
    const uint64_t n_units = b.n_units;
    const uint64_t n_pwords_src = (n_local + 31) / 32;
    const uint64_t n_pwords = 2 * n_units + 2;
    auto release = [&]() {
        for (void* q : {(void*)b.pw, (void*)b.vw, (void*)nm, (void*)bd, (void*)doff}) cudaFreeAsync(q, cs);
        b.pw = b.vw = nullptr;
    };
    cudaError_t e = cudaSuccess;
    // the check's device counters (stream-ordered on the copy stream) and the
    // pinned word its error bits come back to, both kept with the handle
    if (!h->chk_ctr && (e = cudaMallocAsync(&h->chk_ctr, sizeof(kc::DevCounters), cs)) != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaMallocAsync(offsets check)");
    }
    if ((e = pinned_words(h)) != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaMallocHost(offsets check)");
    }
    unsigned* chk_host = reinterpret_cast<unsigned*>(h->pinned);
    for (int c = 0; c <= n_chunks; ++c)
        if (!h->ev_chunk[c] && (e = cudaEventCreateWithFlags(&h->ev_chunk[c], cudaEventDisableTiming)) != cudaSuccess) {
            release();
            return cuda_fail(e, "cudaEventCreate(chunks)");
        }
    ChunkedReads ch;
    ch.n = n_chunks;
    for (int c = 0; c <= n_chunks; ++c) ch.u[c] = n_units * (uint64_t)c / (uint64_t)n_chunks;
    for (int c = 0; c < n_chunks; ++c) ch.ev[c] = h->ev_chunk[c];
    ch.nm = nm;
    ch.bd = bd;
    ch.start_local = b0 - B;
    ch.n_local = n_local;
    // copy stream: offsets, their check, then the chunks
    KC_CUDA(cudaMemsetAsync(b.pw + n_pwords_src, 0, (n_pwords - n_pwords_src) * 8, cs));
    KC_CUDA(cudaMemcpyAsync(doff, offsets, (n_reads + 1) * 8, cudaMemcpyDefault, cs));
    KC_CUDA(cudaMemsetAsync(h->chk_ctr, 0, sizeof(kc::DevCounters), cs));
    KC_CUDA(cudaMemsetAsync(bd, 0, n_units * 8, cs));
    kc::launch_mark_read_starts(doff, n_reads, B, n_local, bd, h->chk_ctr, cs);
    KC_CUDA(cudaMemcpyAsync(chk_host, &h->chk_ctr->err, sizeof(unsigned), cudaMemcpyDeviceToHost, cs));
    KC_CUDA(cudaEventRecord(h->ev_chunk[n_chunks], cs));  // the check
    for (int c = 0; c < n_chunks; ++c) {
        const uint64_t u0 = ch.u[c], u1 = ch.u[c + 1];
        // the chunk's words and the next unit's first word (its last unit's successor)
        const uint64_t w0 = 2 * u0, w1 = std::min<uint64_t>(2 * u1 + 1, n_pwords_src);
        if (w1 > w0) KC_CUDA(cudaMemcpyAsync(b.pw + w0, packed_reads + B / 32 + w0, (w1 - w0) * 8, cudaMemcpyDefault, cs));
        const uint64_t m1 = std::min<uint64_t>(u1 + 1, n_units);
        KC_CUDA(cudaMemcpyAsync(nm + u0, n_mask + B / 64 + u0, (m1 - u0) * 8, cudaMemcpyDefault, cs));
        KC_CUDA(cudaEventRecord(h->ev_chunk[c], cs));
    }
    KC_LAUNCHED("offsets check launch");
    KC_CUDA(cudaEventSynchronize(h->ev_chunk[n_chunks]));
    if (*chk_host & kc::DERR_OFFSETS) {
        KC_CUDA(cudaStreamSynchronize(cs));  // the caller's arrays are no longer read
        release();
        return fail(KC_ERR_ARG, "read offsets decrease");
    }
    // handle's stream: the chunks' valid bits and extraction, the grouping
    KC_CUDA(cudaStreamWaitEvent(st, h->ev_chunk[n_chunks], 0));
    cudaEvent_t t0 = phase_begin(h);
    kc_status s = bucket_batch(h, b, n_local, st, h->params(sample), false, &ch);
    phase_end(h, kPass1, t0);
    if (s != KC_OK) {
        KC_CUDA(cudaStreamSynchronize(cs));
        for (void* q : {(void*)nm, (void*)bd, (void*)doff, (void*)b.pw, (void*)b.vw}) cudaFreeAsync(q, st);
        b.pw = b.vw = nullptr;
        return s;
    }
    h->launches += 4;
    KC_LAUNCHED("ingest launches");
    for (void* q : {(void*)nm, (void*)bd, (void*)doff, (void*)b.pw, (void*)b.vw}) cudaFreeAsync(q, st);
    b.pw = b.vw = nullptr;  // the hashes replace the reads: nothing rescans them
    KC_CUDA(cudaEventSynchronize(h->ev_chunk[n_chunks - 1]));  // caller may reuse its arrays
    return KC_OK;
}

}  // namespace kcapi

extern "C" {

kc_status kc_add_reads(kc_handle h, int sample, const uint64_t* packed_reads, const uint64_t* offsets,
                       const uint64_t* n_mask, uint64_t n_reads) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (h->state != State::Open) return fail(KC_ERR_STATE, "kc_add_reads after kc_finalize");
    if (sample < 0 || sample >= h->n_samples) return fail(KC_ERR_ARG, "sample out of range");
    if (n_reads == 0) return KC_OK;
    if (!offsets) return fail(KC_ERR_ARG, "offsets is null");

    const bool off_dev = is_device_ptr(offsets);
    uint64_t b0, b1;
    if (off_dev) {
        KC_CUDA(pinned_words(h));
        KC_CUDA(cudaMemcpyAsync(h->pinned + 1, offsets, 8, cudaMemcpyDeviceToHost, h->stream));
        KC_CUDA(cudaMemcpyAsync(h->pinned + 2, offsets + n_reads, 8, cudaMemcpyDeviceToHost, h->stream));
        KC_CUDA(cudaStreamSynchronize(h->stream));
        b0 = h->pinned[1];
        b1 = h->pinned[2];
    } else {
        // the full check of host offsets runs below, while the copies are in flight
        b0 = offsets[0];
        b1 = offsets[n_reads];
    }
    if (b1 < b0) return fail(KC_ERR_ARG, "read offsets decrease");
    if (b1 == b0) return KC_OK;
    if (!packed_reads || !n_mask) return fail(KC_ERR_ARG, "packed_reads or n_mask is null");
    choose_partitions(h, b1 - b0, n_reads);

    const uint64_t B = (b0 / 64) * 64;
    const uint64_t n_local = b1 - B;
    const uint64_t n_units = (n_local + 63) / 64;
    const uint64_t n_pwords_src = (n_local + 31) / 32;
    const uint64_t n_pwords = 2 * n_units + 2;
    const bool data_dev = is_device_ptr(packed_reads);
    const bool mask_dev = is_device_ptr(n_mask);

    Batch b;
    b.n_units = n_units;
    b.sample = sample;
    uint64_t *nm = nullptr, *bd = nullptr, *doff = nullptr;
    cudaStream_t st = h->stream;
    // Host inputs are copied on the copy stream (allocated there too), so the
    // copy overlaps kernels already queued on the handle's stream; device
    // inputs are copied on the handle's stream, after the work queued there.
    const bool any_host = !(data_dev && mask_dev && off_dev);
    cudaStream_t cs = any_host ? h->copy_stream : st;
    // Host reads of a large partitioned batch are copied in chunks, each
    // chunk's windows extracted as soon as it lands (ChunkedReads); the
    // offsets go first and are checked on the device before anything touches
    // the handle.
    const int n_chunks = (int)std::min<uint64_t>(kMaxChunks, n_units / kChunkUnits);
    const bool chunked = !data_dev && !mask_dev && n_chunks >= 2 && h->strategy != KC_STRATEGY_DIRECT &&
                         !h->cfg.batched_ingest && scatter_mode_of(h) == 4 && bucket_bytes(h, n_local) <= room_bytes(h);
    // The N mask and offsets serve this call's kernels only: device ones are
    // read where they are (in stream order), host ones copied.  The packed
    // words are always copied: the store is padded for the kernels' loads and
    // may outlive the call.
    const bool own_nm = chunked || !is_local_device_ptr(n_mask, h->device);
    const bool own_off = chunked || !is_local_device_ptr(offsets, h->device);
    cudaError_t e;
    if ((e = cudaMallocAsync(&b.pw, n_pwords * 8, cs)) != cudaSuccess ||
        (e = cudaMallocAsync(&b.vw, n_units * 8, cs)) != cudaSuccess ||
        (own_nm && (e = cudaMallocAsync(&nm, n_units * 8, cs)) != cudaSuccess) ||
        (e = cudaMallocAsync(&bd, n_units * 8, cs)) != cudaSuccess ||
        (own_off && (e = cudaMallocAsync(&doff, (n_reads + 1) * 8, cs)) != cudaSuccess)) {
        cudaFreeAsync(b.pw, cs);
        cudaFreeAsync(b.vw, cs);
        cudaFreeAsync(nm, cs);
        cudaFreeAsync(bd, cs);
        cudaFreeAsync(doff, cs);
        return cuda_fail(e, "cudaMallocAsync(read store)");
    }
    if (chunked) {
        s = add_reads_chunked(h, b, sample, packed_reads, offsets, n_mask, n_reads, b0, b1, n_chunks, nm, bd, doff);
        if (s != KC_OK) return s;
        h->batches.push_back(b);
        h->bases += b1 - b0;
        h->reads += n_reads;
        return KC_OK;
    }
    KC_CUDA(cudaMemcpyAsync(b.pw, packed_reads + B / 32, n_pwords_src * 8, cudaMemcpyDefault, cs));
    KC_CUDA(cudaMemsetAsync(b.pw + n_pwords_src, 0, (n_pwords - n_pwords_src) * 8, cs));
    if (own_nm) KC_CUDA(cudaMemcpyAsync(nm, n_mask + B / 64, n_units * 8, cudaMemcpyDefault, cs));
    if (own_off) KC_CUDA(cudaMemcpyAsync(doff, offsets, (n_reads + 1) * 8, cudaMemcpyDefault, cs));
    const uint64_t* nm_in = own_nm ? nm : n_mask + B / 64;
    const uint64_t* off_in = own_off ? doff : offsets;
    if (!off_dev) {
        bool decreasing = false;
        for (uint64_t r = 0; r < n_reads && !decreasing; ++r) decreasing = offsets[r + 1] < offsets[r];
        if (decreasing) {
            KC_CUDA(cudaStreamSynchronize(cs));
            for (void* q : {(void*)b.pw, (void*)b.vw, (void*)nm, (void*)bd, (void*)doff}) cudaFreeAsync(q, cs);
            return fail(KC_ERR_ARG, "read offsets decrease");
        }
    }
    if (any_host) {
        KC_CUDA(cudaEventRecord(h->ev_copy, cs));
        KC_CUDA(cudaStreamWaitEvent(st, h->ev_copy, 0));
    }
    cudaEvent_t t0 = phase_begin(h);
    KC_CUDA(cudaMemsetAsync(bd, 0, n_units * 8, st));
    kc::launch_mark_read_starts(off_in, n_reads, B, n_local, bd, h->ctr, st);
    kc::launch_build_valid(nm_in, bd, n_units, b0 - B, n_local, h->k, b.vw, h->ctr, h->grid, st);
    phase_end(h, kIngest, t0);
    t0 = phase_begin(h);
    if (h->strategy == KC_STRATEGY_DIRECT) {
        if (h->bloom2)
            kc::launch_prune(b.pw, b.vw, n_units, h->params(sample), h->bloom, h->bloom2, h->ctr, h->grid, st);
        else
            kc::launch_pass1(b.pw, b.vw, n_units, h->params(sample), h->bloom, h->table, h->ctr, h->grid, st);
        h->launches += 3;
    } else if (bucket_bytes(h, n_local) > room_bytes(h)) {
        // the window hashes would not fit the device budget: keep the packed
        // reads (about 3 bits per base), extracted again at kc_finalize one
        // hash range at a time
        b.deferred = true;
        ++h->deferred;
    } else if (h->cfg.batched_ingest) {
        b.pending = true;  // extracted and grouped at kc_finalize, with the batch's other jobs
        b.n_local = n_local;
    } else {
        s = bucket_batch(h, b, n_local, st, h->params(sample), false);
        if (s != KC_OK) {
            for (void* q : {(void*)nm, (void*)bd, (void*)doff, (void*)b.pw, (void*)b.vw}) cudaFreeAsync(q, st);
            if (any_host) cudaEventSynchronize(h->ev_copy);  // the caller's arrays are no longer read
            return s;
        }
        h->launches += 2;
    }
    phase_end(h, kPass1, t0);
    KC_LAUNCHED("ingest launches");
    cudaFreeAsync(nm, st);
    cudaFreeAsync(bd, st);
    cudaFreeAsync(doff, st);
    if (h->strategy != KC_STRATEGY_DIRECT && !b.deferred && !b.pending) {
        // the hashes replace the reads: nothing rescans them
        cudaFreeAsync(b.pw, st);
        cudaFreeAsync(b.vw, st);
        b.pw = b.vw = nullptr;
    }
    h->batches.push_back(b);
    h->bases += b1 - b0;
    h->reads += n_reads;
    if (any_host) KC_CUDA(cudaEventSynchronize(h->ev_copy));  // caller may reuse its arrays
    return KC_OK;
}

kc_status kc_finalize(kc_handle h) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (h->state == State::Finalized) return KC_OK;
    if (h->strategy != KC_STRATEGY_DIRECT) return finalize_partitioned(h);  // sets the state
    s = finalize_direct(h);
    if (s != KC_OK) return s;
    h->state = State::Finalized;
    return KC_OK;
}

kc_status kc_dump(kc_handle h, uint64_t* keys, uint32_t* counts, uint64_t capacity, uint64_t* n_out) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (h->state != State::Finalized) return fail(KC_ERR_STATE, "kc_dump before kc_finalize");
    if (n_out) *n_out = h->n_result;
    if (!keys) return KC_OK;
    if (capacity < h->n_result) return fail(KC_ERR_CAPACITY, "dump capacity smaller than the result");
    if (h->n_result == 0) return KC_OK;
    cudaStream_t st = h->stream;
    if (h->spilled && h->cfg.spill != 2) {
        // copy the runs back and sort them on the device when there is room
        s = resort_spilled(h);
        if (s != KC_OK && s != KC_ERR_OOM_DEVICE) return s;
    }
    if (h->spilled) {  // merge the host runs
        const bool dev_k = is_device_ptr(keys), dev_c = counts && is_device_ptr(counts);
        std::unique_ptr<uint64_t[]> mk;
        std::unique_ptr<uint32_t[]> mc;
        uint64_t* kout = keys;
        uint32_t* cout = counts;
        if (dev_k) {
            mk.reset(new (std::nothrow) uint64_t[h->n_result]);
            if (!mk) return fail(KC_ERR_OOM_HOST, "dump staging");
            kout = mk.get();
        }
        if (dev_c) {
            mc.reset(new (std::nothrow) uint32_t[h->n_result * (size_t)h->n_samples]);
            if (!mc) return fail(KC_ERR_OOM_HOST, "dump staging");
            cout = mc.get();
        }
        merge_runs(h->spill_dir, kout, cout, h->n_samples);
        if (dev_k) KC_CUDA(cudaMemcpyAsync(keys, kout, h->n_result * 8, cudaMemcpyHostToDevice, st));
        if (dev_c)
            KC_CUDA(cudaMemcpyAsync(counts, cout, h->n_result * 4 * (size_t)h->n_samples, cudaMemcpyHostToDevice, st));
        if (dev_k || dev_c) KC_CUDA(cudaStreamSynchronize(st));  // the staging buffers go out of scope
        return KC_OK;
    }
    // pinned host counts of one sample: narrowed straight into them by a
    // kernel on the copy stream (over the host link), while the keys' copy
    // runs on the handle's stream
    void* dc = nullptr;
    const bool counts_mapped = counts && h->n_samples == 1 && !is_device_ptr(counts) && host_mapped(counts, &dc);
    if (counts_mapped) {
        KC_CUDA(cudaEventRecord(h->ev_copy, st));
        KC_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_copy, 0));
        kc::launch_counts_narrow(h->res_vals, h->n_result, static_cast<uint32_t*>(dc), h->copy_stream);
        h->launches += 1;
    }
    KC_CUDA(cudaMemcpyAsync(keys, h->res_keys, h->n_result * 8, cudaMemcpyDefault, st));
    if (counts && !counts_mapped) {
        if (h->n_samples == 2) {
            KC_CUDA(cudaMemcpyAsync(counts, h->res_vals, h->n_result * 8, cudaMemcpyDefault, st));
        } else if (is_device_ptr(counts)) {  // narrowed straight into the caller's device buffer
            kc::launch_counts_narrow(h->res_vals, h->n_result, counts, st);
            h->launches += 1;
        } else {
            uint32_t* narrow = nullptr;
            KC_CUDA(cudaMallocAsync(&narrow, h->n_result * 4, st));
            kc::launch_counts_narrow(h->res_vals, h->n_result, narrow, st);
            h->launches += 1;
            KC_CUDA(cudaMemcpyAsync(counts, narrow, h->n_result * 4, cudaMemcpyDefault, st));
            cudaFreeAsync(narrow, st);
        }
    }
    KC_LAUNCHED("dump launches");
    KC_CUDA(cudaStreamSynchronize(st));
    if (counts_mapped) KC_CUDA(cudaStreamSynchronize(h->copy_stream));
    return KC_OK;
}

kc_status kc_export_bloom(kc_handle h, uint64_t* words, uint64_t first_word, uint64_t n_words) {
    if (!h) return fail(KC_ERR_ARG, "null handle");
    const uint64_t nw = h->bloom_bits / 64;
    if (!words || first_word > nw || n_words > nw - first_word) return fail(KC_ERR_ARG, "filter range");
    KC_CUDA(cudaMemcpyAsync(words, h->bloom + first_word, n_words * 8, cudaMemcpyDefault, h->stream));
    KC_CUDA(cudaStreamSynchronize(h->stream));
    return KC_OK;
}

kc_status kc_export_bloom2(kc_handle h, uint64_t* words, uint64_t first_word, uint64_t n_words) {
    if (!h) return fail(KC_ERR_ARG, "null handle");
    if (!h->bloom2) return fail(KC_ERR_STATE, "no second filter: the handle was not created with prune_chain = 1");
    const uint64_t nw = h->bloom_bits / 64;
    if (!words || first_word > nw || n_words > nw - first_word) return fail(KC_ERR_ARG, "filter range");
    KC_CUDA(cudaMemcpyAsync(words, h->bloom2 + first_word, n_words * 8, cudaMemcpyDefault, h->stream));
    KC_CUDA(cudaStreamSynchronize(h->stream));
    return KC_OK;
}

kc_status kc_stats_get(kc_handle h, kc_stats* out) {
    if (!h || !out) return fail(KC_ERR_ARG, "null argument");
    kc_status s = read_counters(h);
    if (s != KC_OK) return s;
    phase_collect(h);
    std::memset(out, 0, sizeof(*out));
    out->windows = h->host_ctr.windows;
    out->bases = h->bases;
    out->candidates = h->host_ctr.candidates;
    out->table_keys = h->host_ctr.claimed;
    out->result_keys = h->state == State::Finalized ? h->n_result : 0;
    out->partitions = h->strategy == KC_STRATEGY_DIRECT ? 1u : (1u << h->part_bits);
    out->table_log2 = (uint32_t)h->log2_slots;
    out->fallback_partitions = h->fallback_partitions;
    out->split_partitions = h->host_ctr.split_parts;
    out->split_level = h->host_ctr.split_hint;
    out->spilled_bytes = h->spilled_bytes;
    out->strategy = (uint32_t)h->strategy;
    out->owned_windows = h->owner ? h->host_ctr.kept : h->host_ctr.windows;
    out->deferred_batches = h->deferred;
    out->scan_groups = h->scan_groups;
    size_t bytes = h->fixed_bytes + h->res_cap * 16;
    if (h->has_stems) bytes += std::max<uint64_t>(1, h->n_stems) * sizeof(kc_stem_item);
    if (h->has_selection) bytes += std::max<uint64_t>(1, h->n_sel) * 16 + (48ull << h->sel_buckets_log2) + (h->sel_pre ? 4ull * 49152 : 0);
    for (const auto& b : h->batches) {
        if (b.pw) bytes += (2 * b.n_units + 2) * 8 + b.n_units * 8;
        if (b.hdata) bytes += b.hcap * 8 + ((1ull << h->part_bits) + 1) * 8;
    }
    out->device_bytes = bytes;
    out->launches = h->launches;
    out->ms_ingest = h->ms[kIngest];
    out->ms_pass1 = h->ms[kPass1];
    out->ms_pass2 = h->ms[kPass2];
    out->ms_compact = h->ms[kCompact];
    out->ms_sort = h->ms[kSort];
    out->ms_filter_select = h->ms[kFilterSelect];
    out->ms_filter_reads = h->ms[kFilterReads];
    out->filter_selected = h->has_selection ? h->n_sel : 0;
    out->filter_windows = h->filter_windows;
    out->filter_hits = h->filter_hits;
    out->ms_stems = h->ms[kStems];
    out->stem_items = h->has_stems ? h->n_stems : 0;
    return KC_OK;
}

}  // extern "C"

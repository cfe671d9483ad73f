// Continuous-batching job server over the C ABI (kc_server_* in include/kc.h).
//
// Three kinds of host threads drive the GPU:
//   ingest    takes queued jobs in arrival order, admits the next one as soon as
//             its estimated device footprint fits the budget (memory frees up
//             as jobs finish), creates its handle on its own stream and copies
//             its reads to the device (kc_config.batched_ingest: nothing is
//             extracted yet);
//   extract   takes every job copied so far (at most max_batch) and extracts
//             and groups all their reads together (kc_batch_ingest: one
//             persistent launch per phase over a queue of (read batch, unit
//             range) items), without waiting for the device;
//   finalize  takes every job ingested so far (at most max_batch), finalizes
//             them together with one kc_batch_finalize (one persistent
//             consumer launch over all their partitions and one replay of the
//             sort graph), copies each result to host memory, frees the job's
//             device memory and wakes its waiters.
// Jobs that arrive while a batch runs are ingested at once on their own
// streams, so their work overlaps the batch on the device, and they join the
// next batch: a batch never waits for stragglers and a job never waits for a
// whole batch to drain before it starts.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kc.h"
#include "kc_ctx.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kIngestThreads = 2;
constexpr int kFinalizeThreads = 2;
constexpr int kExtractThreads = 2;

struct Job {
    uint64_t id = 0;
    kc_job_spec spec{};
    uint64_t footprint = 0;
    kc_handle h = nullptr;
    Clock::time_point t_submit, t_admit, t_ingested, t_fstart, t_done;
    kc_status status = KC_OK;
    std::string error;
    bool done = false;
    // the result in host memory: pinned pool blocks (class >= 0) or, past the
    // pool's cap, ordinary host memory (class -1)
    uint64_t* keys = nullptr;
    uint32_t* counts = nullptr;
    int keys_class = -1, counts_class = -1;
    uint64_t n_keys = 0;
};

// Pinned host blocks for results, in power-of-two size classes, reused across
// jobs and across servers (one pool per process, kept until it exits): the
// device-to-host copy of a result runs at full speed on the finalize thread,
// and the copy into the caller's memory happens later in kc_server_result, on
// the caller's thread.
struct PinnedPool {
    std::mutex mu;
    std::map<int, std::vector<void*>> free_blocks;
    uint64_t held = 0;
    uint64_t cap = 8ull << 30;
    static int size_class(uint64_t bytes) {
        int c = 20;  // 1 MiB at least
        while (c < 63 && (1ull << c) < bytes) ++c;
        return c;
    }
    // A block of at least `bytes`; *cls = its class, or -1 (ordinary memory)
    void* get(uint64_t bytes, int* cls) {
        const int c = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = free_blocks.find(c);
            if (it != free_blocks.end() && !it->second.empty()) {
                void* p = it->second.back();
                it->second.pop_back();
                *cls = c;
                return p;
            }
            if (held + (1ull << c) <= cap) {
                void* p = nullptr;
                std::lock_guard<std::mutex> sync_lk(kc::sync_api_mutex());
                if (cudaMallocHost(&p, 1ull << c) == cudaSuccess) {
                    held += 1ull << c;
                    *cls = c;
                    return p;
                }
                cudaGetLastError();
            }
        }
        *cls = -1;
        return ::operator new(bytes, std::nothrow);
    }
    void put(void* p, int cls) {
        if (!p) return;
        if (cls < 0) {
            ::operator delete(p);
            return;
        }
        std::lock_guard<std::mutex> lk(mu);
        free_blocks[cls].push_back(p);
    }
};

PinnedPool& result_pool() {
    static PinnedPool* pool = new PinnedPool();  // never destroyed: the CUDA context may be gone at exit
    return *pool;
}

void free_result(PinnedPool& pool, Job& j) {
    pool.put(j.keys, j.keys_class);
    pool.put(j.counts, j.counts_class);
    j.keys = nullptr;
    j.counts = nullptr;
}

}  // namespace

struct kc_server_ctx {
    uint64_t budget = 0;
    int max_batch = 64;
    uint32_t flags = 0;
    std::mutex mu;
    std::condition_variable cv_ingest, cv_extract, cv_final, cv_done;
    std::deque<std::shared_ptr<Job>> pending;   // submitted, not admitted
    std::deque<std::shared_ptr<Job>> copied;    // admitted, reads on the device, not extracted
    std::deque<std::shared_ptr<Job>> ingested;  // admitted and ingested (extracted and grouped)
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_id = 1, in_use = 0, peak = 0;
    bool stop = false;
    // two ingest threads (pageable host copies run in parallel) and two
    // finalize threads, each with its own batch object, so one batch's
    // copy-out overlaps the next batch's kernels
    std::vector<std::thread> t_ingest, t_final;
    std::vector<std::thread> t_extract;
    std::vector<kc_batch> extract_batch;
    std::vector<kc_batch> batch;
    int device = 0;
    // Handles of finished jobs, reset and kept for the next job with the same
    // parameters (oldest first): creating and destroying a handle per job
    // costs a stream, events and the filter's allocation.  Their device bytes
    // count against the budget and the oldest are destroyed to make room.
    struct IdleHandle {
        kc_handle h;
        int k, n_samples, n_hashes;
        uint32_t min_count;
        uint64_t bloom_bits;
        kc_config cfg;
        uint64_t bytes;
    };
    std::deque<IdleHandle> idle;
    uint64_t idle_bytes = 0, reused = 0;
    static constexpr size_t kMaxIdle = 32;
    // finished jobs' handles to reset and keep, and handles to destroy, both
    // taken by a reaper thread so that neither ingest nor finalize waits for
    // a handle's reset or teardown
    struct Parked {
        kc_handle h;
        kc_job_spec spec;
    };
    std::vector<Parked> to_park;
    std::vector<kc_handle> graveyard;
    std::condition_variable cv_reap;
    std::thread t_reap;
    PinnedPool& pool = result_pool();
    // statistics
    std::vector<double> latencies_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_jobs = 0;
    double sum_stage_ms[4] = {};  // queue, ingest, batch wait, finalize + copy-out of completed jobs
    double sum_fin_ms[3] = {};    // per batch: batched finalize, copies to host memory, handle release
    double sum_ingest_ms[2] = {}; // per job: getting a handle, adding its reads
    Clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

// Device bytes a job may hold at its peak (upper bounds): filter; per base the
// packed reads, N mask, read-start and valid bits, the linear and the
// partitioned hash of a window, survivors and result (16 bytes each) and the
// offsets.
uint64_t footprint(const kc_job_spec& s) {
    uint64_t bases = 0, reads = 0;
    for (int i = 0; i < s.n_samples; ++i) {
        if (s.n_reads[i]) bases += s.offsets[i][s.n_reads[i]] - s.offsets[i][0];
        reads += s.n_reads[i];
    }
    return s.bloom_bits / 8 + bases * 50 + reads * 8 + (8ull << 20);
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

void fail_job(kc_server_ctx* S, const std::shared_ptr<Job>& j, kc_status st) {
    j->status = st;
    j->error = kc_last_error();
    if (j->h) kc_destroy(j->h);
    j->h = nullptr;
    j->t_done = Clock::now();
    j->done = true;
    S->in_use -= j->footprint;
    S->failed += 1;
}

// Destroy idle handles, oldest first, while the admitted jobs and the idle
// handles together pass the budget (call with S->mu held; the handles are
// destroyed by the caller, outside the lock).
void evict_idle(kc_server_ctx* S, std::vector<kc_handle>& out) {
    while (!S->idle.empty() && S->in_use + S->idle_bytes > S->budget) {
        out.push_back(S->idle.front().h);
        S->idle_bytes -= S->idle.front().bytes;
        S->idle.pop_front();
    }
}

// Same knobs (the device budget is per job and is set on reuse).
bool same_config(kc_config a, kc_config b) {
    a.device_budget = b.device_budget = 0;
    return std::memcmp(&a, &b, sizeof(a)) == 0;
}

void ingest_loop(kc_server_ctx* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::shared_ptr<Job> j;
        std::vector<kc_handle> evicted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_ingest.wait(lk, [&] {
                return S->stop || (!S->pending.empty() &&
                                   (S->in_use + S->pending.front()->footprint <= S->budget || S->in_use == 0));
            });
            if (S->stop) return;
            j = S->pending.front();
            S->pending.pop_front();
            S->in_use += j->footprint;  // admitted
            S->peak = std::max(S->peak, S->in_use);
            evict_idle(S, evicted);
            if (!evicted.empty()) {
                S->graveyard.insert(S->graveyard.end(), evicted.begin(), evicted.end());
                S->cv_reap.notify_one();
            }
        }
        j->t_admit = Clock::now();
        const kc_job_spec& s = j->spec;
        kc_config cfg;
        kc_default_config(&cfg);
        if (S->flags & KC_SERVER_TUNED) {
            uint64_t bases = 0;
            for (int i = 0; i < s.n_samples; ++i)
                if (s.n_reads[i]) bases += s.offsets[i][s.n_reads[i]] - s.offsets[i][0];
            kc_config tuned;
            int found = 0;
            if (kc_tune_lookup(s.k, s.n_samples, s.bloom_bits, s.n_hashes, s.min_count, bases, &tuned, &found) == KC_OK &&
                found && tuned.strategy == KC_STRATEGY_PARTITIONED)
                cfg = tuned;  // batched finalize needs the partitioned strategy
        }
        cfg.strategy = KC_STRATEGY_PARTITIONED;
        // the job was admitted for its footprint: that is the device memory it
        // may hold (not the device's free memory, which other jobs and
        // processes share)
        cfg.device_budget = j->footprint;
        // reads only at ingest; a batch's jobs are extracted and grouped together
        // at its finalize, by one launch per phase
        cfg.batched_ingest = 1;
        {  // a finished job's handle with the same parameters, already reset
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto it = S->idle.begin(); it != S->idle.end(); ++it)
                if (it->k == s.k && it->n_samples == s.n_samples && it->n_hashes == s.n_hashes &&
                    it->min_count == s.min_count && it->bloom_bits == s.bloom_bits && same_config(it->cfg, cfg)) {
                    j->h = it->h;
                    j->h->cfg.device_budget = cfg.device_budget;
                    S->idle_bytes -= it->bytes;
                    S->idle.erase(it);
                    S->reused += 1;
                    break;
                }
        }
        kc_status st = j->h ? KC_OK
                            : kc_create_ex(s.k, s.n_samples, s.bloom_bits, s.n_hashes, s.min_count, &cfg, nullptr, &j->h);
        const Clock::time_point t_handle = Clock::now();
        for (int i = 0; st == KC_OK && i < s.n_samples; ++i)
            st = kc_add_reads(j->h, i, s.packed[i], s.offsets[i], s.n_mask[i], s.n_reads[i]);
        const Clock::time_point t_added = Clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        S->sum_ingest_ms[0] += ms_between(j->t_admit, t_handle);
        S->sum_ingest_ms[1] += ms_between(t_handle, t_added);
        if (st != KC_OK) {
            fail_job(S, j, st);
            S->cv_done.notify_all();
            S->cv_ingest.notify_all();
            continue;
        }
        S->copied.push_back(j);
        S->cv_extract.notify_all();
    }
}

void extract_loop(kc_server_ctx* S, int idx) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<std::shared_ptr<Job>> run;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_extract.wait(lk, [&] { return S->stop || !S->copied.empty(); });
            if (S->stop) return;
            while (!S->copied.empty() && (int)run.size() < S->max_batch) {
                run.push_back(S->copied.front());
                S->copied.pop_front();
            }
        }
        std::vector<kc_handle> hs;
        for (auto& j : run) hs.push_back(j->h);
        const kc_status st = kc_batch_ingest(S->extract_batch[idx], hs.data(), (int)hs.size());
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto& j : run) {
            if (st != KC_OK) {
                fail_job(S, j, st);
                continue;
            }
            j->t_ingested = Clock::now();
            S->ingested.push_back(j);
        }
        S->cv_final.notify_all();
        if (st != KC_OK) {
            S->cv_done.notify_all();
            S->cv_ingest.notify_all();
        }
    }
}

void finalize_loop(kc_server_ctx* S, int idx) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<std::shared_ptr<Job>> run;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_final.wait(lk, [&] { return S->stop || !S->ingested.empty(); });
            if (S->stop) return;
            while (!S->ingested.empty() && (int)run.size() < S->max_batch) {
                run.push_back(S->ingested.front());
                S->ingested.pop_front();
            }
        }
        std::vector<kc_handle> hs;
        const Clock::time_point t_start = Clock::now();
        for (auto& j : run) {
            hs.push_back(j->h);
            j->t_fstart = t_start;
        }
        kc_status st = kc_batch_finalize(S->batch[idx], hs.data(), (int)hs.size());
        const Clock::time_point t_fin = Clock::now();
        double copy_ms = 0.0, release_ms = 0.0;
        for (auto& j : run) {
            kc_status js = st;
            uint64_t n = 0;
            const Clock::time_point t_c0 = Clock::now();
            if (js == KC_OK) js = kc_dump(j->h, nullptr, nullptr, 0, &n);
            if (js == KC_OK) {
                j->keys = static_cast<uint64_t*>(S->pool.get(std::max<uint64_t>(1, n) * 8, &j->keys_class));
                j->counts = static_cast<uint32_t*>(
                    S->pool.get(std::max<uint64_t>(1, n * (size_t)j->spec.n_samples) * 4, &j->counts_class));
                if (!j->keys || !j->counts) js = KC_ERR_OOM_HOST;
                else if (n) js = kc_dump(j->h, j->keys, j->counts, n, &n);
                j->n_keys = n;
            }
            const Clock::time_point t_c1 = Clock::now();
            copy_ms += ms_between(t_c0, t_c1);
            if (js == KC_OK) {
                // to the reaper: reset (its grouped hashes and batches freed)
                // and kept for a later job with the same parameters
                std::lock_guard<std::mutex> lk(S->mu);
                S->to_park.push_back({j->h, j->spec});
                S->cv_reap.notify_one();
                j->h = nullptr;
            } else {
                free_result(S->pool, *j);
            }
            release_ms += ms_between(t_c1, Clock::now());
            std::lock_guard<std::mutex> lk(S->mu);
            if (js != KC_OK) {
                fail_job(S, j, js);
                continue;
            }
            j->t_done = Clock::now();
            j->done = true;
            S->in_use -= j->footprint;
            S->completed += 1;
            S->latencies_ms.push_back(ms_between(j->t_submit, j->t_done));
            S->sum_stage_ms[0] += ms_between(j->t_submit, j->t_admit);
            S->sum_stage_ms[1] += ms_between(j->t_admit, j->t_ingested);
            S->sum_stage_ms[2] += ms_between(j->t_ingested, j->t_fstart);
            S->sum_stage_ms[3] += ms_between(j->t_fstart, j->t_done);
            S->t_last = j->t_done;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->batches += 1;
            S->batched_jobs += run.size();
            S->sum_fin_ms[0] += ms_between(t_start, t_fin);
            S->sum_fin_ms[1] += copy_ms;
            S->sum_fin_ms[2] += release_ms;
        }
        S->cv_done.notify_all();
        S->cv_ingest.notify_all();
    }
}

void reap_loop(kc_server_ctx* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<kc_handle> dead;
        std::vector<kc_server_ctx::Parked> park;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_reap.wait(lk, [&] { return S->stop || !S->graveyard.empty() || !S->to_park.empty(); });
            dead.swap(S->graveyard);
            park.swap(S->to_park);
            if (dead.empty() && park.empty() && S->stop) return;
        }
        for (auto& p : park) {
            if (S->stop || kc_reset(p.h) != KC_OK) {
                dead.push_back(p.h);
                continue;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->idle.size() >= kc_server_ctx::kMaxIdle) {
                dead.push_back(S->idle.front().h);
                S->idle_bytes -= S->idle.front().bytes;
                S->idle.pop_front();
            }
            kc_server_ctx::IdleHandle ih{p.h, p.spec.k, p.spec.n_samples, p.spec.n_hashes, p.spec.min_count,
                                         p.spec.bloom_bits, p.h->cfg, kcapi::held_bytes(p.h)};
            S->idle.push_back(ih);
            S->idle_bytes += ih.bytes;
        }
        for (kc_handle h : dead) kc_destroy(h);
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

kc_status kc_server_create(uint64_t device_budget_bytes, int max_batch, kc_server* out) {
    return kc_server_create_ex(device_budget_bytes, max_batch, 0, out);
}

kc_status kc_server_create_ex(uint64_t device_budget_bytes, int max_batch, uint32_t flags, kc_server* out) {
    if (!out || device_budget_bytes == 0 || max_batch < 1 || (flags & ~KC_SERVER_TUNED)) return KC_ERR_ARG;
    *out = nullptr;
    kc_server_ctx* S = new (std::nothrow) kc_server_ctx();
    if (!S) return KC_ERR_OOM_HOST;
    S->budget = device_budget_bytes;
    S->max_batch = max_batch;
    S->flags = flags;
    cudaGetDevice(&S->device);
    kc_status st = KC_OK;
    for (int i = 0; st == KC_OK && i < kFinalizeThreads; ++i) {
        kc_batch b = nullptr;
        st = kc_batch_create(nullptr, &b);
        if (st == KC_OK) S->batch.push_back(b);
    }
    for (int i = 0; st == KC_OK && i < kExtractThreads; ++i) {
        kc_batch b = nullptr;
        st = kc_batch_create(nullptr, &b);
        if (st == KC_OK) S->extract_batch.push_back(b);
    }
    if (st != KC_OK) {
        for (kc_batch b : S->batch) kc_batch_destroy(b);
        for (kc_batch b : S->extract_batch) kc_batch_destroy(b);
        delete S;
        return st;
    }
    for (int i = 0; i < kIngestThreads; ++i) S->t_ingest.emplace_back(ingest_loop, S);
    for (int i = 0; i < kExtractThreads; ++i) S->t_extract.emplace_back(extract_loop, S, i);
    for (int i = 0; i < kFinalizeThreads; ++i) S->t_final.emplace_back(finalize_loop, S, i);
    S->t_reap = std::thread(reap_loop, S);
    *out = S;
    return KC_OK;
}

static bool host_memory(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice;
}

kc_status kc_server_submit(kc_server S, const kc_job_spec* spec, uint64_t* job_id) {
    const auto bad = [](const char* msg) {
        kc::set_last_error(msg);
        return KC_ERR_ARG;
    };
    if (!S || !spec || !job_id) return bad("kc_server_submit: null argument");
    if (spec->n_samples < 1 || spec->n_samples > 2) return bad("n_samples must be 1 or 2");
    for (int i = 0; i < spec->n_samples; ++i) {
        if (spec->n_reads[i] && !spec->offsets[i]) return bad("a sample with reads has no offsets");
        if (!host_memory(spec->offsets[i]) || !host_memory(spec->packed[i]) || !host_memory(spec->n_mask[i]))
            return bad("server jobs take host arrays");
    }
    auto j = std::make_shared<Job>();
    j->spec = *spec;
    j->footprint = footprint(*spec);
    j->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->any) {
        S->t_first = j->t_submit;
        S->any = true;
    }
    j->id = S->next_id++;
    S->jobs[j->id] = j;
    S->pending.push_back(j);
    S->submitted += 1;
    *job_id = j->id;
    S->cv_ingest.notify_all();
    return KC_OK;
}

kc_status kc_server_wait(kc_server S, uint64_t job_id, double timeout_s, uint64_t* n_keys, double* latency_ms) {
    if (!S) return KC_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return KC_ERR_ARG;
    std::shared_ptr<Job> j = it->second;
    const auto pred = [&] { return j->done; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, pred);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return KC_ERR_TIMEOUT;
    }
    if (j->status != KC_OK) kc::set_last_error(j->error);  // the job's own message, for this thread
    if (n_keys) *n_keys = j->n_keys;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    return j->status;
}

kc_status kc_server_result(kc_server S, uint64_t job_id, uint64_t* keys, uint32_t* counts, uint64_t capacity,
                           uint64_t* n_out) {
    if (!S) return KC_ERR_ARG;
    std::shared_ptr<Job> j;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->jobs.find(job_id);
        if (it == S->jobs.end()) return KC_ERR_ARG;
        j = it->second;
        if (!j->done) return KC_ERR_STATE;
        if (j->status != KC_OK) return j->status;
        if (n_out) *n_out = j->n_keys;
        if (!keys) return KC_OK;
        if (capacity < j->n_keys) return KC_ERR_CAPACITY;
        S->jobs.erase(it);  // the result is handed over: no other call sees the job now
    }
    // the copy into the caller's memory runs outside the server's lock
    std::memcpy(keys, j->keys, j->n_keys * 8);
    if (counts) std::memcpy(counts, j->counts, j->n_keys * (size_t)j->spec.n_samples * 4);
    free_result(S->pool, *j);
    return KC_OK;
}

kc_status kc_server_stats_get(kc_server S, kc_server_stats* out) {
    if (!S || !out) return KC_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->batched_jobs / (double)S->batches : 0.0;
    out->p50_ms = percentile(S->latencies_ms, 0.50);
    out->p99_ms = percentile(S->latencies_ms, 0.99);
    double sum = 0;
    for (double x : S->latencies_ms) sum += x;
    out->mean_ms = S->latencies_ms.empty() ? 0.0 : sum / (double)S->latencies_ms.size();
    const double span = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    out->jobs_per_s = span > 0 ? (double)S->completed / span : 0.0;
    out->peak_bytes = S->peak;
    out->budget_bytes = S->budget;
    const double nc = S->completed ? (double)S->completed : 1.0;
    out->mean_queue_ms = S->sum_stage_ms[0] / nc;
    out->mean_ingest_ms = S->sum_stage_ms[1] / nc;
    out->mean_batch_wait_ms = S->sum_stage_ms[2] / nc;
    out->mean_finalize_ms = S->sum_stage_ms[3] / nc;
    const double nbat = S->batches ? (double)S->batches : 1.0;
    out->mean_batch_finalize_ms = S->sum_fin_ms[0] / nbat;
    out->mean_batch_copy_ms = S->sum_fin_ms[1] / nbat;
    out->mean_batch_release_ms = S->sum_fin_ms[2] / nbat;
    out->reused_handles = S->reused;
    const double ns = S->submitted ? (double)(S->completed + S->failed) : 1.0;
    out->mean_ingest_handle_ms = S->sum_ingest_ms[0] / (ns > 0 ? ns : 1.0);
    out->mean_ingest_add_ms = S->sum_ingest_ms[1] / (ns > 0 ? ns : 1.0);
    return KC_OK;
}

void kc_server_destroy(kc_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_ingest.notify_all();
    S->cv_extract.notify_all();
    S->cv_final.notify_all();
    S->cv_reap.notify_all();
    for (auto& t : S->t_ingest) t.join();
    for (auto& t : S->t_extract) t.join();
    for (auto& t : S->t_final) t.join();
    if (S->t_reap.joinable()) S->t_reap.join();
    for (kc_handle h : S->graveyard) kc_destroy(h);
    for (auto& p : S->to_park) kc_destroy(p.h);
    for (auto& d : S->copied)
        if (d->h) kc_destroy(d->h);
    for (auto& d : S->ingested)
        if (d->h) kc_destroy(d->h);
    for (auto& ih : S->idle) kc_destroy(ih.h);
    for (auto& kv : S->jobs) free_result(S->pool, *kv.second);  // results never collected
    for (kc_batch b : S->batch) kc_batch_destroy(b);
    for (kc_batch b : S->extract_batch) kc_batch_destroy(b);
    delete S;
}

}  // extern "C"

// Autotuner: runs one counting job under candidate configurations on the
// caller's reads, keeps the fastest, and remembers it per job class in a
// process-wide cache that can be saved to and loaded from a text file.
//
// The paper fixes its work-unit sizes by hand and warns that they must be
// chosen with care (Section III-B); the knobs that play that role here are
// the partition bits (how much of the filter and how many windows one
// consumer CTA takes), the shared-memory table size, the reads per
// extraction CTA (CTAs per SM) and, for the direct strategy, the grid size.
// Everything is timed with CUDA events on the tuner's own stream through the
// public entry points, exactly as a caller would run the job.

#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/kc.h"
#include "kc_internal.h"

namespace {

struct ClassKey {
    int k, n_samples;
    uint64_t bloom_bits;
    int n_hashes, min_gt1, bases_log2, sms;
    bool operator<(const ClassKey& o) const {
        return std::tie(k, n_samples, bloom_bits, n_hashes, min_gt1, bases_log2, sms) <
               std::tie(o.k, o.n_samples, o.bloom_bits, o.n_hashes, o.min_gt1, o.bases_log2, o.sms);
    }
};

struct Entry {
    kc_config cfg;
    double ms;
};

std::mutex g_mu;
std::map<ClassKey, Entry> g_cache;

kc_status tune_fail(kc_status s, const std::string& msg) {
    kc::set_last_error(msg);
    return s;
}

int log2_ceil(uint64_t x) {
    int r = 0;
    while (r < 63 && (1ull << r) < x) ++r;
    return r;
}

kc_status device_sms(int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return tune_fail(KC_ERR_CUDA, "no CUDA device");
    }
    return KC_OK;
}

ClassKey class_of(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count, uint64_t n_bases,
                  int sms) {
    return ClassKey{k, n_samples, bloom_bits, n_hashes, min_count > 1 ? 1 : 0, log2_ceil(std::max<uint64_t>(1, n_bases)),
                    sms};
}

// Bases of a read batch, from its offsets (host or device).
kc_status batch_bases(const kc_tune_input& in, uint64_t* out) {
    *out = 0;
    if (!in.n_reads) return KC_OK;
    if (!in.offsets) return tune_fail(KC_ERR_ARG, "tuning input without offsets");
    uint64_t ends[2];
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    if (cudaMemcpy(&ends[0], in.offsets, 8, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(&ends[1], in.offsets + in.n_reads, 8, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return tune_fail(KC_ERR_ARG, "tuning input offsets are not readable");
    }
    *out = ends[1] >= ends[0] ? ends[1] - ends[0] : 0;
    return KC_OK;
}

// One timed run of the job under cfg: ms from before the first kc_add_reads
// to after kc_finalize, on stream st.
kc_status run_once(const kc_config& cfg, int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                   const kc_tune_input* inputs, int n_inputs, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                   float* ms) {
    kc_handle h = nullptr;
    kc_status s = kc_create_ex(k, n_samples, bloom_bits, n_hashes, min_count, &cfg, st, &h);
    if (s != KC_OK) return s;
    cudaEventRecord(e0, st);
    for (int i = 0; s == KC_OK && i < n_inputs; ++i)
        s = kc_add_reads(h, inputs[i].sample, inputs[i].packed_reads, inputs[i].offsets, inputs[i].n_mask,
                         inputs[i].n_reads);
    if (s == KC_OK) s = kc_finalize(h);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (s == KC_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    kc_destroy(h);
    if (s == KC_OK && e != cudaSuccess) s = tune_fail(KC_ERR_CUDA, std::string("tuning timer: ") + cudaGetErrorString(e));
    return s;
}

// Median over reps runs after one warm-up run; < 0 if the configuration fails.
double time_config(const kc_config& cfg, int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                   const kc_tune_input* inputs, int n_inputs, int reps, cudaStream_t st, cudaEvent_t e0,
                   cudaEvent_t e1, kc_status* hard) {
    std::vector<float> t;
    for (int r = 0; r <= reps; ++r) {
        float ms = 0.f;
        const kc_status s = run_once(cfg, k, n_samples, bloom_bits, n_hashes, min_count, inputs, n_inputs, st, e0, e1, &ms);
        if (s == KC_ERR_ARG || s == KC_ERR_CAPACITY || s == KC_ERR_OOM_DEVICE) return -1.0;  // not a candidate here
        if (s != KC_OK) {
            *hard = s;
            return -1.0;
        }
        if (r > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" {

kc_status kc_autotune(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                      const kc_tune_input* inputs, int n_inputs, int reps, kc_config* best, kc_tune_trial* trials,
                      int max_trials, int* n_trials) {
    kc::set_last_error("");
    if (n_trials) *n_trials = 0;
    if (!best || n_inputs < 0 || (n_inputs > 0 && !inputs) || reps < 1 || reps > 100 || (trials && max_trials < 0))
        return tune_fail(KC_ERR_ARG, "kc_autotune: bad arguments");
    if (bloom_bits < 4096 || (bloom_bits & (bloom_bits - 1)))
        return tune_fail(KC_ERR_ARG, "bloom_bits must be a power of two >= 4096");
    int sms = 0;
    kc_status s = device_sms(&sms);
    if (s != KC_OK) return s;
    uint64_t bases = 0;
    for (int i = 0; i < n_inputs; ++i) {
        uint64_t b = 0;
        if ((s = batch_bases(inputs[i], &b)) != KC_OK) return s;
        bases += b;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        if (st) cudaStreamDestroy(st);
        return tune_fail(KC_ERR_CUDA, "kc_autotune: stream or event creation");
    }
    kc_status hard = KC_OK;
    int written = 0;
    kc_config best_cfg{};
    double best_ms = -1.0;
    auto trial = [&](const kc_config& c) -> double {
        if (hard != KC_OK) return -1.0;
        const double ms = time_config(c, k, n_samples, bloom_bits, n_hashes, min_count, inputs, n_inputs, reps, st, e0,
                                      e1, &hard);
        if (trials && written < max_trials) trials[written++] = kc_tune_trial{c, ms};
        if (ms >= 0 && (best_ms < 0 || ms < best_ms)) {
            best_ms = ms;
            best_cfg = c;
        }
        return ms;
    };
    kc_config base;
    kc_default_config(&base);
    int lw = 0;
    while ((1ull << lw) < bloom_bits / 64) ++lw;

    // partitioned: partition bits for filter slices of 2^13 .. 2^8 words
    base.strategy = KC_STRATEGY_PARTITIONED;
    int best_pb = -1;
    double pb_ms = -1.0;
    for (int slice = 13; slice >= 8; --slice) {
        const int pb = lw - slice;
        if (pb < 1 || pb > 20) continue;
        kc_config c = base;
        c.part_bits = (uint32_t)pb;
        const double ms = trial(c);
        if (ms >= 0 && (pb_ms < 0 || ms < pb_ms)) {
            pb_ms = ms;
            best_pb = pb;
        }
    }
    if (best_pb > 0) {
        // table size, then reads per extraction CTA, at the best partition bits
        kc_config c = base;
        c.part_bits = (uint32_t)best_pb;
        uint32_t best_tl = 0;
        double tl_ms = pb_ms;
        for (uint32_t tl = 10; tl <= 13; ++tl) {
            c.smem_table_log2 = tl;
            const double ms = trial(c);
            if (ms >= 0 && ms < tl_ms) {
                tl_ms = ms;
                best_tl = tl;
            }
        }
        c.smem_table_log2 = best_tl;
        for (uint32_t cps = 2; cps <= 3; ++cps) {
            c.ctas_per_sm = cps;
            trial(c);
        }
    }
    // direct: grid CTAs per SM
    for (uint32_t cps : {4u, 8u, 16u}) {
        kc_config c = base;
        c.strategy = KC_STRATEGY_DIRECT;
        c.part_bits = 0;
        c.ctas_per_sm = cps;
        trial(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (n_trials) *n_trials = written;
    if (hard != KC_OK) return hard;
    if (best_ms < 0) return tune_fail(KC_ERR_ARG, "kc_autotune: no configuration could run this job");
    *best = best_cfg;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[class_of(k, n_samples, bloom_bits, n_hashes, min_count, bases, sms)] = Entry{best_cfg, best_ms};
    return KC_OK;
}

kc_status kc_tune_lookup(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count, uint64_t n_bases,
                         kc_config* out, int* found) {
    if (!out || !found) return tune_fail(KC_ERR_ARG, "kc_tune_lookup: null argument");
    *found = 0;
    int sms = 0;
    kc_status s = device_sms(&sms);
    if (s != KC_OK) return s;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(class_of(k, n_samples, bloom_bits, n_hashes, min_count, n_bases, sms));
    if (it == g_cache.end()) return KC_OK;
    *out = it->second.cfg;
    *found = 1;
    return KC_OK;
}

// File format: a header line, then one line per class:
//   k n_samples bloom_bits n_hashes min_gt1 bases_log2 sms
//   strategy part_bits smem_table_log2 ctas_per_sm scatter_mode split_max ms
kc_status kc_tune_cache_save(const char* path) {
    if (!path) return tune_fail(KC_ERR_ARG, "kc_tune_cache_save: null path");
    std::ostringstream os;
    os << "kc-tune-cache 1\n";
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const auto& kv : g_cache) {
            const ClassKey& c = kv.first;
            const kc_config& f = kv.second.cfg;
            os << c.k << ' ' << c.n_samples << ' ' << c.bloom_bits << ' ' << c.n_hashes << ' ' << c.min_gt1 << ' '
               << c.bases_log2 << ' ' << c.sms << ' ' << f.strategy << ' ' << f.part_bits << ' ' << f.smem_table_log2
               << ' ' << f.ctas_per_sm << ' ' << f.scatter_mode << ' ' << f.split_max << ' ' << kv.second.ms << '\n';
        }
    }
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return tune_fail(KC_ERR_ARG, std::string("cannot write ") + tmp + ": " + std::strerror(errno));
        f << os.str();
        if (!f.good()) return tune_fail(KC_ERR_ARG, std::string("write failed: ") + tmp);
    }
    if (std::rename(tmp.c_str(), path) != 0)
        return tune_fail(KC_ERR_ARG, std::string("cannot replace ") + path + ": " + std::strerror(errno));
    return KC_OK;
}

kc_status kc_tune_cache_load(const char* path) {
    if (!path) return tune_fail(KC_ERR_ARG, "kc_tune_cache_load: null path");
    std::ifstream f(path);
    if (!f) return tune_fail(KC_ERR_ARG, std::string("cannot read ") + path);
    std::string line;
    if (!std::getline(f, line) || line != "kc-tune-cache 1") return tune_fail(KC_ERR_ARG, "not a kc tuning cache file");
    std::map<ClassKey, Entry> add;
    int lineno = 1;
    while (std::getline(f, line)) {
        ++lineno;
        if (line.empty()) continue;
        std::istringstream is(line);
        ClassKey c{};
        kc_config cfg;
        kc_default_config(&cfg);
        double ms = 0;
        uint32_t strategy, pb, tl, cps, sm, split;
        if (!(is >> c.k >> c.n_samples >> c.bloom_bits >> c.n_hashes >> c.min_gt1 >> c.bases_log2 >> c.sms >> strategy >>
              pb >> tl >> cps >> sm >> split >> ms))
            return tune_fail(KC_ERR_ARG, "malformed tuning cache line " + std::to_string(lineno));
        std::string rest;
        if (is >> rest) return tune_fail(KC_ERR_ARG, "trailing fields on tuning cache line " + std::to_string(lineno));
        if (c.k < 1 || c.k > 31 || c.n_samples < 1 || c.n_samples > 2 || c.bloom_bits < 4096 ||
            (c.bloom_bits & (c.bloom_bits - 1)) || c.n_hashes < 1 || c.n_hashes > 10 || strategy > 2 || pb > 20 ||
            (tl && (tl < 10 || tl > 13)) || sm > 4 || (split > 13 && split != KC_SPLIT_NONE))
            return tune_fail(KC_ERR_ARG, "out-of-range value on tuning cache line " + std::to_string(lineno));
        cfg.strategy = strategy;
        cfg.part_bits = pb;
        cfg.smem_table_log2 = tl;
        cfg.ctas_per_sm = cps;
        cfg.scatter_mode = sm;
        cfg.split_max = split;
        add[c] = Entry{cfg, ms};
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : add) g_cache[kv.first] = kv.second;
    return KC_OK;
}

void kc_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.clear();
}

}  // extern "C"

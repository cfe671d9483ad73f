// kc_merge_results: the host-side merge of per-owner results.
//
// Handles that own disjoint hash ranges of one job (kc_config.own_bits) each
// return their keys in ascending order; a key belongs to exactly one owner, so
// the job's result is the union of theirs in key order (the paper's partitions
// by k-mer, each owner with its own structures, Section II-B; the Unify unit
// then writes one ordered table).  Runs are cut into key ranges by splitters
// sampled from them; each range is merged by one host thread with a small heap.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/kc.h"

namespace kc {
void set_last_error(const std::string& msg);
}

namespace {

struct Run {
    const uint64_t* keys;
    const uint32_t* counts;
    uint64_t n;
};

kc_status merge_fail(const std::string& msg) {
    kc::set_last_error(msg);
    return KC_ERR_ARG;
}

}  // namespace

extern "C" kc_status kc_merge_results(int n_runs, const uint64_t* const* keys, const uint32_t* const* counts,
                                      const uint64_t* n, int n_samples, uint64_t* out_keys, uint32_t* out_counts) {
    kc::set_last_error("");
    if (n_runs < 0) return merge_fail("n_runs must be >= 0");
    if (n_samples < 1 || n_samples > 2) return merge_fail("n_samples must be 1 or 2");
    if (n_runs > 0 && (!keys || !n)) return merge_fail("keys or n is null");
    std::vector<Run> runs;
    uint64_t total = 0;
    for (int r = 0; r < n_runs; ++r) {
        if (n[r] == 0) continue;
        if (!keys[r]) return merge_fail("keys of a non-empty run is null");
        if (out_counts && (!counts || !counts[r])) return merge_fail("counts of a non-empty run is null");
        for (uint64_t i = 1; i < n[r]; ++i)
            if (keys[r][i] <= keys[r][i - 1]) return merge_fail("run " + std::to_string(r) + " is not strictly ascending");
        runs.push_back({keys[r], out_counts ? counts[r] : nullptr, n[r]});
        total += n[r];
    }
    if (total == 0) return KC_OK;
    if (!out_keys) return merge_fail("out_keys is null");

    // key-range splitters from a sample of every run
    unsigned T = total >= (1ull << 20) ? std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1u;
    std::vector<uint64_t> split;
    if (T > 1) {
        std::vector<uint64_t> sample;
        for (const Run& r : runs)
            for (uint64_t i = 0; i < r.n; i += std::max<uint64_t>(1, r.n / 256)) sample.push_back(r.keys[i]);
        std::sort(sample.begin(), sample.end());
        for (unsigned t = 1; t < T; ++t) split.push_back(sample[sample.size() * t / T]);
        split.erase(std::unique(split.begin(), split.end()), split.end());
    }
    T = (unsigned)split.size() + 1;
    // run r's part in range t: [cut[t][r], cut[t + 1][r])
    std::vector<std::vector<uint64_t>> cut(T + 1, std::vector<uint64_t>(runs.size()));
    for (size_t r = 0; r < runs.size(); ++r) {
        cut[0][r] = 0;
        for (unsigned t = 1; t < T; ++t)
            cut[t][r] = (uint64_t)(std::lower_bound(runs[r].keys, runs[r].keys + runs[r].n, split[t - 1]) - runs[r].keys);
        cut[T][r] = runs[r].n;
    }
    std::vector<uint64_t> out_off(T + 1, 0);
    for (unsigned t = 0; t < T; ++t) {
        uint64_t m = 0;
        for (size_t r = 0; r < runs.size(); ++r) m += cut[t + 1][r] - cut[t][r];
        out_off[t + 1] = out_off[t] + m;
    }
    std::vector<char> dup(T, 0);
    auto work = [&](unsigned t) {
        using Item = std::pair<uint64_t, size_t>;  // key, run
        std::vector<Item> heap;
        std::vector<uint64_t> pos(runs.size());
        for (size_t r = 0; r < runs.size(); ++r) {
            pos[r] = cut[t][r];
            if (pos[r] < cut[t + 1][r]) heap.push_back({runs[r].keys[pos[r]], r});
        }
        auto greater = [](const Item& a, const Item& b) { return a.first > b.first; };
        std::make_heap(heap.begin(), heap.end(), greater);
        uint64_t o = out_off[t];
        while (!heap.empty()) {
            std::pop_heap(heap.begin(), heap.end(), greater);
            const size_t r = heap.back().second;
            heap.pop_back();
            const uint64_t key = runs[r].keys[pos[r]];
            if (o > out_off[t] && out_keys[o - 1] == key) dup[t] = 1;
            out_keys[o] = key;
            if (out_counts)
                std::memcpy(out_counts + o * (uint64_t)n_samples, runs[r].counts + pos[r] * (uint64_t)n_samples,
                            sizeof(uint32_t) * (size_t)n_samples);
            ++o;
            if (++pos[r] < cut[t + 1][r]) {
                heap.push_back({runs[r].keys[pos[r]], r});
                std::push_heap(heap.begin(), heap.end(), greater);
            }
        }
    };
    if (T == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < T; ++t) pool.emplace_back(work, t);
        for (auto& th : pool) th.join();
    }
    for (unsigned t = 0; t < T; ++t)
        if (dup[t]) return merge_fail("a key appears in two runs: the owned ranges overlap");
    // ranges meet at splitters: a key equal to a splitter lands in the upper range of every run
    return KC_OK;
}

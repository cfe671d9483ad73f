// Batched finalize: many partitioned counting jobs in one set of launches.
//
// Consume: one persistent launch over a device work queue of (job, partition)
// items from every job of the batch.  Each CTA takes the next item, keeps the
// partition's filter slice and table in shared memory (filter update, candidate
// claims, exact recount, survivor compaction; the same steps as the single-job
// consumer) and moves on, so uneven jobs share the GPU without a launch each.
// Sort: every job's survivors are bucketed by the top bits of their key into
// one flat bucket array covering all jobs, scanned once, scattered into each
// job's own result arrays, and each bucket sorted by one warp.  These launches
// read every size and pointer from a device-side batch descriptor, so the
// sequence is captured once in a CUDA graph and replayed for every batch.
// A single kc_finalize is a batch of one.

#include <algorithm>
#include <cstring>
#include <vector>

#include "kc_ctx.h"

namespace kc {

struct JobDesc {
    // consumer
    int part_bits, slice_log2, table_log2, bloom_shift;
    int n_hashes, n_samples, all_candidates, key_bits;
    uint32_t min_count;
    int n_batches;
    uint32_t item_base;  // first queue item of this job
    uint32_t part_base;  // partition of the job's first item
    const uint64_t* const* data;
    const uint64_t* const* starts;
    const int* samples;
    unsigned long long* bloom;
    uint64_t* sv_keys;
    uint64_t* sv_vals;
    uint64_t sv_cap;
    uint64_t* failed;  // per overflowing partition: its first hash not yet counted
    DevCounters* ctr;
    // sort
    int sort_bits;
    int split_max;  // consumer: finest split level 2^split_max before the fallback
    uint64_t bucket_base;  // first bucket of this job in the flat arrays
    uint64_t n_buckets;
    uint64_t* res_keys;
    uint64_t* res_vals;
    uint64_t res_cap;
    uint64_t flat_base;  // this job's first survivor in the batch's survivors, in job order (set by the plan)
    // survivors histogrammed by the consumer itself (the sort's bucket bits
    // fixed before it runs): fixed_bits >= 0, hist_job = the job's first
    // bucket counter, hist_shift = key_bits - fixed_bits; else fixed_bits = -1
    int fixed_bits;
    int hist_shift;
    uint32_t* hist_job;
};

struct BatchDesc {
    const JobDesc* jobs;
    const uint32_t* item_job;
    unsigned long long* counters;  // per job: [2j] survivors, [2j+1] failed partitions
    unsigned int* head;            // work-queue head
    unsigned int* err;             // DERR_* bits of the sort
    uint32_t n_jobs;
    uint32_t n_items;
    uint64_t n_buckets;  // total over jobs
    uint32_t* hist;
    uint64_t* starts;
    uint64_t* cursor;
    unsigned long long* tiles;
    uint64_t n_tiles;
    uint64_t buckets_cap;  // room of hist / starts / cursor
    int all_packable;      // set by the plan: every job's small buckets sort packed (k_warp_sort_q)
    uint64_t n_flat;       // set by the plan: survivors of all jobs
    int hist_early;        // the consumer has histogrammed the survivors: the sort does not
    // the survivors scattered into their buckets, (key, value) side by side in
    // the flat bucket order of all jobs; the bucket sorts write the results
    ulonglong2* pairs;
    uint64_t pairs_cap;
};

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kConsumeThreads = 512;
constexpr int kTile = 4096;
constexpr uint32_t kChunk = 1u << 31;  // hashes a consumer loop indexes with 32 bits

// NH > 0: every job of the batch sets NH bits per key; NH = 0: per job.
//
// A partition whose candidates overflow the shared-memory table is counted
// again in 2, 4, ... 2^split_max sub-ranges of its filter slice: the top bits
// of a window's in-slice word index pick its sub-range, so two sub-ranges
// never share a filter word and each one's filter, claims and recount are
// exactly those of the whole partition restricted to its keys.  Sub-ranges
// already finished stay finished when a later one has to split further.
// Only a partition that overflows at the finest level is left to the global
// fallback.  The finest level a job has needed is kept in its counters, and
// its later partitions start there instead of overflowing again.
template <int NH>
__global__ void __launch_bounds__(kConsumeThreads, 2) k_consume_q(const BatchDesc* __restrict__ D) {
    extern __shared__ unsigned long long s_mem[];
    __shared__ int s_fail, s_hint;
    __shared__ unsigned s_item;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t n_items = D->n_items;
    uint64_t cand = 0, claimed = 0;
    DevCounters* last_ctr = nullptr;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(D->head, 1u);
            s_item = it;
            // the finest level this job's partitions have needed so far
            s_hint = it < n_items ? (int)*(volatile unsigned*)&D->jobs[D->item_job[it]].ctr->split_hint : 0;
        }
        __syncthreads();
        const unsigned item = s_item;
        const int hint = s_hint;
        if (item >= n_items) break;
        const uint32_t j = D->item_job[item];
        const JobDesc& J = D->jobs[j];
        const uint32_t part = J.part_base + (item - J.item_base);
        const uint32_t n_sw = 1u << J.slice_log2;
        const uint32_t T = 1u << J.table_log2;
        const uint32_t tmask = T - 1;
        const int S = J.n_samples;
        const int a = J.part_bits;
        // the job's fields the inner loops use, in registers
        const int bloom_shift = J.bloom_shift;
        const bool all_cand = J.all_candidates != 0;
        unsigned long long* sb = s_mem;
        unsigned long long* sk = s_mem + n_sw;
        uint32_t* sc = reinterpret_cast<uint32_t*>(s_mem + n_sw + T);
        if (J.ctr != last_ctr) {  // per-job candidate counters
            cand = warp_sum(cand);
            claimed = warp_sum(claimed);
            if (lane == 0 && last_ctr) {
                if (cand) atomicAdd(&last_ctr->candidates, (unsigned long long)cand);
                if (claimed) atomicAdd(&last_ctr->claimed, (unsigned long long)claimed);
            }
            cand = claimed = 0;
            last_ctr = J.ctr;
        }
        const uint64_t hpre = (uint64_t)part << (64 - a);
        const unsigned long long empty = hpre ^ (1ull << (64 - a));  // a hash of another partition
        int sl = min(hint, J.split_max);  // split level: the partition is taken as 2^sl sub-ranges
        uint32_t sub = 0;  // the sub-range being counted
        bool overflow = false;
        uint64_t h_left = 0;  // first hash left to the fallback
        for (;;) {
            const uint32_t w_n = n_sw >> sl;
            const uint32_t w_lo = sub * w_n;
            const uint32_t smask = (1u << sl) - 1u;
            const int sub_shift = 64 - a - sl;  // sub-range = h bits [sub_shift, 64 - a)
            // a window belongs to the (sub-range of the) partition iff the top
            // a + sl <= 32 bits of its hash equal those of `range`
            const uint64_t range = hpre | ((uint64_t)sub << sub_shift);
            const uint32_t rhi = (uint32_t)(range >> 32), rmask = ~0u << (32 - a - sl);
            uint64_t c_try = 0, k_try = 0;
            for (uint32_t i = threadIdx.x; i < w_n; i += blockDim.x) sb[w_lo + i] = 0ull;
            for (uint32_t i = threadIdx.x; i < T; i += blockDim.x) sk[i] = empty;
            for (uint32_t i = threadIdx.x; i < T * S; i += blockDim.x) sc[i] = 0u;
            if (threadIdx.x == 0) s_fail = 0;
            __syncthreads();
            bool stop = false;
            // A window of a thread's first 64 iterations over the first batch
            // that finds or claims its key in the filter pass is counted there
            // (bit m of `counted` for iteration m); the recount visits only the
            // other windows.  Each window is counted once, by the pass that
            // found its key: the table only grows, and the recount sees it whole.
            uint32_t counted_lo = 0, counted_hi = 0;
            for (int bt = 0; bt < J.n_batches && !stop; ++bt) {
                const uint64_t lo = J.starts[bt][part];
                const uint64_t n_all = J.starts[bt][part + 1] - lo;
                uint32_t* const scol = sc + J.samples[bt];  // this batch's count column
                // 32-bit indices within chunks of 2^31 hashes (one chunk, in practice)
                for (uint64_t c0 = 0; c0 < n_all && !stop; c0 += kChunk) {
                    const uint64_t* __restrict__ d = J.data[bt] + lo + c0;
                    const uint32_t n = (uint32_t)min(n_all - c0, (uint64_t)kChunk);
                    const bool first = bt == 0 && c0 == 0;
                    // each thread's next hash is in flight while it handles the current one
                    uint64_t hn = threadIdx.x < n ? __ldcg(d + threadIdx.x) : 0ull;
                    uint32_t m = 0;
                    for (uint32_t t = threadIdx.x; t < n; t += kConsumeThreads, ++m) {
                        const uint64_t h = hn;
                        if (t + kConsumeThreads < n) hn = __ldcg(d + t + kConsumeThreads);  // read again by the recount: keep in L2
                        if ((((uint32_t)(h >> 32)) ^ rhi) & rmask) continue;  // run padding, or another sub-range
                        const uint32_t w = (uint32_t)(h >> bloom_shift) & (n_sw - 1);
                        const uint64_t g = mixer64(h);
                        const uint64_t pat = NH > 0 ? bloom_pattern_n<(NH > 0 ? NH : 1)>(g) : bloom_pattern_rt(g, J.n_hashes);
                        const unsigned long long old = atomicOr(sb + w, (unsigned long long)pat);
                        if (all_cand || (old & pat) == pat) {
                            ++c_try;
                            uint32_t slot;
                            const int r = smem_claim(sk, tmask, (uint32_t)h & tmask, h, empty, slot);
                            if (r < 0) {
                                s_fail = 1;
                                stop = true;
                                break;
                            }
                            if (first && m < 64) {
                                atomicAdd(scol + slot * S, 1u);
                                if (m < 32) counted_lo |= 1u << m;
                                else counted_hi |= 1u << (m - 32);
                            }
                            if (r > 0) {
                                ++k_try;
                                if (*(volatile int*)&s_fail) {  // another thread overflowed: give up early
                                    stop = true;
                                    break;
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();
            const int failed = s_fail;
            __syncthreads();
            if (failed) {
                if (sl < J.split_max) {
                    ++sl;
                    sub <<= 1;
                    continue;
                }
                overflow = true;
                h_left = range;
                break;
            }
            cand += c_try;
            claimed += k_try;
            for (int bt = 0; bt < J.n_batches; ++bt) {
                const uint64_t lo = J.starts[bt][part];
                const uint64_t n_all = J.starts[bt][part + 1] - lo;
                uint32_t* const scol = sc + J.samples[bt];
                for (uint64_t c0 = 0; c0 < n_all; c0 += kChunk) {
                    const uint64_t* __restrict__ d = J.data[bt] + lo + c0;
                    const uint32_t n = (uint32_t)min(n_all - c0, (uint64_t)kChunk);
                    uint32_t t0 = threadIdx.x;  // first iteration of the dense loop below
                    if (bt == 0 && c0 == 0) {
                        // iterations m < 64 the filter pass did not count, taken
                        // by their bits; each one's hash is loaded a step ahead
                        const uint32_t iters = threadIdx.x < n ? (n - 1 - threadIdx.x) / kConsumeThreads + 1 : 0;
                        const uint32_t mi = iters < 64 ? iters : 64;
                        const uint64_t in_range = mi == 64 ? ~0ull : (1ull << mi) - 1ull;
                        uint64_t todo = ~(((uint64_t)counted_hi << 32) | counted_lo) & in_range;
                        t0 = threadIdx.x + 64u * kConsumeThreads;
                        uint64_t hn = todo ? __ldcs(d + threadIdx.x + (uint32_t)(__ffsll((long long)todo) - 1) * kConsumeThreads) : 0ull;
                        while (todo) {
                            const uint64_t h = hn;
                            todo &= todo - 1ull;
                            if (todo) hn = __ldcs(d + threadIdx.x + (uint32_t)(__ffsll((long long)todo) - 1) * kConsumeThreads);
                            if ((((uint32_t)(h >> 32)) ^ rhi) & rmask) continue;
                            const int s = smem_find(sk, tmask, (uint32_t)h & tmask, h, empty);
                            if (s >= 0) atomicAdd(scol + (uint32_t)s * S, 1u);
                        }
                    }
                    if (t0 >= n) continue;
                    uint64_t hn = __ldcs(d + t0);
                    for (uint32_t t = t0; t < n; t += kConsumeThreads) {
                        const uint64_t h = hn;
                        if (t + kConsumeThreads < n) hn = sl ? __ldcg(d + t + kConsumeThreads) : __ldcs(d + t + kConsumeThreads);  // last use unless split
                        if ((((uint32_t)(h >> 32)) ^ rhi) & rmask) continue;
                        const int s = smem_find(sk, tmask, (uint32_t)h & tmask, h, empty);
                        if (s >= 0) atomicAdd(scol + (uint32_t)s * S, 1u);
                    }
                }
            }
            __syncthreads();
            for (uint32_t i0 = threadIdx.x & ~31u; i0 < T; i0 += blockDim.x) {
                const uint32_t i = i0 + lane;
                const unsigned long long k1 = sk[i];
                uint64_t v = 0;
                bool keep = false;
                if (k1 != empty) {
                    const uint32_t c0 = sc[i * S];
                    const uint32_t c1 = S == 2 ? sc[i * S + 1] : 0u;
                    keep = (uint64_t)c0 + c1 >= J.min_count;
                    v = (uint64_t)c0 | ((uint64_t)c1 << 32);
                }
                const unsigned ballot = __ballot_sync(kFull, keep);
                if (ballot) {
                    const int leader = __ffs(ballot) - 1;
                    unsigned long long pos0 = 0;
                    if (lane == leader) pos0 = atomicAdd(&D->counters[2 * j], (unsigned long long)__popc(ballot));
                    pos0 = __shfl_sync(kFull, pos0, leader);
                    if (keep) {
                        const uint64_t pos = pos0 + __popc(ballot & lt);
                        if (pos < J.sv_cap) {
                            const uint64_t key = unmixer64(k1);
                            J.sv_keys[pos] = key;
                            J.sv_vals[pos] = v;
                            if (J.hist_job) atomicAdd(J.hist_job + (key >> J.hist_shift), 1u);
                        }
                    }
                }
            }
            unsigned long long* gb = J.bloom + (uint64_t)part * n_sw + w_lo;
            for (uint32_t i = threadIdx.x; i < w_n; i += blockDim.x) gb[i] = sb[w_lo + i];
            __syncthreads();
            if (++sub > smask) break;
        }
        if (threadIdx.x == 0) {
            if (overflow) J.failed[atomicAdd(&D->counters[2 * j + 1], 1ull)] = h_left;
            else if (sl) atomicAdd(&J.ctr->split_parts, 1u);
            if (sl > hint) atomicMax(&J.ctr->split_hint, (unsigned)sl);
        }
    }
    cand = warp_sum(cand);
    claimed = warp_sum(claimed);
    if (lane == 0 && last_ctr) {
        if (cand) atomicAdd(&last_ctr->candidates, (unsigned long long)cand);
        if (claimed) atomicAdd(&last_ctr->claimed, (unsigned long long)claimed);
    }
}

// Start of a batch: the queue head, the sort error bits and every job's
// survivor and failed-partition counters at zero.
__global__ void k_reset_q(const BatchDesc* __restrict__ D) {
    for (uint32_t i = threadIdx.x; i < 2 * D->n_jobs; i += blockDim.x) D->counters[i] = 0ull;
    if (threadIdx.x == 0) {
        *D->head = 0u;
        *D->err = 0u;
    }
}

// Sort plan, on the device once the survivors are counted: per job, bucket
// bits for at most about 32 survivors a bucket and the job's first bucket in
// the flat arrays; the total into D->n_buckets.  More buckets than the arrays
// hold (never, when the host sized them from the survivor capacities) is an
// internal error and sorts nothing.
__global__ void k_plan_q(BatchDesc* __restrict__ D) {
    if (threadIdx.x != 0) return;
    JobDesc* jobs = const_cast<JobDesc*>(D->jobs);
    uint64_t total = 0, flat = 0;
    int packable = 1;
    bool short_arrays = false;
    for (uint32_t j = 0; j < D->n_jobs; ++j) {
        JobDesc& J = jobs[j];
        uint64_t nsv = D->counters[2 * j];
        if (nsv > J.sv_cap) nsv = J.sv_cap;
        if (nsv > J.res_cap) {  // result arrays too short (a sort run ahead of the count): sort nothing
            short_arrays = true;
            nsv = 0;
        }
        J.flat_base = flat;
        flat += nsv;
        if (nsv < 1) nsv = 1;
        int bits = 0;
        if (J.fixed_bits >= 0) bits = J.fixed_bits;  // the consumer's histogram has these buckets
        else
            while (bits < 24 && bits < J.key_bits && (nsv >> bits) > 32) ++bits;
        J.sort_bits = bits;
        J.bucket_base = total;
        J.n_buckets = 1ull << bits;
        total += J.n_buckets;
        if (J.key_bits - bits > 58) packable = 0;
    }
    D->all_packable = packable;
    // short result arrays: no bucket and no survivor is sorted at all (a
    // histogram the consumer took may count that job's survivors), and the
    // host sorts again into larger arrays
    D->n_flat = short_arrays ? 0 : flat;
    *D->err = short_arrays ? DERR_INTERNAL : 0u;
    if (total > D->buckets_cap) {
        atomicOr(D->err, DERR_INTERNAL);
        total = 0;
    }
    D->n_buckets = short_arrays ? 0 : total;
}

__global__ void k_zero_hist_q(const BatchDesc* __restrict__ D) {
    if (D->hist_early) return;  // counted by the consumer
    const uint64_t n = D->n_buckets;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) D->hist[i] = 0u;
}

// Job owning the batch's survivor number i (jobs are in survivor order).
__device__ __forceinline__ uint32_t job_of_survivor(const BatchDesc* D, uint64_t i) {
    uint32_t lo = 0, hi = D->n_jobs;  // invariant: jobs[lo].flat_base <= i
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (D->jobs[mid].flat_base <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// A thread's view of the job that owns its current survivor: the fields the
// histogram and scatter use, reloaded only when the survivor index passes
// into a later job (a thread's indices only grow).
struct SurvivorJob {
    uint32_t j;
    uint64_t lo, hi;  // flat survivor range of job j
    const uint64_t* keys;
    const uint64_t* vals;
    int shift;
    uint64_t n_buckets, bucket_base;
    uint64_t* res_keys;
    uint64_t* res_vals;
    uint64_t res_cap;
    __device__ void load(const BatchDesc* D, uint32_t jj) {
        j = jj;
        const JobDesc& J = D->jobs[jj];
        lo = J.flat_base;
        hi = jj + 1 < D->n_jobs ? D->jobs[jj + 1].flat_base : D->n_flat;
        keys = J.sv_keys;
        vals = J.sv_vals;
        shift = J.key_bits - J.sort_bits;
        n_buckets = J.n_buckets;
        bucket_base = J.bucket_base;
        res_keys = J.res_keys;
        res_vals = J.res_vals;
        res_cap = J.res_cap;
    }
    __device__ void seek(const BatchDesc* D, uint64_t i) {
        while (i >= hi && j + 1 < D->n_jobs) load(D, j + 1);
    }
};

// The survivors of all jobs as one flat range: every thread takes survivors
// across job boundaries, so one job or many keep the whole grid busy.
__global__ void k_prefix_hist_q(const BatchDesc* __restrict__ D) {
    if (D->hist_early) return;  // counted by the consumer
    const uint64_t n = D->n_flat;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    SurvivorJob S;
    S.load(D, job_of_survivor(D, i));
    for (; i < n; i += stride) {
        S.seek(D, i);
        const uint64_t b = S.keys[i - S.lo] >> S.shift;
        if (b < S.n_buckets) atomicAdd(D->hist + S.bucket_base + b, 1u);
        else atomicOr(D->err, DERR_INTERNAL);
    }
}

__device__ __forceinline__ unsigned long long block_scan_ex(unsigned long long x, unsigned long long* total) {
    __shared__ unsigned long long s_w[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    __syncthreads();
    if (lane == 31) s_w[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < nw ? s_w[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    *total = s_w[nw - 1];
    return v - x + (wid ? s_w[wid - 1] : 0ull);
}

// Flat exclusive scan of D->hist over D->n_buckets counters (fixed grid of
// D's tile capacity; tiles past the end exit).
__global__ void __launch_bounds__(1024) k_scan_tiles_q(const BatchDesc* __restrict__ D) {
    const uint64_t n = D->n_buckets;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    if (t0 >= n) return;
    unsigned long long x = 0;
    for (int j = 0; j < kTile / 1024; ++j) {
        const uint64_t i = t0 + (uint64_t)j * 1024 + threadIdx.x;
        if (i < n) x += D->hist[i];
    }
    unsigned long long tot;
    block_scan_ex(x, &tot);
    if (threadIdx.x == 0) D->tiles[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top_q(const BatchDesc* __restrict__ D) {
    const uint64_t n_tiles = (D->n_buckets + kTile - 1) / kTile;
    unsigned long long run_base = 0;
    for (uint64_t c0 = 0; c0 < n_tiles; c0 += 1024) {
        const uint64_t i = c0 + threadIdx.x;
        const unsigned long long x = i < n_tiles ? D->tiles[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_scan_ex(x, &tot);
        if (i < n_tiles) D->tiles[i] = run_base + ex;
        run_base += tot;
    }
}

__global__ void __launch_bounds__(1024) k_scan_apply_q(const BatchDesc* __restrict__ D) {
    const uint64_t n = D->n_buckets;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    if (t0 >= n) return;
    const uint64_t i0 = t0 + (uint64_t)threadIdx.x * 4;
    uint32_t c[4];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = i0 + j < n ? D->hist[i0 + j] : 0u;
        sum += c[j];
    }
    unsigned long long tot;
    unsigned long long run = block_scan_ex(sum, &tot) + D->tiles[blockIdx.x];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) {
            D->starts[i0 + j] = run;
            D->cursor[i0 + j] = run;
        }
        run += c[j];
    }
    if (i0 < n && i0 + 4 >= n) D->starts[n] = run;
}

__global__ void k_scatter_q(const BatchDesc* __restrict__ D) {
    const uint64_t n = D->n_flat;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    SurvivorJob S;
    S.load(D, job_of_survivor(D, i));
    uint64_t job0 = D->starts[S.bucket_base];
    for (; i < n; i += stride) {
        if (i >= S.hi) {
            S.seek(D, i);
            job0 = D->starts[S.bucket_base];
        }
        const uint64_t k = i - S.lo;
        const uint64_t key = S.keys[k];
        const uint64_t val = S.vals[k];
        const uint64_t b = key >> S.shift;
        if (b >= S.n_buckets) {
            atomicOr(D->err, DERR_INTERNAL);
            continue;
        }
        const uint64_t gpos = atomicAdd(reinterpret_cast<unsigned long long*>(D->cursor) + S.bucket_base + b, 1ull);
        if (gpos - job0 >= S.res_cap || gpos >= D->pairs_cap) {
            atomicOr(D->err, DERR_INTERNAL);
            continue;
        }
        D->pairs[gpos] = make_ulonglong2(key, val);  // one 16-byte store
    }
}

// Job owning flat bucket fb (jobs are in bucket order).
__device__ __forceinline__ uint32_t job_of_bucket(const BatchDesc* D, uint64_t fb) {
    uint32_t lo = 0, hi = D->n_jobs;  // invariant: jobs[lo].bucket_base <= fb
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (D->jobs[mid].bucket_base <= fb) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Buckets of 2..64 keys (nearly all of them: the bits are chosen for about
// 32 keys a bucket on average, and canonical keys, the smaller of two
// orientations, are up to twice as dense at the low end of the key space):
// one warp each, packed (warp_sort32_packed / warp_sort64_packed), small
// enough in registers for six 256-thread CTAs per SM, so the loads of many
// buckets are in flight.
__global__ void __launch_bounds__(256, 6) k_warp_sort_q(const BatchDesc* __restrict__ D) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nb = D->n_buckets;
    const bool packable = D->all_packable != 0;
    for (uint64_t fb = warp; fb < nb; fb += n_warps) {
        const uint64_t g0 = D->starts[fb], n64 = D->starts[fb + 1] - g0;
        if (n64 == 0) continue;
        const JobDesc& J = D->jobs[job_of_bucket(D, fb)];
        const uint64_t lo = g0 - D->starts[J.bucket_base];
        const ulonglong2* __restrict__ src = D->pairs + g0;
        if (!packable || n64 == 1 || n64 > 64) {
            // one key, or sorted later in place (k_warp_sort_big_q): the pairs
            // into the result arrays as they are
            for (uint64_t i = lane; i < n64; i += 32) {
                const ulonglong2 q = src[i];
                J.res_keys[lo + i] = q.x;
                J.res_vals[lo + i] = q.y;
            }
            continue;
        }
        const int shift = J.key_bits - J.sort_bits;  // the bucket's keys share the bits above shift (<= 58)
        if (n64 <= 32) {
            const bool in = lane < (int)n64;
            const ulonglong2 q = in ? src[lane] : make_ulonglong2(0ull, 0ull);
            uint64_t k = q.x, v = q.y;
            warp_sort32_core(k, v, in, lane, shift);
            if (in) {
                J.res_keys[lo + lane] = k;
                J.res_vals[lo + lane] = v;
            }
        } else {
            const bool in1 = 32 + lane < (int)n64;
            const ulonglong2 q0 = src[lane];
            const ulonglong2 q1 = in1 ? src[32 + lane] : make_ulonglong2(0ull, 0ull);
            uint64_t k0 = q0.x, v0 = q0.y, k1 = q1.x, v1 = q1.y;
            warp_sort64_core(k0, v0, k1, v1, true, in1, lane, shift);
            J.res_keys[lo + lane] = k0;
            J.res_vals[lo + lane] = v0;
            if (in1) {
                J.res_keys[lo + 32 + lane] = k1;
                J.res_vals[lo + 32 + lane] = v1;
            }
        }
    }
}

// Buckets of 65..256 keys in registers of one warp, and every bucket of a
// batch whose bucket bits leave too many key bits to pack; larger ones are
// flagged for the shared-memory sort.
// The lanes of a warp look at 32 buckets at once; the warp then sorts the
// ones it has to, one after the other.
__global__ void __launch_bounds__(256, 2) k_warp_sort_big_q(const BatchDesc* __restrict__ D) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nb = D->n_buckets;
    const bool all_pack = D->all_packable != 0;
    for (uint64_t base = warp * 32; base < nb; base += n_warps * 32) {
        const uint64_t fb = base + (uint64_t)lane;
        const uint64_t m64 = fb < nb ? D->starts[fb + 1] - D->starts[fb] : 0ull;
        unsigned todo = __ballot_sync(kFull, m64 > 64 || (m64 > 1 && !all_pack));
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint64_t b = base + (uint64_t)src;
            const uint64_t n64 = __shfl_sync(kFull, m64, src);
            if (n64 > 256) {
                if (lane == 0) atomicOr(D->err, DERR_SORT_MEDIUM);
                continue;
            }
            const JobDesc& J = D->jobs[job_of_bucket(D, b)];
            const uint64_t lo = D->starts[b] - D->starts[J.bucket_base];
            const int n = (int)n64;
            if (n <= 32) warp_sort_bucket<1>(J.res_keys, J.res_vals, lo, n, lane);
            else if (n <= 64) warp_sort_bucket<2>(J.res_keys, J.res_vals, lo, n, lane);
            else if (n <= 128) warp_sort_bucket<4>(J.res_keys, J.res_vals, lo, n, lane);
            else warp_sort_bucket<8>(J.res_keys, J.res_vals, lo, n, lane);
        }
    }
}

// Buckets of 257..2048 keys: one CTA each, bitonic network in shared memory
// (mirror form, indices >= n act as +infinity).  Larger ones are flagged.
constexpr int kMedCap = 2048;

__global__ void __launch_bounds__(256) k_medium_sort_q(const BatchDesc* __restrict__ D) {
    __shared__ uint64_t sk[kMedCap];
    __shared__ uint64_t sv[kMedCap];
    for (uint64_t fb = blockIdx.x; fb < D->n_buckets; fb += gridDim.x) {
        const uint64_t n64 = D->starts[fb + 1] - D->starts[fb];
        if (n64 <= 256) continue;
        if (n64 > (uint64_t)kMedCap) {
            if (threadIdx.x == 0) atomicOr(D->err, DERR_SORT_BUCKET);
            continue;
        }
        const JobDesc& J = D->jobs[job_of_bucket(D, fb)];
        const uint64_t lo = D->starts[fb] - D->starts[J.bucket_base];
        const int n = (int)n64;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            sk[i] = J.res_keys[lo + i];
            sv[i] = J.res_vals[lo + i];
        }
        int n2 = 1;
        while (n2 < n) n2 <<= 1;
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1) {
            const int half = size >> 1;
            for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
                const int blk = i / half, off = i % half;
                const int x = blk * size + off, y = blk * size + size - 1 - off;
                if (y < n && sk[x] > sk[y]) {
                    const uint64_t tk = sk[x], tv = sv[x];
                    sk[x] = sk[y];
                    sv[x] = sv[y];
                    sk[y] = tk;
                    sv[y] = tv;
                }
            }
            __syncthreads();
            for (int stride = size >> 2; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
                    const int x = 2 * i - (i & (stride - 1)), y = x + stride;
                    if (y < n && sk[x] > sk[y]) {
                        const uint64_t tk = sk[x], tv = sv[x];
                        sk[x] = sk[y];
                        sv[x] = sv[y];
                        sk[y] = tk;
                        sv[y] = tv;
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            J.res_keys[lo + i] = sk[i];
            J.res_vals[lo + i] = sv[i];
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace kc

using namespace kcapi;

struct kc_batch_ctx {
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0, sm_count = 152, max_optin = 0, max_sm = 0;
    kc::BatchDesc* d_desc = nullptr;
    kc::JobDesc* d_jobs = nullptr;
    uint32_t* d_item_job = nullptr;
    unsigned long long* d_counters = nullptr;
    unsigned int* d_flags = nullptr;  // [0] queue head, [1] sort error bits
    size_t jobs_cap = 0, items_cap = 0;
    uint32_t* d_hist = nullptr;
    uint64_t* d_starts = nullptr;
    uint64_t* d_cursor = nullptr;
    unsigned long long* d_tiles = nullptr;
    uint64_t buckets_cap = 0, tiles_cap = 0;
    cudaGraphExec_t sort_graph = nullptr;
    // captured consumer launches, one per launch shape
    struct ConsumeGraph {
        int nh, n_ctas;
        size_t smem;
        cudaGraphExec_t exec;
    };
    std::vector<ConsumeGraph> consume_graphs;
    std::vector<kc::JobDesc> jobs;
    std::vector<uint32_t> item_job;
    uint64_t launches = 0;
    // pinned host memory the finalize reads its counters back into (so the
    // copies queue behind the kernels and one synchronisation waits for all)
    unsigned char* h_read = nullptr;
    size_t h_read_jobs = 0;
    // the scattered survivors of a batch, (key, value) pairs
    ulonglong2* d_pairs = nullptr;
    size_t pairs_cap = 0;
};

namespace {

template <class T>
kc_status grow(T*& p, size_t& cap, size_t need) {
    if (need <= cap) return KC_OK;
    size_t n = std::max<size_t>(need, cap * 2);
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    KC_CUDA(cudaMalloc(&p, n * sizeof(T)));
    cap = n;
    return KC_OK;
}

kc_status ensure_jobs(kc_batch_ctx* b, size_t n_jobs, size_t n_items) {
    if (n_jobs > b->jobs_cap) {
        size_t n = std::max<size_t>(n_jobs, b->jobs_cap * 2);
        std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
        if (b->d_jobs) cudaFree(b->d_jobs);
        if (b->d_counters) cudaFree(b->d_counters);
        b->d_jobs = nullptr;
        b->d_counters = nullptr;
        b->jobs_cap = 0;
        KC_CUDA(cudaMalloc(&b->d_jobs, n * sizeof(kc::JobDesc)));
        KC_CUDA(cudaMalloc(&b->d_counters, 2 * n * sizeof(unsigned long long)));
        b->jobs_cap = n;
    }
    size_t cap = b->items_cap;
    kc_status s = grow(b->d_item_job, cap, n_items);
    b->items_cap = cap;
    return s;
}

// Readback area for n jobs: the error word, then 2 n queue counters, then n
// device-counter blocks.
kc_status ensure_readback(kc_batch_ctx* b, size_t n) {
    if (n <= b->h_read_jobs) return KC_OK;
    const size_t m = std::max<size_t>(n, 2 * b->h_read_jobs);
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());  // pinning may synchronise the device
    if (b->h_read) cudaFreeHost(b->h_read);
    b->h_read = nullptr;
    b->h_read_jobs = 0;
    KC_CUDA(cudaMallocHost(&b->h_read, 64 + m * (16 + sizeof(kc::DevCounters))));
    b->h_read_jobs = m;
    return KC_OK;
}

kc_status ensure_buckets(kc_batch_ctx* b, uint64_t n_buckets) {
    if (n_buckets <= b->buckets_cap) return KC_OK;
    const uint64_t n = std::max<uint64_t>(n_buckets, 1ull << 16);
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    if (b->d_hist) cudaFree(b->d_hist);
    if (b->d_starts) cudaFree(b->d_starts);
    if (b->d_cursor) cudaFree(b->d_cursor);
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_hist = nullptr;
    b->d_starts = b->d_cursor = nullptr;
    b->d_tiles = nullptr;
    b->buckets_cap = 0;
    const uint64_t tiles = (n + kc::kTile - 1) / kc::kTile;
    KC_CUDA(cudaMalloc(&b->d_hist, n * 4));
    KC_CUDA(cudaMalloc(&b->d_starts, (n + 1) * 8));
    KC_CUDA(cudaMalloc(&b->d_cursor, n * 8));
    KC_CUDA(cudaMalloc(&b->d_tiles, tiles * 8));
    b->buckets_cap = n;
    b->tiles_cap = tiles;
    if (b->sort_graph) {  // the graph holds the old capacities
        cudaGraphExecDestroy(b->sort_graph);
        b->sort_graph = nullptr;
    }
    return KC_OK;
}

// Capture the sort sequence once; it reads everything else from d_desc.
kc_status capture_sort_graph(kc_batch_ctx* b) {
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    cudaGraph_t g = nullptr;
    KC_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    const unsigned grid2 = (unsigned)b->sm_count * 16;  // latency-bound atomics: many threads in flight
    kc::k_plan_q<<<1, 32, 0, b->st>>>(b->d_desc);
    kc::k_zero_hist_q<<<(unsigned)b->sm_count * 4, 256, 0, b->st>>>(b->d_desc);
    kc::k_prefix_hist_q<<<grid2, 256, 0, b->st>>>(b->d_desc);
    kc::k_scan_tiles_q<<<(unsigned)b->tiles_cap, 1024, 0, b->st>>>(b->d_desc);
    kc::k_scan_top_q<<<1, 1024, 0, b->st>>>(b->d_desc);
    kc::k_scan_apply_q<<<(unsigned)b->tiles_cap, 1024, 0, b->st>>>(b->d_desc);
    kc::k_scatter_q<<<grid2, 256, 0, b->st>>>(b->d_desc);
    kc::k_warp_sort_q<<<(unsigned)b->sm_count * 16, 256, 0, b->st>>>(b->d_desc);
    kc::k_warp_sort_big_q<<<(unsigned)b->sm_count * 2, 256, 0, b->st>>>(b->d_desc);
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(sort)");
    e = cudaGraphInstantiate(&b->sort_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(sort)");
    return KC_OK;
}

kc_status upload_desc(kc_batch_ctx* b, uint32_t n_jobs, uint32_t n_items, uint64_t n_buckets, int hist_early = 0) {
    kc::BatchDesc d{};
    d.hist_early = hist_early;
    d.pairs = b->d_pairs;
    d.pairs_cap = b->pairs_cap;
    d.buckets_cap = b->buckets_cap;
    d.jobs = b->d_jobs;
    d.item_job = b->d_item_job;
    d.counters = b->d_counters;
    d.head = b->d_flags;
    d.err = b->d_flags + 1;
    d.n_jobs = n_jobs;
    d.n_items = n_items;
    d.n_buckets = n_buckets;
    d.hist = b->d_hist;
    d.starts = b->d_starts;
    d.cursor = b->d_cursor;
    d.tiles = b->d_tiles;
    d.n_tiles = b->tiles_cap;
    KC_CUDA(cudaMemcpyAsync(b->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, b->st));
    KC_CUDA(cudaMemcpyAsync(b->d_jobs, b->jobs.data(), n_jobs * sizeof(kc::JobDesc), cudaMemcpyHostToDevice, b->st));
    return KC_OK;
}

struct JobWork {
    kc_handle h;
    std::vector<uint64_t> hs;  // partition starts of every batch
    uint64_t total_w = 0, max_w = 0;
    uint64_t* sv_keys = nullptr;
    uint64_t* sv_vals = nullptr;
    uint64_t sv_cap = 0;
    uint64_t* failed = nullptr;
    void* meta = nullptr;
};

void release_work(kc_batch_ctx* b, std::vector<JobWork>& w) {
    for (auto& x : w) {
        if (x.sv_keys) cudaFreeAsync(x.sv_keys, b->st);
        if (x.sv_vals) cudaFreeAsync(x.sv_vals, b->st);
        if (x.failed) cudaFreeAsync(x.failed, b->st);
        if (x.meta) cudaFreeAsync(x.meta, b->st);
        x.sv_keys = x.sv_vals = nullptr;
        x.failed = nullptr;
        x.meta = nullptr;
    }
}

// prepare: set the kernel's shared-memory limit (before any capture);
// otherwise launch it.
template <int NH>
cudaError_t launch_consume_nh(bool prepare, int n_ctas, size_t smem, const kc::BatchDesc* d, cudaStream_t st) {
    if (prepare) return kc::allow_max_dynamic_smem(kc::k_consume_q<NH>);
    kc::k_consume_q<NH><<<n_ctas, kc::kConsumeThreads, smem, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_consume(bool prepare, int nh, int n_ctas, size_t smem, const kc::BatchDesc* d, cudaStream_t st) {
    switch (nh) {
        case 1: return launch_consume_nh<1>(prepare, n_ctas, smem, d, st);
        case 2: return launch_consume_nh<2>(prepare, n_ctas, smem, d, st);
        case 3: return launch_consume_nh<3>(prepare, n_ctas, smem, d, st);
        case 4: return launch_consume_nh<4>(prepare, n_ctas, smem, d, st);
        case 5: return launch_consume_nh<5>(prepare, n_ctas, smem, d, st);
        case 6: return launch_consume_nh<6>(prepare, n_ctas, smem, d, st);
        case 7: return launch_consume_nh<7>(prepare, n_ctas, smem, d, st);
        case 8: return launch_consume_nh<8>(prepare, n_ctas, smem, d, st);
        case 9: return launch_consume_nh<9>(prepare, n_ctas, smem, d, st);
        case 10: return launch_consume_nh<10>(prepare, n_ctas, smem, d, st);
        default: return launch_consume_nh<0>(prepare, n_ctas, smem, d, st);
    }
}

// The batch's counters reset and its persistent consumer launch, captured
// once per launch shape (hash count, grid, shared memory); everything else
// they read comes from the device descriptor.
kc_status consume_graph(kc_batch_ctx* b, int nh, int n_ctas, size_t smem, cudaGraphExec_t* out) {
    for (const auto& g : b->consume_graphs)
        if (g.nh == nh && g.n_ctas == n_ctas && g.smem == smem) {
            *out = g.exec;
            return KC_OK;
        }
    KC_CUDA(launch_consume(true, nh, n_ctas, smem, b->d_desc, b->st));
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    cudaGraph_t g = nullptr;
    KC_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    kc::k_reset_q<<<1, 256, 0, b->st>>>(b->d_desc);
    launch_consume(false, nh, n_ctas, smem, b->d_desc, b->st);
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(consumer)");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(consumer)");
    b->consume_graphs.push_back({nh, n_ctas, smem, exec});
    *out = exec;
    return KC_OK;
}

// Bucket bits of a sort of at most n survivors (about 32 a bucket).
int sort_bits_for(uint64_t n, int key_bits) {
    int bits = 0;
    n = std::max<uint64_t>(1, n);
    while (bits < 24 && bits < key_bits && (n >> bits) > 32) ++bits;
    return bits;
}

// Partitions whose shared-memory table overflowed: rebuild their filter
// slice from zero and count them in a global table (kc_partition.cu kernels).
kc_status run_fallbacks(kc_batch_ctx* b, JobWork& x, uint32_t j, uint32_t n_failed) {
    kc_handle h = x.h;
    const kc::JobDesc& J = b->jobs[j];
    const uint64_t P = 1ull << h->part_bits;
    const size_t nb = h->batches.size();
    std::vector<uint64_t> fl(n_failed);  // first hash of each partition not yet counted
    KC_CUDA(cudaMemcpyAsync(fl.data(), x.failed, n_failed * 8, cudaMemcpyDeviceToHost, b->st));
    unsigned long long n_sv = 0;
    KC_CUDA(cudaMemcpyAsync(&n_sv, b->d_counters + 2 * j, 8, cudaMemcpyDeviceToHost, b->st));
    if (x.hs.empty()) {  // sized from the host's counts: the partition starts were not read yet
        x.hs.resize(nb * (P + 1));
        for (size_t t = 0; t < nb; ++t)
            KC_CUDA(cudaMemcpyAsync(x.hs.data() + t * (P + 1), h->batches[t].hstarts, (P + 1) * 8,
                                    cudaMemcpyDeviceToHost, b->st));
    }
    KC_CUDA(cudaStreamSynchronize(b->st));
    auto windows_of = [&](uint32_t p) {
        uint64_t w = 0;
        for (size_t t = 0; t < nb; ++t) w += x.hs[t * (P + 1) + p + 1] - x.hs[t * (P + 1) + p];
        return w;
    };
    const int a = h->part_bits;
    uint64_t extra = 0;
    for (uint64_t hl : fl) extra += windows_of((uint32_t)(hl >> (64 - a)));
    const uint64_t need = n_sv + extra;
    if (need > x.sv_cap) {
        uint64_t *nk = nullptr, *nv = nullptr;
        cudaError_t e;
        if ((e = cudaMallocAsync(&nk, need * 8, b->st)) != cudaSuccess ||
            (e = cudaMallocAsync(&nv, need * 8, b->st)) != cudaSuccess) {
            if (nk) cudaFreeAsync(nk, b->st);
            return cuda_fail(e, "cudaMallocAsync(fallback survivors)");
        }
        const uint64_t have = std::min<uint64_t>(n_sv, x.sv_cap);
        KC_CUDA(cudaMemcpyAsync(nk, x.sv_keys, have * 8, cudaMemcpyDeviceToDevice, b->st));
        KC_CUDA(cudaMemcpyAsync(nv, x.sv_vals, have * 8, cudaMemcpyDeviceToDevice, b->st));
        cudaFreeAsync(x.sv_keys, b->st);
        cudaFreeAsync(x.sv_vals, b->st);
        x.sv_keys = nk;
        x.sv_vals = nv;
        x.sv_cap = need;
    }
    const uint64_t n_sw = 1ull << h->slice_log2;
    for (uint64_t hl : fl) {
        const uint32_t p = (uint32_t)(hl >> (64 - a));
        const uint64_t w_lo = (hl >> J.bloom_shift) & (n_sw - 1);  // sub-ranges below are finished
        uint64_t slots = 1024;
        while (slots < 2 * windows_of(p)) slots <<= 1;
        kc::Slot* table = nullptr;
        cudaError_t e = cudaMallocAsync(&table, slots * sizeof(kc::Slot), b->st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(fallback table)");
        KC_CUDA(cudaMemsetAsync(table, 0, slots * sizeof(kc::Slot), b->st));
        KC_CUDA(cudaMemsetAsync(h->bloom + p * n_sw + w_lo, 0, (n_sw - w_lo) * 8, b->st));
        kc::FallbackArgs F{};
        F.data = J.data;
        F.starts = J.starts;
        F.samples = J.samples;
        F.part = p;
        F.h_lo = hl;
        F.part_bits = h->part_bits;
        F.bloom_shift = J.bloom_shift;
        F.n_hashes = h->n_hashes;
        F.n_samples = h->n_samples;
        F.all_candidates = J.all_candidates;
        F.min_count = h->min_count;
        F.bloom = reinterpret_cast<unsigned long long*>(h->bloom);
        F.table = table;
        F.table_mask = slots - 1;
        F.out_keys = x.sv_keys;
        F.out_vals = x.sv_vals;
        F.out_cap = x.sv_cap;
        F.n_out = b->d_counters + 2 * j;
        F.ctr = h->ctr;
        for (size_t t = 0; t < nb; ++t) kc::launch_fb_claim(F, (int)t, b->st);
        for (size_t t = 0; t < nb; ++t) kc::launch_fb_recount(F, (int)t, b->st);
        kc::launch_fb_compact(F, b->st);
        h->launches += 2 * nb + 1;
        KC_LAUNCHED("fallback launches");
        cudaFreeAsync(table, b->st);
    }
    h->fallback_partitions += n_failed;
    return KC_OK;
}

}  // namespace

kc_status kc_batch_create_internal(cudaStream_t st, kc_batch_ctx** out) {
    *out = nullptr;
    kc_batch_ctx* b = new (std::nothrow) kc_batch_ctx();
    if (!b) return fail(KC_ERR_OOM_HOST, "host allocation");
    auto bail = [&](kc_status s) {
        kc_batch_destroy_internal(b);
        return s;
    };
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    cudaDeviceGetAttribute(&b->max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    cudaDeviceGetAttribute(&b->max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device);
    if (st) {
        b->st = st;
    } else {
        if ((e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaStreamCreate"));
        b->own_stream = true;
    }
    {
        std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
        if ((e = cudaMalloc(&b->d_desc, sizeof(kc::BatchDesc))) != cudaSuccess ||
            (e = cudaMalloc(&b->d_flags, 2 * sizeof(unsigned int))) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc(batch descriptor)"));
    }
    *out = b;
    return KC_OK;
}

void kc_batch_destroy_internal(kc_batch_ctx* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->sort_graph) cudaGraphExecDestroy(b->sort_graph);
    for (auto& g : b->consume_graphs) cudaGraphExecDestroy(g.exec);
    std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
    cudaFree(b->d_desc);
    cudaFree(b->d_flags);
    cudaFree(b->d_jobs);
    cudaFree(b->d_counters);
    cudaFree(b->d_item_job);
    cudaFree(b->d_hist);
    cudaFree(b->d_starts);
    cudaFree(b->d_cursor);
    cudaFree(b->d_tiles);
    if (b->h_read) cudaFreeHost(b->h_read);
    cudaFree(b->d_pairs);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

// Finalize partitions [part_lo, part_hi) of every job (clamped to the job's
// partition count); the handles become finalized only when `last`.
kc_status finalize_core(kc_batch_ctx* b, kc_handle* hs, int n, uint32_t part_lo, uint32_t part_hi, bool last) {
    if (!b || !hs || n < 0) return fail(KC_ERR_ARG, "null argument");
    if (n == 0) return KC_OK;
    cudaStream_t st = b->st;
    std::vector<JobWork> work((size_t)n);
    const bool one = n == 1 && hs[0]->stream == st;  // no cross-stream ordering needed
    const bool timed = n == 1;                         // phase times go to the only handle
    bool fast = true;  // every job whole: sized from host counts (below)
    for (int j = 0; j < n; ++j) {
        kc_handle h = hs[j];
        if (!h) return fail(KC_ERR_ARG, "null handle in batch");
        if (h->state == State::Poisoned) return fail(KC_ERR_STATE, "handle poisoned by an earlier error; call kc_reset");
        if (h->state != State::Open) return fail(KC_ERR_STATE, "handle already finalized");
        if (h->strategy != KC_STRATEGY_PARTITIONED) return fail(KC_ERR_ARG, "batched finalize needs the partitioned strategy");
        for (int i = 0; i < j; ++i)
            if (hs[i] == h) return fail(KC_ERR_ARG, "handle listed twice");
        work[j].h = h;
        fast = fast && part_lo == 0 && part_hi >= (1u << h->part_bits) && !h->owner && !h->deferred;
    }
    // order the batch after every handle's queued work: at once when the
    // setup reads the grouping back, else just before the consumer, so the
    // setup's uploads queue while the handles' grouping still runs
    const auto order_after_handles = [&]() -> kc_status {
        if (!one)
            for (int j = 0; j < n; ++j) {
                KC_CUDA(cudaEventRecord(hs[j]->ev_main, hs[j]->stream));
                KC_CUDA(cudaStreamWaitEvent(st, hs[j]->ev_main, 0));
            }
        return KC_OK;
    };
    if (!fast) {
        kc_status os = order_after_handles();
        if (os != KC_OK) return os;
    }
    // Partition sizes of every job, and each job's counters (ingest errors):
    // read back when the batch covers part of a job's partitions (spill
    // groups, owned ranges, hash ranges of kept reads).  A job counted whole
    // is sized from the host's counts instead (bases and reads added), so no
    // host round trip sits between its grouping and its consumer; its ingest
    // errors are read after the consumer.
    kc_status rs = ensure_readback(b, (size_t)n);
    if (rs != KC_OK) return rs;
    unsigned& err = *reinterpret_cast<unsigned*>(b->h_read);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b->h_read + 64);
    kc::DevCounters* hc = reinterpret_cast<kc::DevCounters*>(b->h_read + 64 + 16 * (size_t)n);
    if (!fast) {
        for (int j = 0; j < n; ++j) {
            kc_handle h = hs[j];
            const uint64_t P = 1ull << h->part_bits;
            work[j].hs.resize(h->batches.size() * (P + 1));
            for (size_t t = 0; t < h->batches.size(); ++t)
                KC_CUDA(cudaMemcpyAsync(work[j].hs.data() + t * (P + 1), h->batches[t].hstarts, (P + 1) * 8,
                                        cudaMemcpyDeviceToHost, st));
            KC_CUDA(cudaMemcpyAsync(&hc[j], h->ctr, sizeof(kc::DevCounters), cudaMemcpyDeviceToHost, st));
        }
        KC_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < n; ++j) {
            hs[j]->host_ctr = hc[j];
            kc_status s = device_errors(hs[j]);
            if (s != KC_OK) return s;
        }
    }

    // per-job consumer setup
    b->jobs.assign((size_t)n, kc::JobDesc{});
    b->item_job.clear();
    size_t smem_max = 0;
    for (int j = 0; j < n; ++j) {
        JobWork& x = work[j];
        kc_handle h = x.h;
        const uint64_t P = 1ull << h->part_bits;
        // the requested partitions that the handle owns (kc_config.own_bits)
        const uint64_t p_lo = std::max<uint64_t>(std::min<uint64_t>(part_lo, P), h->own_plo);
        const uint64_t p_hi = std::max<uint64_t>(p_lo, std::min<uint64_t>(std::min<uint64_t>(part_hi, P), h->own_phi));
        const size_t nb = h->batches.size();
        if (fast) {
            // windows: at most one per base; about bases - reads (k - 1), spread
            // evenly over the partitions by the hash
            const uint64_t est = h->bases > h->reads * (uint64_t)(h->k - 1) ? h->bases - h->reads * (uint64_t)(h->k - 1) : 0;
            x.total_w = h->bases;
            x.max_w = est / P + est / P / 16 + 64;
        } else {
            for (uint64_t p = p_lo; p < p_hi; ++p) {
                uint64_t w = 0;
                for (size_t t = 0; t < nb; ++t) w += x.hs[t * (P + 1) + p + 1] - x.hs[t * (P + 1) + p];
                x.max_w = std::max(x.max_w, w);
                x.total_w += w;
            }
        }
        // Shared-memory table: one slot per 8 windows of the largest partition
        // (2^10..2^13 slots); partitions with more candidates split.
        int tl = (int)h->cfg.smem_table_log2;
        if (!tl) {
            tl = 10;
            while (tl < 13 && (1ull << tl) < x.max_w / 8) ++tl;
        }
        while (tl > 10 && kc::consume_smem(h->slice_log2, tl, h->n_samples) + 1024 > (size_t)b->max_optin) --tl;
        const size_t smem = kc::consume_smem(h->slice_log2, tl, h->n_samples);
        if (smem + 1024 > (size_t)b->max_optin) {
            release_work(b, work);
            return fail(KC_ERR_INTERNAL, "partition does not fit shared memory");
        }
        smem_max = std::max(smem_max, smem);
        // survivors: a partition holds at most 2^split_max tables of keys and
        // one key per min_count of its windows
        // the consumer tells a window's sub-range by the top 32 bits of its hash
        const int split_max = h->cfg.split_max == KC_SPLIT_NONE ? 0
                              : std::min<int>(std::min<int>(h->slice_log2, 32 - h->part_bits),
                                              h->cfg.split_max ? (int)h->cfg.split_max : 6);
        x.sv_cap = 0;
        if (fast) {  // every survivor has min_count windows, and no partition more than 2^split_max tables
            x.sv_cap = std::min<uint64_t>((p_hi - p_lo) << (tl + split_max), x.total_w / std::max<uint32_t>(1, h->min_count));
        } else {
            for (uint64_t p = p_lo; p < p_hi; ++p) {
                uint64_t w = 0;
                for (size_t t = 0; t < nb; ++t) w += x.hs[t * (P + 1) + p + 1] - x.hs[t * (P + 1) + p];
                x.sv_cap += std::min<uint64_t>(1ull << (tl + split_max), w / std::max<uint32_t>(1, h->min_count));
            }
        }
        x.sv_cap = std::max<uint64_t>(1, x.sv_cap);
        const size_t meta_bytes = std::max<size_t>(16, nb * 20);
        cudaError_t e;
        if ((e = cudaMallocAsync(&x.sv_keys, x.sv_cap * 8, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&x.sv_vals, x.sv_cap * 8, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&x.failed, P * 8, st)) != cudaSuccess ||
            (e = cudaMallocAsync(&x.meta, meta_bytes, st)) != cudaSuccess) {
            release_work(b, work);
            return cuda_fail(e, "cudaMallocAsync(batch consumer)");
        }
        std::vector<unsigned char> hm(meta_bytes, 0);
        for (size_t t = 0; t < nb; ++t) {
            const uint64_t dp = (uint64_t)(uintptr_t)h->batches[t].hdata;
            const uint64_t sp = (uint64_t)(uintptr_t)h->batches[t].hstarts;
            const int smp = h->batches[t].sample;
            std::memcpy(hm.data() + t * 8, &dp, 8);
            std::memcpy(hm.data() + nb * 8 + t * 8, &sp, 8);
            std::memcpy(hm.data() + nb * 16 + t * 4, &smp, 4);
        }
        KC_CUDA(cudaMemcpyAsync(x.meta, hm.data(), meta_bytes, cudaMemcpyHostToDevice, st));
        kc::JobDesc& J = b->jobs[j];
        J.part_bits = h->part_bits;
        J.slice_log2 = h->slice_log2;
        J.table_log2 = tl;
        J.bloom_shift = 64 - h->log2_words;
        J.n_hashes = h->n_hashes;
        J.n_samples = h->n_samples;
        J.all_candidates = h->min_count <= 1 ? 1 : 0;
        J.key_bits = 2 * h->k;
        J.min_count = h->min_count;
        J.split_max = split_max;
        J.fixed_bits = -1;  // the plan chooses the bucket bits (unless set below)
        J.hist_job = nullptr;
        J.n_batches = (int)nb;
        J.item_base = (uint32_t)b->item_job.size();
        J.part_base = (uint32_t)p_lo;
        J.data = reinterpret_cast<const uint64_t* const*>(x.meta);
        J.starts = reinterpret_cast<const uint64_t* const*>(static_cast<char*>(x.meta) + nb * 8);
        J.samples = reinterpret_cast<const int*>(static_cast<char*>(x.meta) + nb * 16);
        J.bloom = reinterpret_cast<unsigned long long*>(h->bloom);
        J.sv_keys = x.sv_keys;
        J.sv_vals = x.sv_vals;
        J.sv_cap = x.sv_cap;
        J.failed = x.failed;
        J.ctr = h->ctr;
        for (uint64_t p = p_lo; p < p_hi; ++p) b->item_job.push_back((uint32_t)j);
    }
    const uint32_t n_items = (uint32_t)b->item_job.size();
    kc_status s = ensure_jobs(b, (size_t)n, n_items);
    if (s != KC_OK) {
        release_work(b, work);
        return s;
    }
    KC_CUDA(cudaMemcpyAsync(b->d_item_job, b->item_job.data(), n_items * 4, cudaMemcpyHostToDevice, st));
    // Whole jobs whose handles still hold result arrays from their last job:
    // the sort graph runs right behind the consumer into those arrays, with
    // bucket arrays for that many survivors, and one host round trip checks
    // both (no partition left to the fallback, every job's survivors within
    // its arrays); otherwise the sort runs again after the fallbacks, into
    // arrays of the right size.
    // The bucket bits are then fixed in advance (for the kept arrays' size),
    // so the consumer histograms the survivors as it writes them and the sort
    // graph skips its histogram pass.
    bool spec = fast;
    for (int j = 0; j < n && spec; ++j) spec = hs[j]->res_keys != nullptr && hs[j]->res_cap > 0;
    uint64_t spec_buckets = 0;
    if (spec) {
        for (int j = 0; j < n; ++j) {
            kc::JobDesc& J = b->jobs[j];
            J.fixed_bits = sort_bits_for(std::min<uint64_t>(hs[j]->res_cap, J.sv_cap), J.key_bits);
            J.hist_shift = J.key_bits - J.fixed_bits;
            spec_buckets += 1ull << J.fixed_bits;
            J.res_keys = hs[j]->res_keys;
            J.res_vals = hs[j]->res_vals;
            J.res_cap = hs[j]->res_cap;
        }
        uint64_t spec_pairs = 0;
        for (int j = 0; j < n; ++j) spec_pairs += hs[j]->res_cap;
        if ((s = ensure_buckets(b, spec_buckets)) != KC_OK || (s = grow(b->d_pairs, b->pairs_cap, spec_pairs)) != KC_OK ||
            (!b->sort_graph && (s = capture_sort_graph(b)) != KC_OK)) {
            release_work(b, work);
            return s;
        }
        uint64_t first = 0;  // the plan gives the jobs their buckets in this order
        for (int j = 0; j < n; ++j) {
            b->jobs[j].hist_job = b->d_hist + first;
            first += 1ull << b->jobs[j].fixed_bits;
        }
        KC_CUDA(cudaMemsetAsync(b->d_hist, 0, spec_buckets * 4, st));
    }
    if ((s = upload_desc(b, (uint32_t)n, n_items, 0, spec ? 1 : 0)) != KC_OK) {
        release_work(b, work);
        return s;
    }
    int nh = hs[0]->n_hashes;
    for (int j = 1; j < n; ++j)
        if (hs[j]->n_hashes != nh) nh = 0;
    const int per_sm = std::max(1, std::min(4, b->max_sm / (int)(smem_max + 2048)));
    // a persistent grid (CTAs without an item exit at once), so the captured
    // launch depends on the hash count and shared memory alone
    const int n_ctas = b->sm_count * per_sm;
    cudaGraphExec_t cons = nullptr;
    if ((s = consume_graph(b, nh, n_ctas, smem_max, &cons)) != KC_OK) {
        release_work(b, work);
        return s;
    }

    if (fast && (s = order_after_handles()) != KC_OK) {
        release_work(b, work);
        return s;
    }
    // consume: one persistent launch over the (job, partition) queue
    cudaEvent_t t0 = timed ? phase_begin(hs[0], st) : nullptr;
    KC_CUDA(cudaGraphLaunch(cons, st));
    if (timed) phase_end(hs[0], kPass2, t0, st);
    err = 0;
    if (spec) {
        t0 = timed ? phase_begin(hs[0], st) : nullptr;
        KC_CUDA(cudaGraphLaunch(b->sort_graph, st));
        if (timed) phase_end(hs[0], kSort, t0, st);
        KC_CUDA(cudaMemcpyAsync(&err, b->d_flags + 1, 4, cudaMemcpyDeviceToHost, st));
    }
    KC_CUDA(cudaMemcpyAsync(cnt, b->d_counters, 2 * (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    if (fast)
        for (int j = 0; j < n; ++j) KC_CUDA(cudaMemcpyAsync(&hc[j], hs[j]->ctr, sizeof(kc::DevCounters), cudaMemcpyDeviceToHost, st));
    KC_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) work[j].h->launches += spec ? 11 : 2;
    if (fast) {
        for (int j = 0; j < n; ++j) {
            hs[j]->host_ctr = hc[j];
            kc_status s = device_errors(hs[j]);
            if (s != KC_OK) {
                release_work(b, work);
                return s;
            }
        }
    }

    // partitions whose table overflowed (rare): counted in global tables
    bool any_fb = false;
    for (int j = 0; j < n; ++j) any_fb |= cnt[2 * j + 1] != 0;
    bool sorted = spec && !any_fb && !(err & kc::DERR_INTERNAL);
    for (int j = 0; j < n && sorted; ++j) sorted = std::min<uint64_t>(cnt[2 * j], b->jobs[j].sv_cap) <= hs[j]->res_cap;
    if (sorted)
        for (int j = 0; j < n; ++j) hs[j]->n_result = std::min<uint64_t>(cnt[2 * j], b->jobs[j].sv_cap);
    if (any_fb) {
        for (int j = 0; j < n; ++j) {
            if (!cnt[2 * j + 1]) continue;
            t0 = timed ? phase_begin(hs[0], st) : nullptr;
            s = run_fallbacks(b, work[j], (uint32_t)j, (uint32_t)cnt[2 * j + 1]);
            if (timed) phase_end(hs[0], kCompact, t0, st);
            if (s != KC_OK) {
                release_work(b, work);
                return s;
            }
            kc::JobDesc& J = b->jobs[j];
            J.sv_keys = work[j].sv_keys;
            J.sv_vals = work[j].sv_vals;
            J.sv_cap = work[j].sv_cap;
        }
        KC_CUDA(cudaMemcpyAsync(cnt, b->d_counters, 2 * (size_t)n * 8, cudaMemcpyDeviceToHost, st));
        for (int j = 0; j < n; ++j) KC_CUDA(cudaMemcpyAsync(&hc[j], hs[j]->ctr, sizeof(kc::DevCounters), cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < n; ++j) {
            hs[j]->host_ctr = hc[j];
            if ((s = device_errors(hs[j])) != KC_OK) {
                release_work(b, work);
                return s;
            }
        }
    }

    // sort: result arrays of each job's survivor count (a job's arrays are
    // kept for its next job when large enough), bucket arrays for as many
    // buckets as the plan will give; the plan itself runs on the device
    if (!sorted) {
    for (int j = 0; j < n; ++j) {  // the plan chooses the bits and the sort histograms again
        b->jobs[j].fixed_bits = -1;
        b->jobs[j].hist_job = nullptr;
    }
    uint64_t bucket_need = 0, pairs_need = 0;
    for (int j = 0; j < n; ++j) {
        kc_handle h = hs[j];
        kc::JobDesc& J = b->jobs[j];
        const uint64_t nsv = std::min<uint64_t>(cnt[2 * j], J.sv_cap);
        bucket_need += 1ull << sort_bits_for(nsv, J.key_bits);
        pairs_need += nsv;
        const uint64_t cap = std::max<uint64_t>(1, nsv);
        if (!h->res_keys || h->res_cap < cap) {
            free_result(h);
            cudaError_t e;
            if ((e = cudaMallocAsync(&h->res_keys, cap * 8, st)) != cudaSuccess ||
                (e = cudaMallocAsync(&h->res_vals, cap * 8, st)) != cudaSuccess) {
                free_result(h);
                release_work(b, work);
                return cuda_fail(e, "cudaMallocAsync(result)");
            }
            h->res_cap = cap;
        }
        h->n_result = nsv;
        J.res_keys = h->res_keys;
        J.res_vals = h->res_vals;
        J.res_cap = h->res_cap;
    }
    if ((s = ensure_buckets(b, bucket_need)) != KC_OK ||
        (s = grow(b->d_pairs, b->pairs_cap, std::max<uint64_t>(1, pairs_need))) != KC_OK ||
        (s = upload_desc(b, (uint32_t)n, n_items, 0)) != KC_OK ||
        (!b->sort_graph && (s = capture_sort_graph(b)) != KC_OK)) {
        release_work(b, work);
        return s;
    }
    t0 = timed ? phase_begin(hs[0], st) : nullptr;
    KC_CUDA(cudaGraphLaunch(b->sort_graph, st));
    if (timed) phase_end(hs[0], kSort, t0, st);
    KC_CUDA(cudaMemcpyAsync(&err, b->d_flags + 1, 4, cudaMemcpyDeviceToHost, st));
    KC_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) work[j].h->launches += 9;
    }  // !sorted
    if (err & kc::DERR_INTERNAL) {
        release_work(b, work);
        for (int j = 0; j < n; ++j) hs[j]->state = State::Poisoned;
        return fail(KC_ERR_INTERNAL, "sort: key outside its bucket range");
    }
    t0 = timed && (err & (kc::DERR_SORT_MEDIUM | kc::DERR_SORT_BUCKET)) ? phase_begin(hs[0], st) : nullptr;
    if (err & kc::DERR_SORT_MEDIUM) {
        kc::k_medium_sort_q<<<(unsigned)b->sm_count * 4, 256, 0, st>>>(b->d_desc);
        KC_LAUNCHED("batched medium sort launch");
        KC_CUDA(cudaMemcpyAsync(&err, b->d_flags + 1, 4, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < n; ++j) hs[j]->launches += 1;
    }
    if (err & kc::DERR_SORT_BUCKET) {  // rare: buckets above 2048 keys, sorted in global memory
        // the plan is on the device: read back the jobs' bucket ranges and the starts
        std::vector<kc::JobDesc> jd((size_t)n);
        uint64_t nbk = 0;
        KC_CUDA(cudaMemcpyAsync(jd.data(), b->d_jobs, n * sizeof(kc::JobDesc), cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        for (const auto& J : jd) nbk = std::max<uint64_t>(nbk, J.bucket_base + J.n_buckets);
        std::vector<uint64_t> starts(nbk + 1);
        KC_CUDA(cudaMemcpyAsync(starts.data(), b->d_starts, (nbk + 1) * 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < n; ++j) {
            const kc::JobDesc& J = jd[j];
            const uint64_t job0 = starts[J.bucket_base];
            for (uint64_t q = 0; q < J.n_buckets; ++q) {
                const uint64_t lo = starts[J.bucket_base + q], m = starts[J.bucket_base + q + 1] - lo;
                if (m > 2048) {
                    kc::launch_bitonic_global(J.res_keys + (lo - job0), J.res_vals + (lo - job0), m, st);
                    hs[j]->launches += 1;
                }
            }
        }
        KC_LAUNCHED("batched global sort launches");
    }
    if (t0) phase_end(hs[0], kSort, t0, st);
    release_work(b, work);
    KC_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < n; ++j) {
        kc_handle h = hs[j];
        h->host_ctr.survivors = h->n_result;
        if (!one) {  // the handle's later work is ordered after the batch
            KC_CUDA(cudaEventRecord(h->ev_copy, st));
            KC_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copy, 0));
        }
        phase_collect(h);
        if (last) h->state = State::Finalized;
    }
    b->launches += 11;
    return KC_OK;
}

// Out-of-core finalize of one handle: the partitions are processed in
// kSpillGroups hash-prefix groups in turn; each group's sorted survivors are
// copied to pinned host memory on the handle's side stream while the next
// group runs, and recorded in the spill directory (first partition, number
// of partitions, host location, items).  kc_dump merges the sorted runs.
constexpr uint32_t kSpillGroups = 64;

// Finalize partitions [part_lo, part_hi) of h and copy their sorted result to
// pinned host memory on the handle's side stream (one spill run).
kc_status spill_group(kc_batch_ctx* b, kc_handle h, uint32_t part_lo, uint32_t part_hi, bool last) {
    kc_status s = finalize_core(b, &h, 1, part_lo, part_hi, last);
    if (s != KC_OK) return s;
    SpillRun run;
    run.first_part = part_lo;
    run.n_parts = part_hi - part_lo;
    run.n_items = h->n_result;
    if (run.n_items) {
        run.host = spill_alloc(h, 2 * run.n_items);
        if (!run.host) return fail(KC_ERR_OOM_HOST, "pinned host memory for a spilled run");
        // the copy waits for the group's sort; the next group runs meanwhile
        KC_CUDA(cudaEventRecord(h->ev_main, b->st));
        KC_CUDA(cudaStreamWaitEvent(h->copy_stream, h->ev_main, 0));
        KC_CUDA(cudaMemcpyAsync(run.host, h->res_keys, run.n_items * 8, cudaMemcpyDeviceToHost, h->copy_stream));
        KC_CUDA(cudaMemcpyAsync(run.host + run.n_items, h->res_vals, run.n_items * 8, cudaMemcpyDeviceToHost,
                                h->copy_stream));
    }
    if (h->res_keys) cudaFreeAsync(h->res_keys, h->copy_stream);
    if (h->res_vals) cudaFreeAsync(h->res_vals, h->copy_stream);
    h->res_keys = h->res_vals = nullptr;
    h->res_cap = 0;
    h->spill_dir.push_back(run);
    h->spilled_bytes += run.n_items * 16;
    return KC_OK;
}

kc_status finish_spill(kc_handle h) {
    KC_CUDA(cudaStreamSynchronize(h->copy_stream));
    uint64_t total = 0;
    for (const auto& r : h->spill_dir) total += r.n_items;
    h->n_result = total;
    h->host_ctr.survivors = total;
    h->spilled = true;
    return KC_OK;
}

// Spill groups of partitions [g * per, (g + 1) * per) that the handle owns.
std::vector<uint32_t> owned_groups(kc_handle h, uint32_t G, uint32_t per, uint32_t g_lo, uint32_t g_hi) {
    std::vector<uint32_t> out;
    for (uint32_t g = g_lo; g < g_hi; ++g)
        if ((g + 1) * per > h->own_plo && g * per < h->own_phi) out.push_back(g);
    return out;
}

kc_status finalize_spilled(kc_batch_ctx* b, kc_handle h) {
    const uint32_t P = 1u << h->part_bits;
    const uint32_t G = std::min(P, kSpillGroups), per = P / G;
    release_spill(h);
    const std::vector<uint32_t> groups = owned_groups(h, G, per, 0, G);
    for (size_t i = 0; i < groups.size(); ++i) {
        const uint32_t g = groups[i];
        kc_status s = spill_group(b, h, g * per, (g + 1) * per, i + 1 == groups.size());
        if (s != KC_OK) return s;
    }
    return finish_spill(h);
}

// Out-of-core finalize of a handle with batches kept as reads (their hashes
// would have passed the device budget).  The hash space is cut into S scan
// ranges, S a power of two chosen so that one range's grouped hashes fit the
// room left; for each range every kept batch is extracted and grouped again
// in pieces, keeping only the range's windows, and the range's spill groups
// are finalized and spilled as by finalize_spilled.  Batches grouped at
// kc_add_reads take part in every range as they are.
kc_status finalize_grouped(kc_batch_ctx* b, kc_handle h) {
    const uint32_t P = 1u << h->part_bits;
    const uint32_t G = std::min(P, kSpillGroups), per = P / G;
    uint64_t kept_bases = 0;
    for (const auto& bt : h->batches)
        if (bt.deferred) kept_bases += bt.n_units * 64;
    // one range: its grouped hashes (8 bytes per window) plus the linear
    // hashes of the piece being grouped, about as large, plus the survivors
    // of one spill group; S = G at most
    const uint64_t room = room_bytes(h);
    uint32_t S = 1;
    while (S < G && 3 * (8 * kept_bases / S) > room) S <<= 1;
    h->scan_groups = S;
    const uint64_t piece_units = std::max<uint64_t>(1ull << 16, (kept_bases / 64) / S + 1);
    release_spill(h);
    std::vector<Batch> kept = h->batches;
    std::vector<uint32_t> all_groups = owned_groups(h, G, per, 0, G);
    const uint32_t last_group = all_groups.empty() ? 0 : all_groups.back();
    cudaStream_t st = h->stream;
    kc_status s = KC_OK;
    for (uint32_t r = 0; r < S && s == KC_OK; ++r) {
        const std::vector<uint32_t> groups = owned_groups(h, G, per, r * (G / S), (r + 1) * (G / S));
        if (groups.empty()) continue;
        // hash range of scan range r, within the handle's own range
        const int pb = h->part_bits;
        const uint64_t p0 = (uint64_t)r * (P / S), p1 = (uint64_t)(r + 1) * (P / S);
        kc::PassParams base = h->params(0);
        base.h_lo = std::max<uint64_t>(h->own_h_lo, p0 << (64 - pb));
        base.h_hi = std::min<uint64_t>(h->own_h_hi, (p1 << (64 - pb)) - 1ull);  // p1 = P wraps to 0: ~0
        std::vector<Batch> pieces;
        cudaEvent_t t0 = phase_begin(h);
        for (const Batch& bt : kept) {
            if (!bt.deferred) {
                pieces.push_back(bt);
                continue;
            }
            for (uint64_t u0 = 0; u0 < bt.n_units && s == KC_OK; u0 += piece_units) {
                Batch pc;
                pc.sample = bt.sample;
                pc.pw = bt.pw + 2 * u0;  // the word after the piece is the next unit's first word (or padding)
                pc.vw = bt.vw + u0;
                pc.n_units = std::min(piece_units, bt.n_units - u0);
                kc::PassParams p = base;
                p.sample = bt.sample;
                s = bucket_batch(h, pc, pc.n_units * 64, st, p, true);
                h->launches += 5;
                pc.pw = pc.vw = nullptr;  // the piece borrows the kept reads
                pc.deferred = true;       // marks hashes to free after the range
                if (s == KC_OK) pieces.push_back(pc);
            }
        }
        phase_end(h, kPass1, t0);
        if (s == KC_OK) {
            h->batches = pieces;
            for (uint32_t g : groups) {
                s = spill_group(b, h, g * per, (g + 1) * per, g == last_group);
                if (s != KC_OK) break;
            }
        }
        for (Batch& pc : pieces)
            if (pc.deferred) {
                if (pc.hdata) cudaFreeAsync(pc.hdata, st);
                if (pc.hstarts) cudaFreeAsync(pc.hstarts, st);
            }
        h->batches = kept;
    }
    if (s != KC_OK) return s;
    return finish_spill(h);
}

// The batches kc_add_reads kept for the batched ingest, of every handle of
// the batch: extracted and grouped on the batch's stream, which waits for each
// handle's stream first; each handle's stream then waits for the grouping.
kc_status ingest_batches(kc_batch_ctx* b, kc_handle* hs, int n) {
    bool any = false;
    for (int j = 0; j < n; ++j) {
        kc_handle h = hs[j];
        if (!h || h->state != State::Open || h->strategy != KC_STRATEGY_PARTITIONED) continue;
        for (const Batch& bt : h->batches) any |= bt.pending;
    }
    if (!any) return KC_OK;
    std::vector<kc_handle> open;
    for (int j = 0; j < n; ++j) {
        kc_handle h = hs[j];
        if (!h || h->state != State::Open || h->strategy != KC_STRATEGY_PARTITIONED) continue;
        for (kc_handle o : open)
            if (o == h) return fail(KC_ERR_ARG, "handle listed twice");
        open.push_back(h);
        KC_CUDA(cudaEventRecord(h->ev_main, h->stream));
        KC_CUDA(cudaStreamWaitEvent(b->st, h->ev_main, 0));
    }
    kc_status s = ingest_pending(open.data(), (int)open.size(), b->st, b->sm_count);
    for (kc_handle h : open) {
        KC_CUDA(cudaEventRecord(h->ev_main, b->st));
        KC_CUDA(cudaStreamWaitEvent(h->stream, h->ev_main, 0));
    }
    return s;
}

kc_status kc_batch_finalize_internal(kc_batch_ctx* b, kc_handle* hs, int n) {
    if (b && hs && n > 0) {
        kc_status s = ingest_batches(b, hs, n);
        if (s != KC_OK) return s;
    }
    if (n == 1 && hs && hs[0] && hs[0]->strategy == KC_STRATEGY_PARTITIONED && hs[0]->state == State::Open) {
        kc_handle h = hs[0];
        if (h->deferred) return finalize_grouped(b, h);
        if (h->cfg.spill) return finalize_spilled(b, h);
        // survivors and sorted result, 16 bytes each per key, at most one
        // key per min_count windows (and per base): spill when they would
        // not fit
        if (32 * (h->bases / std::max<uint32_t>(1, h->min_count)) > room_bytes(h)) return finalize_spilled(b, h);
    }
    if (!hs || n <= 1) return finalize_core(b, hs, n, 0, 0xffffffffu, true);
    // handles whose reads passed the device budget are finalized alone, in
    // hash ranges; the others together
    std::vector<kc_handle> rest;
    for (int j = 0; j < n; ++j) {
        if (hs[j] && hs[j]->deferred && hs[j]->strategy == KC_STRATEGY_PARTITIONED && hs[j]->state == State::Open) {
            kc_status s = finalize_grouped(b, hs[j]);
            if (s != KC_OK) return s;
        } else {
            rest.push_back(hs[j]);
        }
    }
    return finalize_core(b, rest.data(), (int)rest.size(), 0, 0xffffffffu, true);
}

extern "C" {

kc_status kc_batch_create(void* stream, kc_batch* out) {
    if (!out) return fail(KC_ERR_ARG, "out is null");
    kc_batch_ctx* b = nullptr;
    kc_status s = kc_batch_create_internal((cudaStream_t)stream, &b);
    *out = b;
    return s;
}

kc_status kc_batch_finalize(kc_batch b, kc_handle* handles, int n) { return kc_batch_finalize_internal(b, handles, n); }

kc_status kc_batch_ingest(kc_batch b, kc_handle* handles, int n) {
    if (!b || (!handles && n > 0) || n < 0) return fail(KC_ERR_ARG, "null batch or handle list");
    for (int j = 0; j < n; ++j) {
        if (!handles[j]) return fail(KC_ERR_ARG, "null handle in batch");
        for (int i = 0; i < j; ++i)
            if (handles[i] == handles[j]) return fail(KC_ERR_ARG, "handle listed twice");
    }
    return ingest_batches(b, handles, n);
}

void kc_batch_destroy(kc_batch b) { kc_batch_destroy_internal(b); }

}  // extern "C"

// Host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "kc_device.cuh"

namespace kc {

// Message returned by kc_last_error() on this thread.
void set_last_error(const std::string& msg);

// Held while a stream is being captured into a graph and around every CUDA
// call that may synchronise the device or the legacy stream (cudaMalloc,
// cudaFree, cudaMallocHost, cudaFreeHost, cudaMemcpy), so that none of them
// lands inside another host thread's capture.
std::mutex& sync_api_mutex();

struct Grid {
    int sm_count = 152;
    int block = 256;
    int ctas_per_sm = 8;
    int ctas() const { return sm_count * ctas_per_sm; }
};

// Ingest: read-start bits from offsets, then valid-window-start bits.
void launch_mark_read_starts(const uint64_t* offsets, uint64_t n_reads, uint64_t base, uint64_t n_local,
                             uint64_t* bd, DevCounters* ctr, cudaStream_t st);
void launch_build_valid(const uint64_t* nmask, const uint64_t* bd, uint64_t n_vwords, uint64_t start_local,
                        uint64_t n_local, int k, uint64_t* vout, DevCounters* ctr, const Grid& g, cudaStream_t st);
// The same for words [w_begin, w_end) only (a chunk whose N-mask words up to
// w_end, inclusive when w_end < n_vwords, are on the device).
void launch_build_valid_range(const uint64_t* nmask, const uint64_t* bd, uint64_t n_vwords, uint64_t w_begin,
                              uint64_t w_end, uint64_t start_local, uint64_t n_local, int k, uint64_t* vout,
                              DevCounters* ctr, const Grid& g, cudaStream_t st);

// Pass 1: filter update, candidates claimed in the table.
void launch_pass1(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, uint64_t* bloom,
                  Slot* table, DevCounters* ctr, const Grid& g, cudaStream_t st);
// Pass 2: exact recount of the keys held in the table.
void launch_pass2(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, Slot* table,
                  DevCounters* ctr, const Grid& g, cudaStream_t st);

// Compaction of slots with summed count >= min_count, with a histogram of the
// survivors' top key bits (bucket = key >> prefix_shift).
void launch_compact(const Slot* table, uint64_t n_slots, int n_samples, uint32_t min_count, uint64_t* keys,
                    uint64_t* vals, DevCounters* ctr, uint32_t* hist, int prefix_shift, const Grid& g,
                    cudaStream_t st);
// starts[0..n] = exclusive scan of hist[0..n); cursor[0..n) = starts[0..n).
// Above 4096 counters a three-kernel multi-CTA scan with a small stream-
// ordered temporary (n <= 2^25).
cudaError_t launch_scan(const uint32_t* hist, uint64_t n, uint64_t* starts, uint64_t* cursor, cudaStream_t st);
// Scatter survivors (at most cap of them) into their buckets; keys whose
// bucket or position would fall outside the arrays set DERR_INTERNAL.
void launch_scatter(const uint64_t* keys, const uint64_t* vals, DevCounters* ctr, uint64_t cap, int prefix_shift,
                    uint64_t n_buckets, uint64_t* cursor, uint64_t* out_keys, uint64_t* out_vals, const Grid& g,
                    cudaStream_t st);
// Sort every bucket of at most warp_sort_capacity() keys in place, one warp
// per bucket; larger buckets set DERR_SORT_MEDIUM and are left alone.
void launch_bucket_sort_warp(uint64_t* keys, uint64_t* vals, const uint64_t* starts, uint64_t n_buckets, int shift,
                             DevCounters* ctr, const Grid& g, cudaStream_t st);
int warp_sort_capacity();
// Sort buckets of warp_sort_capacity()+1 .. bucket_sort_capacity() keys in
// shared memory, one CTA per bucket; larger buckets set DERR_SORT_BUCKET and
// are left for launch_bitonic_global.
void launch_bucket_sort(uint64_t* keys, uint64_t* vals, const uint64_t* starts, uint64_t n_buckets,
                        DevCounters* ctr, cudaStream_t st);
int bucket_sort_capacity();
void launch_bitonic_global(uint64_t* keys, uint64_t* vals, uint64_t n, cudaStream_t st);

void launch_counts_narrow(const uint64_t* vals, uint64_t n, uint32_t* out, cudaStream_t st);

// ---- partitioned strategy (kc_partition.cu) --------------------------------

struct FallbackArgs {
    const uint64_t* const* data;
    const uint64_t* const* starts;
    const int* samples;
    uint32_t part;
    uint64_t h_lo;  // hashes of the partition below h_lo are already counted
    int part_bits;
    int bloom_shift;
    int n_hashes;
    int n_samples;
    int all_candidates;
    uint32_t min_count;
    unsigned long long* bloom;
    Slot* table;
    uint64_t table_mask;
    uint64_t* out_keys;
    uint64_t* out_vals;
    uint64_t out_cap;
    unsigned long long* n_out;
    DevCounters* ctr;
};

size_t bucket_pass_smem(int a);
void launch_bucket_count(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                         int n_ctas, const PassParams& p, int a, uint32_t* counts, cudaStream_t st);
void launch_bucket_offsets(const uint32_t* counts, int n_ctas, int a, int pad4, uint64_t* rel, uint32_t* total,
                           cudaStream_t st);
void launch_bucket_base(uint64_t* rel, const uint64_t* starts, int n_ctas, int a, cudaStream_t st);
size_t staged_scatter_smem(int a);
size_t staged_seg_smem(int a);
// A run of hashes handled by one CTA: src + off .. src + off + len; group =
// the level-1 group the run belongs to (0 with a single level).
struct SegDesc {
    uint64_t off, len, group, pad;
};
// mode 4: the extraction pass writes every CTA's hashes to its own segment of
// a linear array (plus counts); the staged scatter then moves the segments.
// accumulate: add the CTAs' counts to their rows (a later piece of the same
// segments, launched with the same number of CTAs).
// Windows outside [p.h_lo, p.h_hi] are dropped (their number kept goes to
// ctr->kept when the range is not the whole hash space).
void launch_extract_count(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                          int n_ctas, const PassParams& p, int a, uint32_t* counts, uint64_t* g_cursor, SegDesc* seg,
                          uint64_t* lin, DevCounters* ctr, cudaStream_t st,
                          bool accumulate = false);
// Staged scatter of segment c into its runs: bucket (h >> (64 - a1 - a2)) mod
// 2^a2; with a1 > 0 only hashes of the segment's level-1 group.  Segment c
// comes in n_pieces pieces segs[c], segs[c + n_segs], ...
void launch_scatter_staged_seg(const uint64_t* src, const SegDesc* segs, int n_segs, int n_pieces, int a1, int a2,
                               const uint64_t* base, uint64_t* out, cudaStream_t st);
// Batched ingest: the read batches of several jobs extracted and grouped by
// one set of launches.  Each batch is cut into items of whole units; the
// extraction and the staged scatter are persistent kernels over the item
// queue, the per-bucket offsets, scans and run bases cover every batch in one
// launch each.  Per batch: histogram rows and segments of its items, its
// linear hashes, the runs' relative and absolute bases, its bucket totals and
// starts (the batch's partition starts) and its grouped hashes.
struct IngestBatch {
    const uint64_t* pw;
    const uint64_t* vw;
    uint64_t n_units;
    PassParams p;
    int a;             // bucket bits (the first grouping level)
    uint32_t item0;    // first item of the batch in the queue
    uint32_t n_items;  // items of upi units (the last one shorter)
    uint64_t upi;
    uint32_t* counts;   // [n_items][2^a]
    SegDesc* seg;       // [n_items]
    uint64_t* lin;      // linear hashes
    unsigned long long* g_cursor;
    DevCounters* ctr;
    uint64_t* rel;      // [n_items][2^a]: run starts, relative, then absolute
    uint32_t* total;    // [2^a]
    uint64_t* starts;   // [2^a + 1]
    uint64_t* out;      // grouped hashes
    uint64_t bucket_off;  // first (batch, bucket) index of the batch: sum of 2^a over earlier batches
    uint64_t rel_off;     // first (item, bucket) index: sum of n_items 2^a over earlier batches
};
struct IngestPlan {
    const IngestBatch* batches;
    const uint32_t* item_batch;  // batch of every item
    unsigned int* head;          // [0] extraction queue, [1] scatter queue
    uint32_t n_batches, n_items;
    uint64_t n_buckets;  // sum of 2^a
    uint64_t n_rel;      // sum of n_items 2^a
    int max_a;
};
size_t ingest_scatter_smem(int max_a);
// The five launches; `plan` is on the device, its arrays too.  ranged: some
// batch keeps only a hash range; all_k31: every batch has k = 31.
void launch_ingest(const IngestPlan* plan, const IngestPlan& host_plan, bool ranged, bool all_k31, int sm_count,
                   cudaStream_t st);
// Level-2 re-bucketing of level-1 groups: per-segment counts, per-(group,
// partition) offsets and totals (padded to 4), absolute run starts.
void launch_count_seg(const uint64_t* src, const SegDesc* segs, int n_segs, int a1, int a2, uint32_t* counts,
                      cudaStream_t st);
void launch_regroup_offsets(const uint32_t* counts, const uint32_t* vlo, int a1, int a2, uint64_t* rel,
                            uint32_t* total, cudaStream_t st);
void launch_regroup_base(uint64_t* rel, const uint64_t* starts, const SegDesc* segs, uint64_t n_segs, int a2,
                         cudaStream_t st);
void launch_bucket_scatter(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                           int n_ctas, const PassParams& p, int a, int mode, const uint64_t* base, uint64_t* cursor,
                           uint64_t* out, cudaStream_t st);
size_t consume_smem(int slice_log2, int table_log2, int n_samples);
void launch_fb_claim(const FallbackArgs& F, int bt, cudaStream_t st);
void launch_fb_recount(const FallbackArgs& F, int bt, cudaStream_t st);
void launch_fb_compact(const FallbackArgs& F, cudaStream_t st);
void launch_prefix_hist(const uint64_t* keys, DevCounters* ctr, uint64_t cap, int shift, uint64_t n_buckets,
                        uint32_t* hist, const Grid& g, cudaStream_t st);

// The device's opt-in shared memory per block (cached per device).
int max_optin_smem();

// Let func launch with as much dynamic shared memory as the device allows
// beside its static shared memory.  The attribute belongs to the function and
// is shared by every host thread, so it is always set to the same value, the
// maximum, never to one launch's need: jobs launching on other threads cannot
// lower it under each other.
template <typename F>
inline cudaError_t allow_max_dynamic_smem(F func) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_optin_smem() - (int)fa.sharedSizeBytes);
}

}  // namespace kc

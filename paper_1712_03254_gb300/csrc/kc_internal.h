// Host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kc_device.cuh"

namespace kc {

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
void launch_scan(const uint32_t* hist, uint64_t n, uint64_t* starts, uint64_t* cursor, cudaStream_t st);
void launch_scatter(const uint64_t* keys, const uint64_t* vals, const DevCounters* ctr, int prefix_shift,
                    uint64_t* cursor, uint64_t* out_keys, uint64_t* out_vals, const Grid& g, cudaStream_t st);
// Sort every bucket in place; buckets larger than the shared-memory tile set
// DERR_SORT_BUCKET and are left for launch_bitonic_global.
void launch_bucket_sort(uint64_t* keys, uint64_t* vals, const uint64_t* starts, uint64_t n_buckets,
                        DevCounters* ctr, cudaStream_t st);
int bucket_sort_capacity();
void launch_bitonic_global(uint64_t* keys, uint64_t* vals, uint64_t n, cudaStream_t st);

void launch_counts_narrow(const uint64_t* vals, uint64_t n, uint32_t* out, cudaStream_t st);

}  // namespace kc

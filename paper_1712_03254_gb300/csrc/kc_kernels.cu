// Kernels of the k-mer counting path and their launchers (sm_103a).
//
// Ingest      read-start bits from the offsets, then one "valid window start"
//             bit per base (no unknown base inside, window inside one read).
// Pass 1      per valid window: canonical key, mixer hash, one 64-bit atomicOr
//             on the key's filter word; the returned old word tells whether all
//             of the key's bits were set before (Section III, Prune: "seen
//             before"), and such candidates are claimed in the table.
// Pass 2      exact recount: every valid window probes the table and counts its
//             key if the key is there (Section II-B, Count unit re-reading the
//             input).
// Compaction  keys whose summed count reaches min_count (this removes the
//             filter's false positives, Section III, Unify), histogrammed by
//             their top key bits.
// Sort        bucket by top key bits, then sort each bucket in shared memory
//             (bitonic network), giving ascending keys.

#include <atomic>

#include "kc_internal.h"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t cover_pair_hi(uint64_t hi, uint64_t lo, int len) {
    // Position p (MSB first over the 128-bit pair) of the result is the OR of
    // positions p .. p+len-1 of the input; only the first 64 positions are kept.
    int c = 1;
    while (2 * c <= len) {
        const uint64_t nh = hi | (hi << c) | (lo >> (64 - c));
        const uint64_t nl = lo | (lo << c);
        hi = nh;
        lo = nl;
        c *= 2;
    }
    if (len > c) {
        const int s = len - c;
        hi = hi | (hi << s) | (lo >> (64 - s));
    }
    return hi;
}

__global__ void k_mark_read_starts(const uint64_t* __restrict__ offsets, uint64_t n_reads, uint64_t base,
                                   uint64_t n_local, unsigned long long* __restrict__ bd,
                                   DevCounters* __restrict__ ctr) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n_reads; r += stride) {
        const uint64_t o = offsets[r];
        if (r < n_reads && offsets[r + 1] < o) atomicOr(&ctr->err, DERR_OFFSETS);
        if (o < base) {
            atomicOr(&ctr->err, DERR_OFFSETS);
            continue;
        }
        const uint64_t i = o - base;
        if (i < n_local) atomicOr(bd + (i >> 6), 0x8000000000000000ull >> (i & 63));
    }
}

// Words [w_begin, w_end) of the batch's n_vwords valid-window words.
__global__ void k_build_valid(const uint64_t* __restrict__ nmask, const uint64_t* __restrict__ bd,
                              uint64_t n_vwords, uint64_t w_begin, uint64_t w_end, uint64_t start_local,
                              uint64_t n_local, int k, uint64_t* __restrict__ vout, DevCounters* __restrict__ ctr) {
    unsigned long long local = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = w_begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < w_end; w += stride) {
        const uint64_t n_hi = nmask[w], n_lo = w + 1 < n_vwords ? nmask[w + 1] : 0ull;
        uint64_t bad = cover_pair_hi(n_hi, n_lo, k);
        if (k >= 2) {
            const uint64_t b_hi = bd[w], b_lo = w + 1 < n_vwords ? bd[w + 1] : 0ull;
            // a read start at positions j+1 .. j+k-1 breaks the window at j
            const uint64_t c_hi = cover_pair_hi(b_hi, b_lo, k - 1);
            const uint64_t c_lo_first = cover_pair_hi(b_lo, 0ull, k - 1);  // position 64 of the pair
            bad |= (c_hi << 1) | (c_lo_first >> 63);
        }
        uint64_t valid = ~bad;
        const uint64_t p0 = w * 64;
        // windows must start at or after the first read's first base
        if (p0 + 64 <= start_local) valid = 0;
        else if (p0 < start_local) valid &= ~0ull >> (start_local - p0);
        // and end at or before the last read's last base
        if (n_local < (uint64_t)k || p0 > n_local - k) {
            valid = 0;
        } else {
            const uint64_t last = n_local - k - p0;  // last valid offset in this word
            if (last < 63) valid &= ~(~0ull >> (last + 1));
        }
        vout[w] = valid;
        local += __popcll(valid);
    }
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&ctr->windows, local);
}

__global__ void __launch_bounds__(256) k_pass1(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                               uint64_t n_units, PassParams p,
                                               unsigned long long* __restrict__ bloom, Slot* __restrict__ table,
                                               DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cand = 0, claimed = 0;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const UnitWords uw = load_unit(pw, vw, base + lane, n_units, lane);
        uint64_t vm = uw.v;
        // Warp-uniform trip count with a reconvergence point per window, so
        // the lanes stay together instead of splitting into sub-warps at the
        // candidate branch.
        const int n_iter = __reduce_max_sync(kFull, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = mixer64(key);
                const uint64_t pat = bloom_pattern(mixer64(h), p.n_hashes);
                const unsigned long long old = atomicOr(bloom + (h >> p.bloom_shift), (unsigned long long)pat);
                if (p.all_candidates || (old & pat) == pat) {
                    ++cand;
                    claimed += table_claim(table, p.table_mask, h >> p.table_shift, key + 1, ctr);
                }
            }
            __syncwarp();
        }
    }
    cand = warp_sum(cand);
    claimed = warp_sum(claimed);
    if (lane == 0) {
        if (cand) atomicAdd(&ctr->candidates, cand);
        if (claimed) atomicAdd(&ctr->claimed, claimed);
    }
}

__global__ void __launch_bounds__(256) k_pass2(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                               uint64_t n_units, PassParams p, Slot* __restrict__ table,
                                               DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const UnitWords uw = load_unit(pw, vw, base + lane, n_units, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(kFull, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = mixer64(key);
                table_count(table, p.table_mask, h >> p.table_shift, key + 1, p.sample, ctr);
            }
            __syncwarp();
        }
    }
}

__global__ void k_compact(const Slot* __restrict__ table, uint64_t n_slots, int n_samples, uint32_t min_count,
                          uint64_t* __restrict__ keys, uint64_t* __restrict__ vals, DevCounters* __restrict__ ctr,
                          uint32_t* __restrict__ hist, int prefix_shift) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (uint64_t base = warp * 32; base < n_slots; base += n_warps * 32) {
        const uint64_t i = base + lane;
        bool keep = false;
        ulonglong2 v = make_ulonglong2(0, 0);
        if (i < n_slots) {
            v = __ldcs(reinterpret_cast<const ulonglong2*>(table) + i);
            if (v.x != 0ull) {
                uint64_t sum = (uint32_t)v.y;
                if (n_samples == 2) sum += (uint32_t)(v.y >> 32);
                keep = sum >= min_count;
            }
        }
        const unsigned ballot = __ballot_sync(kFull, keep);
        if (ballot == 0u) continue;
        const int leader = __ffs(ballot) - 1;
        unsigned long long pos0 = 0;
        if (lane == leader) pos0 = atomicAdd(&ctr->survivors, (unsigned long long)__popc(ballot));
        pos0 = __shfl_sync(kFull, pos0, leader);
        if (keep) {
            const uint64_t pos = pos0 + __popc(ballot & lt);
            const uint64_t key = v.x - 1;
            keys[pos] = key;
            vals[pos] = v.y;
            if (hist) atomicAdd(hist + (key >> prefix_shift), 1u);
        }
    }
}

// Exclusive scan of n counters with one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(const uint32_t* __restrict__ hist, uint64_t n,
                                               uint64_t* __restrict__ starts, uint64_t* __restrict__ cursor) {
    __shared__ unsigned long long warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = (uint64_t)t * chunk, hi = lo + chunk < n ? lo + chunk : n;
    unsigned long long sum = 0;
    for (uint64_t i = lo; i < hi; ++i) sum += hist[i];
    // inclusive warp scan
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = x - sum + (wid ? warp_tot[wid - 1] : 0ull);
    for (uint64_t i = lo; i < hi; ++i) {
        starts[i] = run;
        cursor[i] = run;
        run += hist[i];
    }
    if (t == (int)blockDim.x - 1) starts[n] = warp_tot[(blockDim.x >> 5) - 1];
}

// Multi-CTA exclusive scan for long counter arrays: per-tile sums, a scan of
// the tile sums, then every tile rescanned with its offset.
constexpr int kScanTile = 4096;

__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long x, unsigned long long* total) {
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

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ hist, uint64_t n,
                                                     unsigned long long* __restrict__ tile_sums) {
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    unsigned long long x = 0;
    for (int j = 0; j < kScanTile / 1024; ++j) {
        const uint64_t i = t0 + (uint64_t)j * 1024 + threadIdx.x;
        if (i < n) x += hist[i];
    }
    unsigned long long tot;
    block_exclusive_scan(x, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long* __restrict__ tile_sums, int n_tiles) {
    // one CTA; n_tiles <= 1024 * 8
    unsigned long long x[8];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = threadIdx.x * 8 + j;
        x[j] = i < n_tiles ? tile_sums[i] : 0ull;
        sum += x[j];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan(sum, &tot);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = threadIdx.x * 8 + j;
        if (i < n_tiles) tile_sums[i] = run;
        run += x[j];
    }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const uint32_t* __restrict__ hist, uint64_t n,
                                                     const unsigned long long* __restrict__ tile_off,
                                                     uint64_t* __restrict__ starts, uint64_t* __restrict__ cursor) {
    // each thread takes 4 consecutive counters of the tile
    const uint64_t t0 = (uint64_t)blockIdx.x * kScanTile;
    const uint64_t i0 = t0 + (uint64_t)threadIdx.x * 4;
    uint32_t c[4];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = i0 + j < n ? hist[i0 + j] : 0u;
        sum += c[j];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan(sum, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) {
            starts[i0 + j] = run;
            cursor[i0 + j] = run;
        }
        run += c[j];
    }
    if (i0 < n && i0 + 4 >= n) starts[n] = run;  // the thread holding the last counter
}

__global__ void k_scatter(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                          DevCounters* __restrict__ ctr, uint64_t cap, int prefix_shift, uint64_t n_buckets,
                          unsigned long long* __restrict__ cursor, uint64_t* __restrict__ out_keys,
                          uint64_t* __restrict__ out_vals) {
    const uint64_t n = ctr->survivors < cap ? ctr->survivors : cap;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t key = keys[i];
        const uint64_t b = key >> prefix_shift;
        if (b >= n_buckets) {
            atomicOr(&ctr->err, DERR_INTERNAL);
            continue;
        }
        const uint64_t pos = atomicAdd(cursor + b, 1ull);
        if (pos >= cap) {
            atomicOr(&ctr->err, DERR_INTERNAL);
            continue;
        }
        out_keys[pos] = key;
        out_vals[pos] = vals[i];
    }
}

constexpr int kSortCap = 2048;    // keys per shared-memory tile
constexpr int kWarpSortMax = 256; // keys one warp sorts in registers
constexpr int kSortThreads = 256;

// Ascending bitonic network in the "mirror" form: every comparator puts the
// minimum at the lower index, so indices >= n behave as +infinity and need no
// padding.
__global__ void __launch_bounds__(kSortThreads) k_bucket_sort(uint64_t* __restrict__ keys,
                                                              uint64_t* __restrict__ vals,
                                                              const uint64_t* __restrict__ starts,
                                                              DevCounters* __restrict__ ctr) {
    extern __shared__ uint64_t smem[];
    uint64_t* sk = smem;
    uint64_t* sv = smem + kSortCap;
    const uint64_t lo = starts[blockIdx.x];
    const uint64_t n64 = starts[blockIdx.x + 1] - lo;
    if (n64 <= (uint64_t)kWarpSortMax) return;  // sorted by k_bucket_sort_warp
    if (n64 > (uint64_t)kSortCap) {
        if (threadIdx.x == 0) atomicOr(&ctr->err, DERR_SORT_BUCKET);
        return;
    }
    const int n = (int)n64;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sk[i] = keys[lo + i];
        sv[i] = vals[lo + i];
    }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1) {
        const int half = size >> 1;
        for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
            const int blk = i / half, off = i % half;
            const int a = blk * size + off, b = blk * size + size - 1 - off;
            if (b < n && sk[a] > sk[b]) {
                const uint64_t tk = sk[a], tv = sv[a];
                sk[a] = sk[b];
                sv[a] = sv[b];
                sk[b] = tk;
                sv[b] = tv;
            }
        }
        __syncthreads();
        for (int stride = size >> 2; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
                const int a = 2 * i - (i & (stride - 1)), b = a + stride;
                if (b < n && sk[a] > sk[b]) {
                    const uint64_t tk = sk[a], tv = sv[a];
                    sk[a] = sk[b];
                    sv[a] = sv[b];
                    sk[b] = tk;
                    sv[b] = tv;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        keys[lo + i] = sk[i];
        vals[lo + i] = sv[i];
    }
}

// shift: the keys of a bucket share their bits above `shift` (buckets are
// key-prefix ranges); buckets of up to 32 keys then sort packed.
__global__ void __launch_bounds__(256, 2) k_bucket_sort_warp(uint64_t* __restrict__ keys, uint64_t* __restrict__ vals,
                                                          const uint64_t* __restrict__ starts, uint64_t n_buckets,
                                                          int shift, DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = warp; b < n_buckets; b += n_warps) {
        const uint64_t lo = starts[b];
        const uint64_t n64 = starts[b + 1] - lo;
        if (n64 <= 1) continue;
        if (n64 > (uint64_t)kWarpSortMax) {
            if (lane == 0) atomicOr(&ctr->err, DERR_SORT_MEDIUM);
            continue;
        }
        const int n = (int)n64;
        if (n <= 32 && shift <= 59) warp_sort32_packed(keys, vals, lo, n, lane, shift);
        else if (n <= 64 && shift <= 58) warp_sort64_packed(keys, vals, lo, n, lane, shift);
        else if (n <= 32) warp_sort_bucket<1>(keys, vals, lo, n, lane);
        else if (n <= 64) warp_sort_bucket<2>(keys, vals, lo, n, lane);
        else if (n <= 128) warp_sort_bucket<4>(keys, vals, lo, n, lane);
        else warp_sort_bucket<8>(keys, vals, lo, n, lane);
    }
}

// One comparator stage of the same network over global memory.
__global__ void k_bitonic_step(uint64_t* __restrict__ keys, uint64_t* __restrict__ vals, uint64_t n,
                               uint64_t n2, uint64_t size, uint64_t stride, int mirror) {
    const uint64_t pairs = n2 >> 1;
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += gstride) {
        uint64_t a, b;
        if (mirror) {
            const uint64_t half = size >> 1, blk = i / half, off = i % half;
            a = blk * size + off;
            b = blk * size + size - 1 - off;
        } else {
            a = 2 * i - (i & (stride - 1));
            b = a + stride;
        }
        if (b < n && keys[a] > keys[b]) {
            const uint64_t tk = keys[a], tv = vals[a];
            keys[a] = keys[b];
            vals[a] = vals[b];
            keys[b] = tk;
            vals[b] = tv;
        }
    }
}

__global__ void k_counts_narrow(const uint64_t* __restrict__ vals, uint64_t n, uint32_t* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (uint32_t)vals[i];
}

unsigned grid_for(uint64_t work, int block, int max_ctas) {
    uint64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (uint64_t)max_ctas) g = (uint64_t)max_ctas;
    return (unsigned)g;
}

}  // namespace

void launch_mark_read_starts(const uint64_t* offsets, uint64_t n_reads, uint64_t base, uint64_t n_local,
                             uint64_t* bd, DevCounters* ctr, cudaStream_t st) {
    k_mark_read_starts<<<grid_for(n_reads + 1, 256, 4096), 256, 0, st>>>(
        offsets, n_reads, base, n_local, reinterpret_cast<unsigned long long*>(bd), ctr);
}

void launch_build_valid(const uint64_t* nmask, const uint64_t* bd, uint64_t n_vwords, uint64_t start_local,
                        uint64_t n_local, int k, uint64_t* vout, DevCounters* ctr, const Grid& g, cudaStream_t st) {
    launch_build_valid_range(nmask, bd, n_vwords, 0, n_vwords, start_local, n_local, k, vout, ctr, g, st);
}

void launch_build_valid_range(const uint64_t* nmask, const uint64_t* bd, uint64_t n_vwords, uint64_t w_begin,
                              uint64_t w_end, uint64_t start_local, uint64_t n_local, int k, uint64_t* vout,
                              DevCounters* ctr, const Grid& g, cudaStream_t st) {
    k_build_valid<<<grid_for(w_end - w_begin, 256, g.sm_count * 8), 256, 0, st>>>(nmask, bd, n_vwords, w_begin, w_end,
                                                                                   start_local, n_local, k, vout, ctr);
}

void launch_pass1(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, uint64_t* bloom,
                  Slot* table, DevCounters* ctr, const Grid& g, cudaStream_t st) {
    k_pass1<<<grid_for(n_units, 256, g.ctas()), 256, 0, st>>>(
        pw, vw, n_units, p, reinterpret_cast<unsigned long long*>(bloom), table, ctr);
}

void launch_pass2(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, Slot* table,
                  DevCounters* ctr, const Grid& g, cudaStream_t st) {
    k_pass2<<<grid_for(n_units, 256, g.ctas()), 256, 0, st>>>(pw, vw, n_units, p, table, ctr);
}

void launch_compact(const Slot* table, uint64_t n_slots, int n_samples, uint32_t min_count, uint64_t* keys,
                    uint64_t* vals, DevCounters* ctr, uint32_t* hist, int prefix_shift, const Grid& g,
                    cudaStream_t st) {
    k_compact<<<grid_for(n_slots, 256, g.sm_count * 8), 256, 0, st>>>(table, n_slots, n_samples, min_count, keys,
                                                                       vals, ctr, hist, prefix_shift);
}

cudaError_t launch_scan(const uint32_t* hist, uint64_t n, uint64_t* starts, uint64_t* cursor, cudaStream_t st) {
    if (n <= (uint64_t)kScanTile) {
        k_scan<<<1, 1024, 0, st>>>(hist, n, starts, cursor);
        return cudaSuccess;
    }
    const uint64_t n_tiles = (n + kScanTile - 1) / kScanTile;
    if (n_tiles > 8192) return cudaErrorInvalidValue;
    unsigned long long* tile = nullptr;
    cudaError_t e = cudaMallocAsync(&tile, n_tiles * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_scan_tiles<<<(unsigned)n_tiles, 1024, 0, st>>>(hist, n, tile);
    k_scan_top<<<1, 1024, 0, st>>>(tile, (int)n_tiles);
    k_scan_apply<<<(unsigned)n_tiles, 1024, 0, st>>>(hist, n, tile, starts, cursor);
    return cudaFreeAsync(tile, st);
}

void launch_scatter(const uint64_t* keys, const uint64_t* vals, DevCounters* ctr, uint64_t cap, int prefix_shift,
                    uint64_t n_buckets, uint64_t* cursor, uint64_t* out_keys, uint64_t* out_vals, const Grid& g,
                    cudaStream_t st) {
    k_scatter<<<g.sm_count * 8, 256, 0, st>>>(keys, vals, ctr, cap, prefix_shift, n_buckets,
                                               reinterpret_cast<unsigned long long*>(cursor), out_keys, out_vals);
}

int bucket_sort_capacity() { return kSortCap; }

void launch_bucket_sort_warp(uint64_t* keys, uint64_t* vals, const uint64_t* starts, uint64_t n_buckets, int shift,
                             DevCounters* ctr, const Grid& g, cudaStream_t st) {
    const uint64_t warps = n_buckets;
    unsigned grid = (unsigned)((warps + 7) / 8);
    const unsigned cap = (unsigned)g.sm_count * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_bucket_sort_warp<<<grid, 256, 0, st>>>(keys, vals, starts, n_buckets, shift, ctr);
}

int warp_sort_capacity() { return kWarpSortMax; }

void launch_bucket_sort(uint64_t* keys, uint64_t* vals, const uint64_t* starts, uint64_t n_buckets,
                        DevCounters* ctr, cudaStream_t st) {
    const size_t smem = 2 * sizeof(uint64_t) * kSortCap;
    static bool attr_set = false;
    if (!attr_set) {
        allow_max_dynamic_smem(k_bucket_sort);
        attr_set = true;
    }
    k_bucket_sort<<<(unsigned)n_buckets, kSortThreads, smem, st>>>(keys, vals, starts, ctr);
}

void launch_bitonic_global(uint64_t* keys, uint64_t* vals, uint64_t n, cudaStream_t st) {
    if (n <= 1) return;
    uint64_t n2 = 1;
    while (n2 < n) n2 <<= 1;
    const unsigned grid = grid_for(n2 >> 1, 256, 152 * 16);
    for (uint64_t size = 2; size <= n2; size <<= 1) {
        k_bitonic_step<<<grid, 256, 0, st>>>(keys, vals, n, n2, size, 0, 1);
        for (uint64_t stride = size >> 2; stride > 0; stride >>= 1)
            k_bitonic_step<<<grid, 256, 0, st>>>(keys, vals, n, n2, size, stride, 0);
    }
}

void launch_counts_narrow(const uint64_t* vals, uint64_t n, uint32_t* out, cudaStream_t st) {
    if (n == 0) return;
    k_counts_narrow<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(vals, n, out);
}

int max_optin_smem() {
    static std::atomic<int> cache[64];  // per device; 0 = not queried yet
    int dev = 0;
    cudaGetDevice(&dev);
    int v = dev >= 0 && dev < 64 ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (!v) {
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (dev >= 0 && dev < 64) cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

}  // namespace kc

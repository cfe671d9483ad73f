// Downstream of the count (sm_103a): the result in the paper's 16-byte k-mer
// item form, its joint count spectrum, and the Filter unit.
//
// Items     Section III-D: one k-mer item is 8 bytes of k-mer, 4 bytes holding
//           the two samples' counts and 4 bytes of padding.  Counts are kept
//           as uint32 by the library; the item stores each as 16 bits,
//           clamped to 65535.
// Spectrum  number of result keys per pair of clamped counts: the per-sample
//           imbalance summary of a joint normal/tumoral table.
// Filter    Section II-B: the Filter unit selects the k-mers whose
//           frequencies differ between the normal and the tumoral sample,
//           then reads the input again and looks every k-mer up in the table
//           to find the reads that carry selected k-mers.  Selection:
//           count[t] >= min_tumor, count[n] <= max_normal, count[t] >=
//           ratio * count[n] (the paper gives no threshold).  The selected
//           keys are compacted in key order and stored in a lookup table of
//           32-byte buckets (four keys, one sector); the rescan computes every
//           valid window's canonical key and probes the table, and a hit adds
//           one to its read's count.

#include <algorithm>
#include <cstring>

#include "kc_ctx.h"

namespace kc {
namespace {

constexpr unsigned long long kSelEmpty = ~0ull;  // keys are below 4^31: never a key
constexpr int kTileThreads = 256;
constexpr int kTileRounds = 16;
constexpr uint64_t kTileItems = (uint64_t)kTileThreads * kTileRounds;

struct SelSpec {
    int tumor;
    uint32_t min_tumor, max_normal, ratio;
};

// Packed counts: sample 0 in the low 32 bits, sample 1 in the high 32 bits.
__device__ __forceinline__ bool is_selected(uint64_t v, const SelSpec& s) {
    const uint64_t c0 = (uint32_t)v, c1 = v >> 32;
    const uint64_t t = s.tumor ? c1 : c0, n = s.tumor ? c0 : c1;
    return t >= s.min_tumor && n <= s.max_normal && t >= (uint64_t)s.ratio * n;
}

// Ordered compaction in tiles of kTileItems: the first kernel counts a tile's
// kept items, a scan gives each tile its output start, the second kernel
// writes the kept items of a tile in their input order.
struct SelectPred {
    const uint64_t* vals;
    SelSpec spec;
    __device__ bool operator()(uint64_t i) const { return is_selected(vals[i], spec); }
};

struct HitPred {
    const uint32_t* hits;
    __device__ bool operator()(uint64_t i) const { return hits[i] != 0u; }
};

template <typename Pred>
__global__ void __launch_bounds__(kTileThreads) k_tile_count(Pred pred, uint64_t n, uint32_t* __restrict__ counts) {
    const uint64_t base = (uint64_t)blockIdx.x * kTileItems;
    int total = 0;
#pragma unroll 4
    for (int r = 0; r < kTileRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kTileThreads + threadIdx.x;
        total += __syncthreads_count(i < n && pred(i));
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)total;
}

// Writer for the selection: key and packed counts.
struct SelectWrite {
    const uint64_t* keys;
    const uint64_t* vals;
    uint64_t* out_keys;
    uint64_t* out_vals;
    __device__ void operator()(uint64_t i, uint64_t pos) const {
        out_keys[pos] = keys[i];
        out_vals[pos] = vals[i];
    }
};

// Writer for candidate reads: the read's index.
struct IndexWrite {
    uint64_t* out;
    __device__ void operator()(uint64_t i, uint64_t pos) const { out[pos] = i; }
};

template <typename Pred, typename Write>
__global__ void __launch_bounds__(kTileThreads) k_tile_write(Pred pred, Write write, uint64_t n,
                                                             const uint64_t* __restrict__ starts) {
    __shared__ uint32_t warp_base[kTileThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * kTileItems;
    uint64_t out = starts[blockIdx.x];
    for (int r = 0; r < kTileRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kTileThreads + threadIdx.x;
        const bool keep = i < n && pred(i);
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_base[warp] = (uint32_t)__popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int w = 0; w < kTileThreads / 32; ++w) {
                const uint32_t c = warp_base[w];
                warp_base[w] = acc;
                acc += c;
            }
            warp_base[kTileThreads / 32] = acc;
        }
        __syncthreads();
        if (keep) write(i, out + warp_base[warp] + (uint32_t)__popc(ballot & ((1u << lane) - 1u)));
        out += warp_base[kTileThreads / 32];
        __syncthreads();  // warp_base is rewritten by the next round
    }
}

// Lookup table of the selected keys: n_buckets buckets of four keys (one
// 32-byte sector), kSelEmpty = free.  A key goes to the first free slot of
// its bucket (h >> (64 - log2 buckets)) or of the buckets after it, so slots
// of a bucket fill in order and a bucket whose last slot is free ends every
// probe sequence through it.
__global__ void k_sel_insert(const uint64_t* __restrict__ keys, uint64_t n, unsigned long long* __restrict__ table,
                             int bucket_shift, uint64_t bucket_mask, DevCounters* __restrict__ ctr) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = keys[i];
        uint64_t b = mixer64(key) >> bucket_shift;
        bool placed = false;
        for (uint64_t probe = 0; probe <= bucket_mask && !placed; ++probe) {
            for (int s = 0; s < 4 && !placed; ++s) {
                const unsigned long long prev = atomicCAS(table + 4 * b + s, kSelEmpty, key);
                placed = prev == kSelEmpty || prev == key;
            }
            b = (b + 1) & bucket_mask;
        }
        if (!placed) atomicOr(&ctr->err, DERR_INTERNAL);  // cannot happen: the table is at most half full
    }
}

__device__ __forceinline__ bool sel_contains(const unsigned long long* __restrict__ table, uint64_t b,
                                             uint64_t bucket_mask, unsigned long long key) {
    for (uint64_t probe = 0; probe <= bucket_mask; ++probe) {
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(table + 4 * b);
        const ulonglong2 a = __ldg(q), c = __ldg(q + 1);
        if (a.x == key || a.y == key || c.x == key || c.y == key) return true;
        if (c.y == kSelEmpty) return false;
        b = (b + 1) & bucket_mask;
    }
    return false;
}

// Upper bound: the read whose base range holds position pos (offsets are the
// caller's, non-decreasing, n_reads + 1 of them, offsets[0] <= pos).
__device__ __forceinline__ uint64_t read_of(const uint64_t* __restrict__ offsets, uint64_t n_reads, uint64_t pos) {
    uint64_t lo = 0, hi = n_reads;  // invariant: offsets[lo] <= pos < offsets[hi]
    while (hi - lo > 1) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (offsets[mid] <= pos) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Filter rescan: one lane per 64-base unit, as the recount pass; every valid
// window's canonical key probes the selection, and a hit adds one to its
// read.  Hits are rare, so the read lookup and the atomic add cost little.
__global__ void __launch_bounds__(256) k_filter_hits(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                                     uint64_t n_units, PassParams p, uint64_t base_pos,
                                                     const unsigned long long* __restrict__ table, int bucket_shift,
                                                     uint64_t bucket_mask, const uint64_t* __restrict__ offsets,
                                                     uint64_t n_reads, unsigned int* __restrict__ hits,
                                                     DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long found = 0;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const uint64_t u = base + lane;
        const UnitWords uw = load_unit(pw, vw, u, n_units, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(0xffffffffu, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                if (sel_contains(table, mixer64(key) >> bucket_shift, bucket_mask, key)) {
                    const uint64_t r = read_of(offsets, n_reads, base_pos + u * 64 + (uint64_t)j);
                    atomicAdd(hits + r, 1u);
                    ++found;
                }
            }
            __syncwarp();
        }
    }
    found = warp_sum(found);
    if (lane == 0 && found) atomicAdd(&ctr->candidates, found);
}

__global__ void k_items16(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals, uint64_t n,
                          int n_samples, ulonglong2* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t v = vals[i];
        const uint64_t lo = (uint32_t)v, hi = n_samples == 2 ? v >> 32 : 0ull;
        const uint64_t c0 = lo < 65535u ? lo : 65535u, c1 = hi < 65535u ? hi : 65535u;
        out[i] = make_ulonglong2(keys[i], c0 | (c1 << 16));  // padding (bytes 12..15) zero
    }
}

// Spectrum with a per-CTA shared-memory histogram (n_bins <= kSmemBins) or
// straight global atomics.
constexpr int kSmemBins = 8192;

__device__ __forceinline__ uint64_t spectrum_bin(uint64_t v, int n_samples, uint64_t cap) {
    const uint64_t lo = (uint32_t)v, hi = v >> 32;
    const uint64_t c0 = lo < cap ? lo : cap;
    if (n_samples == 1) return c0;
    return c0 * (cap + 1) + (hi < cap ? hi : cap);
}

__global__ void __launch_bounds__(256) k_spectrum(const uint64_t* __restrict__ vals, uint64_t n, int n_samples,
                                                  uint64_t cap, uint64_t n_bins,
                                                  unsigned long long* __restrict__ hist) {
    __shared__ unsigned int local[kSmemBins];
    const bool shared = n_bins <= (uint64_t)kSmemBins;
    if (shared)
        for (uint64_t b = threadIdx.x; b < n_bins; b += blockDim.x) local[b] = 0u;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t b = spectrum_bin(vals[i], n_samples, cap);
        if (shared) atomicAdd(local + b, 1u);
        else atomicAdd(hist + b, 1ull);
    }
    __syncthreads();
    if (shared)
        for (uint64_t b = threadIdx.x; b < n_bins; b += blockDim.x)
            if (local[b]) atomicAdd(hist + b, (unsigned long long)local[b]);
}

unsigned grid_of(uint64_t n, unsigned block, unsigned cap) {
    uint64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace
}  // namespace kc

namespace kcapi {

void free_selection(kc_handle h) {
    if (h->sel_keys) cudaFreeAsync(h->sel_keys, h->stream);
    if (h->sel_vals) cudaFreeAsync(h->sel_vals, h->stream);
    if (h->sel_table) cudaFreeAsync(h->sel_table, h->stream);
    h->sel_keys = h->sel_vals = h->sel_table = nullptr;
    h->n_sel = 0;
    h->sel_buckets_log2 = 0;
    h->has_selection = false;
}

namespace {

// The result on the device: a spilled result is copied back and sorted there.
kc_status device_result(kc_handle h, const char* who) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (h->state != State::Finalized) return fail(KC_ERR_STATE, std::string(who) + " before kc_finalize");
    if (!h->spilled || h->n_result == 0) return KC_OK;
    s = resort_spilled(h);
    if (s == KC_ERR_OOM_DEVICE)
        return fail(KC_ERR_OOM_DEVICE, std::string(who) + ": the spilled result does not fit on the device");
    return s;
}

// Ordered compaction of n items into the writer's arrays; *kept = how many.
template <typename Pred, typename Write>
kc_status compact_ordered(kc_handle h, Pred pred, Write write, uint64_t n, uint64_t* kept, bool do_write) {
    cudaStream_t st = h->stream;
    const uint64_t n_tiles = std::max<uint64_t>(1, (n + kc::kTileItems - 1) / kc::kTileItems);
    uint32_t* counts = nullptr;
    uint64_t *starts = nullptr, *cursor = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync(&counts, n_tiles * 4, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&starts, (n_tiles + 1) * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&cursor, n_tiles * 8, st)) != cudaSuccess) {
        if (counts) cudaFreeAsync(counts, st);
        if (starts) cudaFreeAsync(starts, st);
        return cuda_fail(e, "cudaMallocAsync(compaction tiles)");
    }
    kc::k_tile_count<Pred><<<(unsigned)n_tiles, kc::kTileThreads, 0, st>>>(pred, n, counts);
    e = kc::launch_scan(counts, n_tiles, starts, cursor, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(counts, st);
        cudaFreeAsync(starts, st);
        cudaFreeAsync(cursor, st);
        return cuda_fail(e, "tile scan");
    }
    h->launches += 2;
    if (do_write) {
        kc::k_tile_write<Pred, Write><<<(unsigned)n_tiles, kc::kTileThreads, 0, st>>>(pred, write, n, starts);
        h->launches += 1;
    }
    KC_LAUNCHED("ordered compaction launches");
    KC_CUDA(cudaMemcpyAsync(kept, starts + n_tiles, 8, cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(counts, st);
    cudaFreeAsync(starts, st);
    cudaFreeAsync(cursor, st);
    KC_CUDA(cudaStreamSynchronize(st));
    return KC_OK;
}

}  // namespace
}  // namespace kcapi

using namespace kcapi;

extern "C" {

kc_status kc_export_items(kc_handle h, kc_item16* items, uint64_t capacity, uint64_t* n_out) {
    kc_status s = device_result(h, "kc_export_items");
    if (s != KC_OK) return s;
    if (n_out) *n_out = h->n_result;
    if (!items) return KC_OK;
    if (capacity < h->n_result) return fail(KC_ERR_CAPACITY, "item capacity smaller than the result");
    const uint64_t n = h->n_result;
    if (n == 0) return KC_OK;
    cudaStream_t st = h->stream;
    const bool dev = is_device_ptr(items);
    if (dev && reinterpret_cast<uintptr_t>(items) % 16 != 0) return fail(KC_ERR_ARG, "device items must be 16-byte aligned");
    ulonglong2* out = reinterpret_cast<ulonglong2*>(items);
    if (!dev) KC_CUDA(cudaMallocAsync(&out, n * 16, st));
    kc::k_items16<<<kc::grid_of(n, 256, h->grid.sm_count * 8), 256, 0, st>>>(h->res_keys, h->res_vals, n,
                                                                             h->n_samples, out);
    h->launches += 1;
    KC_LAUNCHED("item export launch");
    if (!dev) {
        KC_CUDA(cudaMemcpyAsync(items, out, n * 16, cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(out, st);
    }
    KC_CUDA(cudaStreamSynchronize(st));
    return KC_OK;
}

kc_status kc_spectrum(kc_handle h, uint32_t cap, uint64_t* hist) {
    kc_status s = device_result(h, "kc_spectrum");
    if (s != KC_OK) return s;
    if (cap < 1 || cap > KC_SPECTRUM_MAX_CAP || !hist) return fail(KC_ERR_ARG, "spectrum cap out of range or null hist");
    const uint64_t side = (uint64_t)cap + 1;
    const uint64_t n_bins = h->n_samples == 2 ? side * side : side;
    cudaStream_t st = h->stream;
    const bool dev = is_device_ptr(hist);
    uint64_t* out = hist;
    if (!dev) KC_CUDA(cudaMallocAsync(&out, n_bins * 8, st));
    KC_CUDA(cudaMemsetAsync(out, 0, n_bins * 8, st));
    if (h->n_result) {
        kc::k_spectrum<<<kc::grid_of(h->n_result, 256, h->grid.sm_count * 2), 256, 0, st>>>(
            h->res_vals, h->n_result, h->n_samples, cap, n_bins, reinterpret_cast<unsigned long long*>(out));
        h->launches += 1;
        KC_LAUNCHED("spectrum launch");
    }
    if (!dev) {
        KC_CUDA(cudaMemcpyAsync(hist, out, n_bins * 8, cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(out, st);
    }
    KC_CUDA(cudaStreamSynchronize(st));
    return KC_OK;
}

kc_status kc_filter_select(kc_handle h, const kc_filter_spec* spec, uint64_t* n_selected) {
    kc_status s = device_result(h, "kc_filter_select");
    if (s != KC_OK) return s;
    if (h->n_samples != 2) return fail(KC_ERR_STATE, "kc_filter_select needs a two-sample (normal/tumoral) job");
    if (!spec || spec->tumor < 0 || spec->tumor > 1) return fail(KC_ERR_ARG, "filter spec: tumor must be 0 or 1");
    free_selection(h);
    cudaStream_t st = h->stream;
    const uint64_t n = h->n_result;
    kc::SelSpec ss{spec->tumor, spec->min_tumor, spec->max_normal, spec->ratio};
    kc::SelectPred pred{h->res_vals, ss};
    uint64_t kept = 0;
    cudaEvent_t t0 = phase_begin(h);
    // count first, then allocate exactly and write
    s = compact_ordered(h, pred, kc::SelectWrite{}, n, &kept, false);
    if (s != KC_OK) return s;
    const uint64_t cap = std::max<uint64_t>(1, kept);
    int lb = 8;  // buckets of four keys, at most half full
    while ((4ull << lb) < 2 * kept) ++lb;
    const uint64_t n_buckets = 1ull << lb;
    cudaError_t e;
    if ((e = cudaMallocAsync(&h->sel_keys, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&h->sel_vals, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&h->sel_table, n_buckets * 32, st)) != cudaSuccess) {
        free_selection(h);
        return cuda_fail(e, "cudaMallocAsync(selection)");
    }
    h->sel_buckets_log2 = lb;
    KC_CUDA(cudaMemsetAsync(h->sel_table, 0xff, n_buckets * 32, st));
    if (kept) {
        s = compact_ordered(h, pred, kc::SelectWrite{h->res_keys, h->res_vals, h->sel_keys, h->sel_vals}, n, &kept,
                            true);
        if (s != KC_OK) {
            free_selection(h);
            return s;
        }
        kc::k_sel_insert<<<kc::grid_of(kept, 256, h->grid.sm_count * 8), 256, 0, st>>>(
            h->sel_keys, kept, reinterpret_cast<unsigned long long*>(h->sel_table), 64 - lb, n_buckets - 1, h->ctr);
        h->launches += 1;
        KC_LAUNCHED("selection table launch");
    }
    phase_end(h, kFilterSelect, t0);
    s = read_counters(h);
    if (s != KC_OK) return s;
    phase_collect(h);
    if (h->host_ctr.err & kc::DERR_INTERNAL) {
        h->state = State::Poisoned;
        return fail(KC_ERR_INTERNAL, "selection table: no free slot");
    }
    h->n_sel = kept;
    h->has_selection = true;
    if (n_selected) *n_selected = kept;
    return KC_OK;
}

kc_status kc_filter_keys(kc_handle h, uint64_t* keys, uint32_t* counts, uint64_t capacity, uint64_t* n_out) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (!h->has_selection) return fail(KC_ERR_STATE, "kc_filter_keys before kc_filter_select");
    if (n_out) *n_out = h->n_sel;
    if (!keys) return KC_OK;
    if (capacity < h->n_sel) return fail(KC_ERR_CAPACITY, "key capacity smaller than the selection");
    if (h->n_sel == 0) return KC_OK;
    KC_CUDA(cudaMemcpyAsync(keys, h->sel_keys, h->n_sel * 8, cudaMemcpyDefault, h->stream));
    if (counts) KC_CUDA(cudaMemcpyAsync(counts, h->sel_vals, h->n_sel * 8, cudaMemcpyDefault, h->stream));
    KC_CUDA(cudaStreamSynchronize(h->stream));
    return KC_OK;
}

kc_status kc_filter_reads(kc_handle h, const uint64_t* packed_reads, const uint64_t* offsets, const uint64_t* n_mask,
                          uint64_t n_reads, uint32_t* hits, uint64_t* candidates, uint64_t* n_candidates) {
    kc_status s = check_open(h);
    if (s != KC_OK) return s;
    if (!h->has_selection) return fail(KC_ERR_STATE, "kc_filter_reads before kc_filter_select");
    if (n_candidates) *n_candidates = 0;
    if (n_reads == 0) return KC_OK;
    if (!offsets || !hits) return fail(KC_ERR_ARG, "offsets or hits is null");
    cudaStream_t st = h->stream;

    const bool off_dev = is_device_ptr(offsets);
    uint64_t b0, b1;
    if (off_dev) {
        uint64_t ends[2];
        KC_CUDA(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_reads, 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        b0 = ends[0];
        b1 = ends[1];
    } else {
        b0 = offsets[0];
        b1 = offsets[n_reads];
        for (uint64_t r = 0; r < n_reads; ++r)
            if (offsets[r + 1] < offsets[r]) return fail(KC_ERR_ARG, "read offsets decrease");
    }
    if (b1 < b0) return fail(KC_ERR_ARG, "read offsets decrease");
    if (b1 > b0 && (!packed_reads || !n_mask)) return fail(KC_ERR_ARG, "packed_reads or n_mask is null");

    const bool hits_dev = is_device_ptr(hits);
    const bool cand_dev = candidates && is_device_ptr(candidates);
    const uint64_t B = (b0 / 64) * 64;
    const uint64_t n_local = b1 - B;
    const uint64_t n_units = std::max<uint64_t>(1, (n_local + 63) / 64);
    const uint64_t n_pwords_src = (n_local + 31) / 32;
    const uint64_t n_pwords = 2 * n_units + 2;

    uint64_t *pw = nullptr, *vw = nullptr, *nm = nullptr, *bd = nullptr, *doff = nullptr, *dcand = nullptr;
    uint32_t* dhits = hits_dev ? hits : nullptr;
    kc::DevCounters* fctr = nullptr;
    auto release = [&]() {
        for (void* q : {(void*)pw, (void*)vw, (void*)nm, (void*)bd, (void*)doff, (void*)fctr})
            if (q) cudaFreeAsync(q, st);
        if (dhits && !hits_dev) cudaFreeAsync(dhits, st);
        if (dcand && !cand_dev) cudaFreeAsync(dcand, st);
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMallocAsync(&pw, n_pwords * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&vw, n_units * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&nm, n_units * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&bd, n_units * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&doff, (n_reads + 1) * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&fctr, sizeof(kc::DevCounters), st)) != cudaSuccess ||
        (!hits_dev && (e = cudaMallocAsync(&dhits, n_reads * 4, st)) != cudaSuccess) ||
        (candidates && !cand_dev && (e = cudaMallocAsync(&dcand, n_reads * 8, st)) != cudaSuccess)) {
        release();
        return cuda_fail(e, "cudaMallocAsync(filter reads)");
    }
    if (cand_dev) dcand = candidates;
    auto run = [&]() -> kc_status {
        KC_CUDA(cudaMemsetAsync(fctr, 0, sizeof(kc::DevCounters), st));
        KC_CUDA(cudaMemsetAsync(dhits, 0, n_reads * 4, st));
        KC_CUDA(cudaMemsetAsync(pw, 0, n_pwords * 8, st));
        KC_CUDA(cudaMemsetAsync(nm, 0, n_units * 8, st));
        if (n_pwords_src) KC_CUDA(cudaMemcpyAsync(pw, packed_reads + B / 32, n_pwords_src * 8, cudaMemcpyDefault, st));
        if (n_local) KC_CUDA(cudaMemcpyAsync(nm, n_mask + B / 64, ((n_local + 63) / 64) * 8, cudaMemcpyDefault, st));
        KC_CUDA(cudaMemcpyAsync(doff, offsets, (n_reads + 1) * 8, cudaMemcpyDefault, st));
        KC_CUDA(cudaMemsetAsync(bd, 0, n_units * 8, st));
        kc::launch_mark_read_starts(doff, n_reads, B, n_local, bd, fctr, st);
        kc::launch_build_valid(nm, bd, n_units, b0 - B, n_local, h->k, vw, fctr, h->grid, st);
        cudaEvent_t t0 = phase_begin(h);
        kc::k_filter_hits<<<kc::grid_of(n_units, 256, h->grid.sm_count * 8), 256, 0, st>>>(
            pw, vw, n_units, h->params(0), B, reinterpret_cast<const unsigned long long*>(h->sel_table),
            64 - h->sel_buckets_log2, (1ull << h->sel_buckets_log2) - 1, doff, n_reads, dhits, fctr);
        phase_end(h, kFilterReads, t0);
        h->launches += 3;
        KC_LAUNCHED("filter rescan launches");
        kc::DevCounters c{};
        KC_CUDA(cudaMemcpyAsync(&c, fctr, sizeof(c), cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        if (c.err & kc::DERR_OFFSETS) return fail(KC_ERR_ARG, "read offsets decrease or start before the first word");
        h->filter_windows += c.windows;
        h->filter_hits += c.candidates;
        uint64_t n_cand = 0;
        kc_status s2 = compact_ordered(h, kc::HitPred{dhits}, kc::IndexWrite{dcand}, n_reads, &n_cand,
                                       candidates != nullptr);
        if (s2 != KC_OK) return s2;
        if (!hits_dev) KC_CUDA(cudaMemcpyAsync(hits, dhits, n_reads * 4, cudaMemcpyDeviceToHost, st));
        if (candidates && !cand_dev && n_cand)
            KC_CUDA(cudaMemcpyAsync(candidates, dcand, n_cand * 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        phase_collect(h);
        if (n_candidates) *n_candidates = n_cand;
        return KC_OK;
    };
    s = run();
    if (s != KC_OK) cudaStreamSynchronize(st);  // nothing in flight may touch the caller's arrays after return
    release();
    return s;
}

}  // extern "C"

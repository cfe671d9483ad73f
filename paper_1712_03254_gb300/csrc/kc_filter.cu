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
//           keys are compacted in key order and both orientations of each are
//           stored in a lookup table of 16-byte buckets of four fingerprints;
//           the rescan rolls every valid window's forward code and probes
//           the table; hits are marked per 64-base unit and then counted per
//           read.

#include <algorithm>
#include <atomic>
#include <cstring>

#include "kc_ctx.h"

namespace kc {
namespace {

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

// Selection table.  It holds both orientations of every selected k-mer (the
// forward code of a window then finds its canonical key without the reverse
// complement): 2^lb buckets of four slots.  A slot is a 32-bit fingerprint
// (0 = free) in the bucket's 16-byte fingerprint word, with the 64-bit code
// in a parallel array, read only when a fingerprint matches; at most a
// quarter of the slots are taken.  A code goes to the first free slot of its
// bucket or of the buckets after it, so slots fill in order and a bucket
// whose last slot is free ends every probe through it.
// Hash: Fibonacci hashing, h = code * 2^64/golden ratio; bucket = top lb bits
// of h, fingerprint = the 32 bits below them with the lowest bit set.
//
// Small selections also get a prefilter that the rescan keeps in shared
// memory: kPreWords 32-bit words, each entry setting two bits of one word
// (word from the top 32 bits of h, bits from h's bits 14..18 and 20..24).  A
// window whose two bits are not both set is not in the table, and most
// windows are rejected there instead of by a random global load.
constexpr uint32_t kPreWords = 49152;                 // 192 KiB of shared memory
constexpr uint64_t kPreMaxEntries = kPreWords * 32 / 4;  // at most a quarter of its bits per entry pair

struct SelTable {
    unsigned int* fp;      // 4 per bucket
    unsigned long long* code;  // 4 per bucket
    unsigned int* pre;     // kPreWords prefilter words (null: no prefilter)
    int lb;
    uint64_t mask;         // buckets - 1
};

__device__ __forceinline__ uint64_t sel_h(uint64_t code) { return code * 0x9e3779b97f4a7c15ull; }

__device__ __forceinline__ void sel_hash(uint64_t code, int lb, uint64_t& bucket, unsigned& fp) {
    const uint64_t h = sel_h(code);
    bucket = h >> (64 - lb);
    fp = (unsigned)(h >> (32 - lb)) | 1u;  // never 0 (0 marks a free slot)
}

__device__ __forceinline__ uint32_t pre_word(uint64_t h) {
    return (uint32_t)(((h >> 32) * (uint64_t)kPreWords) >> 32);
}

__device__ __forceinline__ uint32_t pre_bits(uint64_t h) {
    return (1u << ((uint32_t)(h >> 20) & 31u)) | (1u << ((uint32_t)(h >> 14) & 31u));
}

__device__ __forceinline__ bool sel_insert(const SelTable& T, uint64_t code) {
    uint64_t b;
    unsigned fp;
    sel_hash(code, T.lb, b, fp);
    if (T.pre) {
        const uint64_t h = sel_h(code);
        atomicOr(T.pre + pre_word(h), pre_bits(h));
    }
    for (uint64_t probe = 0; probe <= T.mask; ++probe) {
        for (int s = 0; s < 4; ++s)
            if (atomicCAS(T.fp + 4 * b + s, 0u, fp) == 0u) {
                T.code[4 * b + s] = code;
                return true;
            }
        b = (b + 1) & T.mask;
    }
    return false;
}

// Both orientations of every selected canonical key.
__global__ void k_sel_insert(const uint64_t* __restrict__ keys, uint64_t n, SelTable T, PassParams p,
                             DevCounters* __restrict__ ctr) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t key = keys[i];
        const uint64_t rc = reverse_pairs(key ^ p.kmask) >> p.rc_shift;
        bool ok = sel_insert(T, key);
        if (rc != key) ok = ok && sel_insert(T, rc);  // an even-k palindrome is its own reverse complement
        if (!ok) atomicOr(&ctr->err, DERR_INTERNAL);  // cannot happen: the table is at most half full
    }
}

// Matching slots of a bucket word: confirm against the stored codes.
__device__ __forceinline__ bool sel_confirm(const SelTable& T, uint64_t b, uint4 q, unsigned fp, uint64_t code) {
    const unsigned f[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (f[s] == fp && __ldg(T.code + 4 * b + s) == code) return true;
    return false;
}

// Probe from the bucket after b on (rare: b's slots are all taken).
__device__ __forceinline__ bool sel_probe_rest(const SelTable& T, uint64_t b, unsigned fp, uint64_t code) {
    for (uint64_t probe = 0; probe < T.mask; ++probe) {
        b = (b + 1) & T.mask;
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(T.fp) + b);
        if ((q.x == fp || q.y == fp || q.z == fp || q.w == fp) && sel_confirm(T, b, q, fp, code)) return true;
        if (q.w == 0u) return false;
    }
    return false;
}

// Filter rescan: one lane per 64-base unit; the lane walks its unit's 64
// window starts with the rolling forward code and probes the selection for
// four windows at a time (four 16-byte bucket loads in flight).  PRE: one
// 1024-thread CTA per SM holds the prefilter in shared memory and loads a
// bucket only for windows that pass it.  Hits go to the unit's hit mask (bit
// 63 - j: the window starting at base j of the unit, as the valid-window
// bits), written once per unit; k_read_hits turns the masks into hits per
// read.
constexpr int kFilterThreads = 256;
constexpr int kFilterThreadsPre = 1024;

template <bool PRE>
__global__ void __launch_bounds__(PRE ? kFilterThreadsPre : kFilterThreads, PRE ? 1 : 4)
    k_filter_hits(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw, uint64_t n_units, PassParams p,
                  SelTable T, uint64_t* __restrict__ hitmask, DevCounters* __restrict__ ctr) {
    extern __shared__ uint4 s_pre4[];
    const uint32_t* s_pre = reinterpret_cast<const uint32_t*>(s_pre4);
    if (PRE) {
        const uint4* g = reinterpret_cast<const uint4*>(T.pre);
        for (uint32_t i = threadIdx.x; i < kPreWords / 4; i += blockDim.x) s_pre4[i] = __ldg(g + i);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int kk = 64 - p.rc_shift;  // 2k
    const uint4* fpw = reinterpret_cast<const uint4*>(T.fp);
    unsigned long long found = 0;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const uint64_t u = base + lane;
        const UnitWords uw = load_unit(pw, vw, u, n_units, lane);
        uint64_t vm = uw.v, hm = 0;
        // forward code of window j, and the bases entering at the next steps
        uint64_t fwd = uw.w0 >> p.rc_shift;
        uint64_t x = (uw.w0 << kk) | (uw.w1 >> p.rc_shift);
        uint64_t y = (uw.w1 << kk) | (uw.w2 >> p.rc_shift);
        for (int j0 = 0; j0 < 64 && vm; j0 += 4, vm <<= 4) {
            uint64_t code[4], b[4];
            unsigned fp[4];
            bool probe[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                code[t] = fwd;
                const uint64_t h = sel_h(fwd);
                b[t] = h >> (64 - T.lb);
                fp[t] = (unsigned)(h >> (32 - T.lb)) | 1u;
                probe[t] = (vm >> (63 - t)) & 1ull;
                if (PRE && probe[t]) {
                    const uint32_t m = pre_bits(h);
                    probe[t] = (s_pre[pre_word(h)] & m) == m;
                }
                fwd = ((fwd << 2) | (x >> 62)) & p.kmask;
                x = (x << 2) | (y >> 62);
                y <<= 2;
            }
            if (!(probe[0] || probe[1] || probe[2] || probe[3])) continue;
            uint4 q[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                q[t] = make_uint4(0u, 0u, 0u, 0u);
                if (probe[t]) q[t] = __ldg(fpw + b[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool match = q[t].x == fp[t] || q[t].y == fp[t] || q[t].z == fp[t] || q[t].w == fp[t];
                if (!match && q[t].w == 0u) continue;  // not in the table (skipped windows read as empty)
                bool hit = match && sel_confirm(T, b[t], q[t], fp[t], code[t]);
                if (!hit && q[t].w != 0u) hit = sel_probe_rest(T, b[t], fp[t], code[t]);
                if (hit) hm |= 0x8000000000000000ull >> (j0 + t);
            }
        }
        if (u < n_units) hitmask[u] = hm;
        found += __popcll(hm);
    }
    found = warp_sum(found);
    if (lane == 0 && found) atomicAdd(&ctr->candidates, found);
}

// hits[r] = hit-mask bits inside read r's bases (local positions o0 .. o1 - 1;
// the mask has bits only at valid window starts, which lie inside reads).
// Thread per read.
__global__ void k_read_hits(const uint64_t* __restrict__ offsets, uint64_t n_reads, uint64_t base,
                            uint64_t n_units, const uint64_t* __restrict__ hitmask, unsigned int* __restrict__ hits) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += stride) {
        const uint64_t o0 = offsets[r] - base, o1 = offsets[r + 1] - base;
        unsigned n = 0;
        if (o1 > o0) {
            const uint64_t u0 = o0 >> 6, u1 = (o1 - 1) >> 6;
            for (uint64_t u = u0; u <= u1 && u < n_units; ++u) {
                uint64_t m = hitmask[u];
                if (u == u0) m &= ~0ull >> (o0 & 63);                 // from base o0 on
                const int e = (int)((o1 - 1) & 63);
                if (u == u1 && e < 63) m &= ~(~0ull >> (e + 1));      // up to base o1 - 1
                n += (unsigned)__popcll(m);
            }
        }
        hits[r] = n;
    }
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

// Stem-grouped items.  A result key K = x S y (first base x, stem S of k-2
// bases, last base y) fills entry (x, y) of stem S when S is canonical (not
// above its reverse complement S'); otherwise its reverse complement
// y' S' x' (complements y', x') fills entry (y', x') of stem S'.  A stem that
// is its own reverse complement gets both entries.  One record per entry:
// key = stem << 4 | entry, value = the key's packed counts; records are
// claimed with one atomic per warp.
__global__ void k_stem_records(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals, uint64_t n,
                               int k, uint64_t* __restrict__ rec_keys, uint64_t* __restrict__ rec_vals,
                               DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const int sb = 2 * (k - 2);  // stem bits, 2..58
    const uint64_t smask = (1ull << sb) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n_round = (n + 31) & ~31ull;  // whole warps take part in every round
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t r0 = 0, r1 = 0, v = 0;
        int cnt = 0;
        if (i < n) {
            const uint64_t K = keys[i];
            v = vals[i];
            const uint64_t x = K >> (2 * k - 2), y = K & 3ull;
            const uint64_t S = (K >> 2) & smask;
            const uint64_t Sr = reverse_pairs(S ^ smask) >> (64 - sb);
            const uint64_t e_fwd = 4 * x + y, e_rev = 4 * (3 - y) + (3 - x);
            if (S < Sr) {
                r0 = (S << 4) | e_fwd;
                cnt = 1;
            } else if (S > Sr) {
                r0 = (Sr << 4) | e_rev;
                cnt = 1;
            } else {
                r0 = (S << 4) | e_fwd;
                r1 = (S << 4) | e_rev;
                cnt = e_rev == e_fwd ? 1 : 2;  // equal only for a k-mer that is its own reverse complement
            }
        }
        // warp-aggregated claim of cnt slots per lane
        unsigned incl = (unsigned)cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && total) base = atomicAdd(&ctr->survivors, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        const uint64_t pos = base + incl - cnt;
        if (cnt >= 1) {
            rec_keys[pos] = r0;
            rec_vals[pos] = v;
        }
        if (cnt == 2) {
            rec_keys[pos + 1] = r1;
            rec_vals[pos + 1] = v;
        }
    }
}

// A sorted record starts an item when its stem differs from the previous one.
struct StemStartPred {
    const uint64_t* rec_keys;
    __device__ bool operator()(uint64_t i) const { return i == 0 || (rec_keys[i] >> 4) != (rec_keys[i - 1] >> 4); }
};

// One thread per item: its records are starts[j] .. starts[j+1] - 1 (n_rec
// for the last); 72 bytes = stem, 16 counts of sample 0, 16 of sample 1, as
// nine 64-bit words (count e of a sample in bits 16 (e % 4) of word e / 4).
__global__ void k_stem_items(const uint64_t* __restrict__ rec_keys, const uint64_t* __restrict__ rec_vals,
                             uint64_t n_rec, const uint64_t* __restrict__ starts, uint64_t n_items, int n_samples,
                             uint64_t* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_items; j += stride) {
        const uint64_t s0 = starts[j], s1 = j + 1 < n_items ? starts[j + 1] : n_rec;
        uint64_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (uint64_t r = s0; r < s1; ++r) {
            const int e = (int)(rec_keys[r] & 15ull);
            const uint64_t v = rec_vals[r];
            const uint64_t lo = (uint32_t)v, hi = n_samples == 2 ? v >> 32 : 0ull;
            const uint64_t c0 = lo < 65535u ? lo : 65535u, c1 = hi < 65535u ? hi : 65535u;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((e >> 2) == q) {  // registers stay registers: the word is chosen by unrolled compares
                    w[q] |= c0 << (16 * (e & 3));
                    w[4 + q] |= c1 << (16 * (e & 3));
                }
        }
        uint64_t* o = out + 9 * j;
        o[0] = rec_keys[s0] >> 4;
#pragma unroll
        for (int q = 0; q < 8; ++q) o[1 + q] = w[q];
    }
}

unsigned grid_of(uint64_t n, unsigned block, unsigned cap) {
    uint64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Resident CTAs of k_filter_hits<false> per SM: its grid fills the SMs
// once, no partial second wave.
int filter_blocks_per_sm() {
    static std::atomic<int> cached{0};
    int v = cached.load(std::memory_order_relaxed);
    if (!v) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_filter_hits<false>, kFilterThreads, 0) !=
                cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 4;
        }
        cached.store(v, std::memory_order_relaxed);
    }
    return v;
}

// k_filter_hits<true> takes 192 KiB of dynamic shared memory (set once per
// device; the value is the same for every caller).
cudaError_t filter_pre_smem_attr() {
    static std::atomic<int> done[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    cudaError_t e = allow_max_dynamic_smem(k_filter_hits<true>);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(1, std::memory_order_relaxed);
    return e;
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
    h->sel_pre = false;
    h->has_selection = false;
}

void free_stems(kc_handle h) {
    if (h->stem_items) cudaFreeAsync(h->stem_items, h->stream);
    h->stem_items = nullptr;
    h->n_stems = 0;
    h->has_stems = false;
}

namespace {

// Bytes per selection bucket: four 32-bit fingerprints and four 64-bit codes.
constexpr uint64_t kSelBucketBytes = 16 + 32;

kc::SelTable sel_table_of(kc_handle h) {
    kc::SelTable T;
    const uint64_t n_buckets = 1ull << h->sel_buckets_log2;
    T.fp = reinterpret_cast<unsigned int*>(h->sel_table);
    T.code = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->sel_table) + 16 * n_buckets);
    T.pre = h->sel_pre ? reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(h->sel_table) +
                                                          kSelBucketBytes * n_buckets)
                       : nullptr;
    T.lb = h->sel_buckets_log2;
    T.mask = n_buckets - 1;
    return T;
}

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

// Build the stem items of the result on the device (kept until kc_reset).
static kc_status build_stems(kc_handle h) {
    cudaStream_t st = h->stream;
    const uint64_t n = h->n_result;
    const uint64_t cap = std::max<uint64_t>(1, 2 * n);
    uint64_t *rk = nullptr, *rv = nullptr, *sk = nullptr, *sv = nullptr, *starts = nullptr;
    kc::DevCounters* sctr = nullptr;
    auto release = [&]() {
        for (void* q : {(void*)rk, (void*)rv, (void*)sk, (void*)sv, (void*)starts, (void*)sctr})
            if (q) cudaFreeAsync(q, st);
    };
    cudaError_t e;
    if ((e = cudaMallocAsync(&rk, cap * 8, st)) != cudaSuccess || (e = cudaMallocAsync(&rv, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&sk, cap * 8, st)) != cudaSuccess || (e = cudaMallocAsync(&sv, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&sctr, sizeof(kc::DevCounters), st)) != cudaSuccess) {
        release();
        return cuda_fail(e, "cudaMallocAsync(stem records)");
    }
    auto run = [&]() -> kc_status {
        KC_CUDA(cudaMemsetAsync(sctr, 0, sizeof(kc::DevCounters), st));
        cudaEvent_t t0 = phase_begin(h);
        if (n)
            kc::k_stem_records<<<kc::grid_of(n, 256, h->grid.sm_count * 8), 256, 0, st>>>(
                h->res_keys, h->res_vals, n, h->k, rk, rv, sctr);
        phase_end(h, kStems, t0);
        h->launches += 1;
        KC_LAUNCHED("stem record launch");
        uint64_t n_rec = 0;
        KC_CUDA(cudaMemcpyAsync(&n_rec, &sctr->survivors, 8, cudaMemcpyDeviceToHost, st));
        KC_CUDA(cudaStreamSynchronize(st));
        if (n_rec > cap) {
            h->state = State::Poisoned;
            return fail(KC_ERR_INTERNAL, "stem records: more than two per key");
        }
        kc_status s = sort_pairs(h, rk, rv, n_rec, 2 * (h->k - 2) + 4, sctr, sk, sv, kStems);
        if (s != KC_OK) return s;
        KC_CUDA(cudaMallocAsync(&starts, std::max<uint64_t>(1, n_rec) * 8, st));
        uint64_t n_items = 0;
        t0 = phase_begin(h);
        s = compact_ordered(h, kc::StemStartPred{sk}, kc::IndexWrite{starts}, n_rec, &n_items, true);
        if (s != KC_OK) return s;
        KC_CUDA(cudaMallocAsync(&h->stem_items, std::max<uint64_t>(1, n_items) * sizeof(kc_stem_item), st));
        if (n_items)
            kc::k_stem_items<<<kc::grid_of(n_items, 256, h->grid.sm_count * 8), 256, 0, st>>>(
                sk, sv, n_rec, starts, n_items, h->n_samples, reinterpret_cast<uint64_t*>(h->stem_items));
        phase_end(h, kStems, t0);
        h->launches += 1;
        KC_LAUNCHED("stem item launch");
        KC_CUDA(cudaStreamSynchronize(st));
        phase_collect(h);
        h->n_stems = n_items;
        h->has_stems = true;
        return KC_OK;
    };
    kc_status s = run();
    if (s != KC_OK) {
        cudaStreamSynchronize(st);
        free_stems(h);
    }
    release();
    return s;
}

kc_status kc_export_stems(kc_handle h, kc_stem_item* items, uint64_t capacity, uint64_t* n_out) {
    kc_status s = device_result(h, "kc_export_stems");
    if (s != KC_OK) return s;
    if (h->k < 3) return fail(KC_ERR_STATE, "kc_export_stems needs k >= 3 (a stem is the middle k - 2 bases)");
    if (!h->has_stems && (s = build_stems(h)) != KC_OK) return s;
    if (n_out) *n_out = h->n_stems;
    if (!items) return KC_OK;
    if (capacity < h->n_stems) return fail(KC_ERR_CAPACITY, "item capacity smaller than the stem table");
    if (h->n_stems == 0) return KC_OK;
    KC_CUDA(cudaMemcpyAsync(items, h->stem_items, h->n_stems * sizeof(kc_stem_item), cudaMemcpyDefault, h->stream));
    KC_CUDA(cudaStreamSynchronize(h->stream));
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
    // buckets of four slots for both orientations of every key, at most a
    // quarter full: about 2 % of the buckets are full and make a miss probe on
    int lb = 8;
    while ((1ull << lb) < 2 * kept) ++lb;
    if (lb > 32) return fail(KC_ERR_CAPACITY, "selection larger than 2^31 keys");
    const uint64_t n_buckets = 1ull << lb;
    cudaError_t e;
    const bool pre = 2 * kept <= kc::kPreMaxEntries;
    const uint64_t table_bytes = n_buckets * kSelBucketBytes + (pre ? kc::kPreWords * 4ull : 0);
    if ((e = cudaMallocAsync(&h->sel_keys, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&h->sel_vals, cap * 8, st)) != cudaSuccess ||
        (e = cudaMallocAsync(&h->sel_table, table_bytes, st)) != cudaSuccess) {
        free_selection(h);
        return cuda_fail(e, "cudaMallocAsync(selection)");
    }
    h->sel_buckets_log2 = lb;
    h->sel_pre = pre;
    KC_CUDA(cudaMemsetAsync(h->sel_table, 0, n_buckets * 16, st));  // fingerprints: all slots free
    if (pre)
        KC_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(h->sel_table) + n_buckets * kSelBucketBytes, 0,
                                kc::kPreWords * 4ull, st));
    if (kept) {
        s = compact_ordered(h, pred, kc::SelectWrite{h->res_keys, h->res_vals, h->sel_keys, h->sel_vals}, n, &kept,
                            true);
        if (s != KC_OK) {
            free_selection(h);
            return s;
        }
        kc::k_sel_insert<<<kc::grid_of(kept, 256, h->grid.sm_count * 8), 256, 0, st>>>(
            h->sel_keys, kept, sel_table_of(h), h->params(0), h->ctr);
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
    if (n_reads >= (1ull << 32)) return fail(KC_ERR_ARG, "at most 2^32 - 1 reads per kc_filter_reads call");

    const bool hits_dev = is_device_ptr(hits);
    const bool cand_dev = candidates && is_device_ptr(candidates);
    const uint64_t B = (b0 / 64) * 64;
    const uint64_t n_local = b1 - B;
    const uint64_t n_units = std::max<uint64_t>(1, (n_local + 63) / 64);
    const uint64_t n_pwords_src = (n_local + 31) / 32;
    const uint64_t n_pwords = 2 * n_units + 2;

    uint64_t *pw = nullptr, *vw = nullptr, *nm = nullptr, *bd = nullptr, *doff = nullptr, *dcand = nullptr;
    uint32_t* dhits = hits_dev ? hits : nullptr;
    uint64_t* hitmask = nullptr;
    kc::DevCounters* fctr = nullptr;
    auto release = [&]() {
        for (void* q : {(void*)pw, (void*)vw, (void*)nm, (void*)bd, (void*)doff, (void*)fctr, (void*)hitmask})
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
        (e = cudaMallocAsync(&hitmask, n_units * 8, st)) != cudaSuccess ||
        (!hits_dev && (e = cudaMallocAsync(&dhits, n_reads * 4, st)) != cudaSuccess) ||
        (candidates && !cand_dev && (e = cudaMallocAsync(&dcand, n_reads * 8, st)) != cudaSuccess)) {
        release();
        return cuda_fail(e, "cudaMallocAsync(filter reads)");
    }
    if (cand_dev) dcand = candidates;
    auto run = [&]() -> kc_status {
        KC_CUDA(cudaMemsetAsync(fctr, 0, sizeof(kc::DevCounters), st));
        KC_CUDA(cudaMemsetAsync(pw, 0, n_pwords * 8, st));
        KC_CUDA(cudaMemsetAsync(nm, 0, n_units * 8, st));
        if (n_pwords_src) KC_CUDA(cudaMemcpyAsync(pw, packed_reads + B / 32, n_pwords_src * 8, cudaMemcpyDefault, st));
        if (n_local) KC_CUDA(cudaMemcpyAsync(nm, n_mask + B / 64, ((n_local + 63) / 64) * 8, cudaMemcpyDefault, st));
        KC_CUDA(cudaMemcpyAsync(doff, offsets, (n_reads + 1) * 8, cudaMemcpyDefault, st));
        KC_CUDA(cudaMemsetAsync(bd, 0, n_units * 8, st));
        kc::launch_mark_read_starts(doff, n_reads, B, n_local, bd, fctr, st);
        kc::launch_build_valid(nm, bd, n_units, b0 - B, n_local, h->k, vw, fctr, h->grid, st);
        const kc::SelTable T = sel_table_of(h);
        if (T.pre) {
            KC_CUDA(kc::filter_pre_smem_attr());
            const unsigned grid = kc::grid_of(n_units, kc::kFilterThreadsPre, (unsigned)h->grid.sm_count);
            cudaEvent_t t0 = phase_begin(h);
            kc::k_filter_hits<true><<<grid, kc::kFilterThreadsPre, kc::kPreWords * 4, st>>>(
                pw, vw, n_units, h->params(0), T, hitmask, fctr);
            phase_end(h, kFilterReads, t0);
        } else {
            const unsigned grid = kc::grid_of(n_units, kc::kFilterThreads,
                                              (unsigned)(h->grid.sm_count * kc::filter_blocks_per_sm()));
            cudaEvent_t t0 = phase_begin(h);
            kc::k_filter_hits<false><<<grid, kc::kFilterThreads, 0, st>>>(pw, vw, n_units, h->params(0), T,
                                                                         hitmask, fctr);
            phase_end(h, kFilterReads, t0);
        }
        kc::k_read_hits<<<kc::grid_of(n_reads, 256, h->grid.sm_count * 8), 256, 0, st>>>(doff, n_reads, B, n_units,
                                                                                         hitmask, dhits);
        h->launches += 4;
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

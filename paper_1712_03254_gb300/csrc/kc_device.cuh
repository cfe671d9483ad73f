// Device-side building blocks of the k-mer counting path (sm_103a).
//
// Reads are kept on the device as 2-bit codes, 32 bases per 64-bit word,
// first base in the most significant bits, plus one "valid window start" bit
// per base (V).  A window of k <= 31 bases starting inside a 64-base unit
// never reaches past the first word of the next unit, so a lane that owns one
// unit (two packed words, one V word) only needs the next lane's first word,
// which it gets with a warp shuffle.
#pragma once

#include <cstdint>

namespace kc {

struct __align__(16) Slot {
    unsigned long long key1;  // key + 1; 0 marks an empty slot
    unsigned int cnt[2];      // per-sample counts (cnt[1] unused with one sample)
};
static_assert(sizeof(Slot) == 16, "a table item is 8 bytes of key and 8 of counts (Section III-D)");

// Device-wide counters and error bits of one job.
struct DevCounters {
    unsigned long long windows;     // valid windows (V bits) of all batches
    unsigned long long candidates;  // windows whose filter bits were all set already
    unsigned long long claimed;     // keys inserted into the table
    unsigned long long survivors;   // keys written by the compaction
    unsigned int err;               // DERR_* bits
    unsigned int split_parts;       // partitions counted in sub-ranges
    unsigned int split_hint;        // split level the job's partitions start at
    unsigned int pad0;
    unsigned long long kept;        // windows kept by hash-range restricted extractions
    unsigned int pad[2];
};
static_assert(sizeof(DevCounters) == 64, "device counters: 64 bytes");

enum : unsigned int {
    DERR_TABLE_FULL = 1u,      // a probe sequence visited every slot
    DERR_COUNT_OVERFLOW = 2u,  // a per-sample count passed 2^32 - 1
    DERR_OFFSETS = 4u,         // decreasing read offsets
    DERR_SORT_BUCKET = 8u,     // a sort bucket exceeded the shared-memory tile
    DERR_INTERNAL = 16u,       // a self-check failed (index out of range)
    DERR_SORT_MEDIUM = 32u,    // a sort bucket exceeded one warp's registers
};

// Parameters shared by the extraction passes.
struct PassParams {
    int k;
    int rc_shift;            // 64 - 2k
    unsigned long long kmask;  // 2k low bits
    int bloom_shift;         // 64 - log2(words)
    int n_hashes;
    int table_shift;         // 64 - log2(slots)
    unsigned long long table_mask;
    int all_candidates;      // min_count <= 1: every window goes to the table
    int sample;
    // Hash range kept by the partitioned extraction: a window is kept iff
    // h_lo <= h <= h_hi (0 and ~0: every window).  It restricts a handle to the
    // keys it owns, or to one hash range of an out-of-core job at a time.
    unsigned long long h_lo, h_hi;
};

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014): golden-ratio
// increment, then two xor-shift-multiply rounds and a closing xor-shift.
__device__ __forceinline__ uint64_t mixer64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Inverse of mixer64: undo the closing xor-shift, the two multiplies (by the
// multipliers' inverses modulo 2^64) and xor-shifts, then the increment.
// x ^= x >> s is undone by x ^ (x >> s) ^ (x >> 2s) ^ ... while the shift fits.
__device__ __forceinline__ uint64_t unmixer64(uint64_t z) {
    z ^= (z >> 31) ^ (z >> 62);
    z *= 0x319642b2d24d8ec3ull;  // inverse of 0x94d049bb133111eb
    z ^= (z >> 27) ^ (z >> 54);
    z *= 0x96de1b173f119089ull;  // inverse of 0xbf58476d1ce4e5b9
    z ^= (z >> 30) ^ (z >> 60);
    return z - 0x9e3779b97f4a7c15ull;
}
static_assert(0x319642b2d24d8ec3ull * 0x94d049bb133111ebull == 1ull, "multiplier inverse");
static_assert(0x96de1b173f119089ull * 0xbf58476d1ce4e5b9ull == 1ull, "multiplier inverse");

// Reverse the order of the 32 two-bit groups of x.
__device__ __forceinline__ uint64_t reverse_pairs(uint64_t x) {
    x = __brevll(x);
    return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// Forward 2k-bit code of the window starting at base j (0..63) of a unit whose
// words are w0, w1 and the following word w2.
__device__ __forceinline__ uint64_t window_code(uint64_t w0, uint64_t w1, uint64_t w2, int j, int rc_shift) {
    const bool second = j >= 32;
    const uint64_t hi = second ? w1 : w0;
    const uint64_t lo = second ? w2 : w1;
    const int off = 2 * (j & 31);
    const uint64_t x = off ? (hi << off) | (lo >> (64 - off)) : hi;
    return x >> rc_shift;
}

// Canonical key: the smaller of the forward code and the code of the reverse
// complement (complement = code ^ 3, then reverse the base order).
__device__ __forceinline__ uint64_t canonical_key(uint64_t fwd, const PassParams& p) {
    const uint64_t rc = reverse_pairs(fwd ^ p.kmask) >> p.rc_shift;
    return fwd < rc ? fwd : rc;
}

// Rolling codes over the 64 window starts of a unit: the forward and
// reverse-complement codes of window j, updated by one base per step instead
// of being cut out of the unit's words for every window.  `x` and `y` hold the
// bases entering at the next steps (base j + k first, as the top two bits of
// x), taken from the unit's words w0, w1 and the following word w2.
struct RollingWindow {
    uint64_t fwd, rc, x, y;
};

__device__ __forceinline__ RollingWindow rolling_start(uint64_t w0, uint64_t w1, uint64_t w2, const PassParams& p) {
    RollingWindow r;
    const int kk = 64 - p.rc_shift;  // 2k, in 2..62
    r.fwd = w0 >> p.rc_shift;
    r.rc = reverse_pairs(r.fwd ^ p.kmask) >> p.rc_shift;
    r.x = (w0 << kk) | (w1 >> p.rc_shift);
    r.y = (w1 << kk) | (w2 >> p.rc_shift);
    return r;
}

// Window j -> window j + 1: the base leaving is dropped by the mask (forward)
// or shifted out (reverse complement), the entering base b adds b at the low
// end of the forward code and its complement 3 - b at the high end of the
// reverse complement.
__device__ __forceinline__ void rolling_step(RollingWindow& r, const PassParams& p) {
    const uint64_t b = r.x >> 62;
    r.fwd = ((r.fwd << 2) | b) & p.kmask;
    r.rc = (r.rc >> 2) | ((b ^ 3ull) << (62 - p.rc_shift));
    r.x = (r.x << 2) | (r.y >> 62);
    r.y <<= 2;
}

// rolling_step with k = K a compile-time constant (every shift an immediate).
template <int K>
__device__ __forceinline__ void rolling_step_k(RollingWindow& r) {
    constexpr uint64_t kmask = K >= 32 ? ~0ull : (1ull << (2 * K)) - 1ull;
    const uint64_t b = r.x >> 62;
    r.fwd = ((r.fwd << 2) | b) & kmask;
    r.rc = (r.rc >> 2) | ((b ^ 3ull) << (2 * K - 2));
    r.x = (r.x << 2) | (r.y >> 62);
    r.y <<= 2;
}

// shl.b32 clamps its shift amount at 32: x << b is 0 for b >= 32.
__device__ __forceinline__ uint32_t shl_clamped(uint32_t x, uint32_t b) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(b));
    return r;
}

// Bits of one key in its filter word: bit (g >> 6i) & 63 for i < n_hashes,
// assembled in two 32-bit halves (bit b >= 32 is bit b ^ 32 of the high half).
template <int NH>
__device__ __forceinline__ uint64_t bloom_pattern_n(uint64_t g) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        const uint32_t bit = (uint32_t)(g >> (6 * i)) & 63u;
        lo |= shl_clamped(1u, bit);
        hi |= shl_clamped(1u, bit ^ 32u);
    }
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t bloom_pattern(uint64_t g, int n_hashes) {
    uint64_t pat = 0;
#pragma unroll
    for (int i = 0; i < 10; ++i)
        if (i < n_hashes) pat |= 1ull << ((g >> (6 * i)) & 63);
    return pat;
}

// Load the unit's words; lanes of a warp hold consecutive units, so the word
// after the unit comes from the next lane (the last lane loads it itself).
// The packed buffer is padded to 2 * n_units + 2 zero-filled words, so every
// unit has both of its words and a successor word in bounds.
struct UnitWords {
    uint64_t w0, w1, w2, v;
};

// Units at or beyond u_end are inactive (zero words); the last active lane
// loads its successor word itself, since that unit may belong to another
// lane group or CTA.  All 32 lanes must call this together.
__device__ __forceinline__ UnitWords load_unit(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                               uint64_t u, uint64_t u_end, int lane) {
    UnitWords r{0, 0, 0, 0};
    const bool in = u < u_end;
    if (in) {
        r.v = __ldg(vw + u);
        const ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2*>(pw) + u);
        r.w0 = p.x;
        r.w1 = p.y;
    }
    r.w2 = __shfl_down_sync(0xffffffffu, r.w0, 1);
    if (in && (lane == 31 || u + 1 >= u_end)) r.w2 = __ldg(pw + 2 * u + 2);
    return r;
}

// Insert key (stored as key + 1) by linear probing.  Returns 1 if this call
// claimed a new slot.  A probe sequence that wraps the whole table sets
// DERR_TABLE_FULL and gives up.
__device__ __forceinline__ int table_claim(Slot* __restrict__ table, uint64_t mask, uint64_t s, uint64_t stored,
                                           DevCounters* ctr) {
    for (uint64_t i = 0; i <= mask; ++i) {
        const unsigned long long cur = __ldcg(&table[s].key1);
        if (cur == stored) return 0;
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&table[s].key1, 0ull, (unsigned long long)stored);
            if (prev == 0ull) return 1;
            if (prev == stored) return 0;
        }
        s = (s + 1) & mask;
    }
    atomicOr(&ctr->err, DERR_TABLE_FULL);
    return 0;
}

// Add one occurrence of key to its slot if the key is in the table.
__device__ __forceinline__ void table_count(Slot* __restrict__ table, uint64_t mask, uint64_t s, uint64_t stored,
                                            int sample, DevCounters* ctr) {
    for (uint64_t i = 0; i <= mask; ++i) {
        const unsigned long long cur = __ldcg(&table[s].key1);
        if (cur == stored) {
            const unsigned int old = atomicAdd(&table[s].cnt[sample], 1u);
            if (old == 0xffffffffu) atomicOr(&ctr->err, DERR_COUNT_OVERFLOW);
            return;
        }
        if (cur == 0ull) return;
        s = (s + 1) & mask;
    }
}

// Warp-per-bucket sort: the bucket's keys sit in registers, R per lane
// (element r*32 + lane), padded with ~0 keys; a bitonic network runs with
// register compare-exchanges for strides >= 32 and shuffles below.
template <int R>
__device__ __forceinline__ void warp_bitonic(uint64_t (&k)[R], uint64_t (&v)[R], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * R; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int rs = stride >> 5;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((r & rs) == 0) {  // compile-time: pairs within the lane
                        const int q = r | rs;
                        const bool asc = (((r << 5) | lane) & size) == 0;
                        const bool sw = (k[r] > k[q]) == asc;  // selects, no branch: lanes stay converged
                        const uint64_t ka = k[r], kb = k[q], va = v[r], vb = v[q];
                        k[r] = sw ? kb : ka;
                        k[q] = sw ? ka : kb;
                        v[r] = sw ? vb : va;
                        v[q] = sw ? va : vb;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = (r << 5) | lane;
                    const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[r], stride);
                    const uint64_t ov = __shfl_xor_sync(0xffffffffu, v[r], stride);
                    const bool asc = (i & size) == 0;
                    const bool lower = (i & stride) == 0;
                    // keep the smaller key when this lane's end of the pair should hold it
                    const bool want_min = lower == asc;
                    const bool take_other = want_min ? ok < k[r] : ok > k[r];
                    k[r] = take_other ? ok : k[r];
                    v[r] = take_other ? ov : v[r];
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void warp_sort_bucket(uint64_t* __restrict__ keys, uint64_t* __restrict__ vals,
                                                 uint64_t lo, int n, int lane) {
    uint64_t k[R], v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = (r << 5) | lane;
        k[r] = i < n ? keys[lo + i] : ~0ull;
        v[r] = i < n ? vals[lo + i] : 0ull;
    }
    warp_bitonic<R>(k, v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = (r << 5) | lane;
        if (i < n) {
            keys[lo + i] = k[r];
            vals[lo + i] = v[r];
        }
    }
}

// Warp sort of a bucket of n <= 32 (key, value) pairs whose keys all share
// the bits above bit `shift` (shift <= 59: the bucket is a key-prefix range),
// one pair per lane (k, v; in = lane < n).  Each lane packs its key's low
// `shift` bits with its lane index into one word, the bitonic network
// exchanges that single word (the lane index breaks ties between equal keys),
// and each value then follows its key through the lane index.  Lanes >= n
// hold ~0, which sorts last (a packed word equals ~0 only at lane 31, i.e.
// when n = 32 and no lane is empty).  On return lane i holds the i-th pair.
__device__ __forceinline__ void warp_sort32_core(uint64_t& k, uint64_t& v, bool in, int lane, int shift) {
    const uint64_t low_mask = (1ull << shift) - 1ull;
    uint64_t p = in ? (((k & low_mask) << 5) | (uint64_t)lane) : ~0ull;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, p, stride);
            const bool asc = (lane & size) == 0;
            const bool lower = (lane & stride) == 0;
            const bool take = (lower == asc) ? (o < p) : (o > p);
            p = take ? o : p;
        }
    }
    v = __shfl_sync(0xffffffffu, v, (int)(p & 31ull));
    k = (k & ~low_mask) | (p >> 5);
}

__device__ __forceinline__ void warp_sort32_packed(uint64_t* __restrict__ keys, uint64_t* __restrict__ vals,
                                                   uint64_t lo, int n, int lane, int shift) {
    const bool in = lane < n;
    uint64_t k = in ? keys[lo + lane] : 0ull;
    uint64_t v = in ? vals[lo + lane] : 0ull;
    warp_sort32_core(k, v, in, lane, shift);
    if (in) {
        keys[lo + lane] = k;
        vals[lo + lane] = v;
    }
}

// The same for 33..64 pairs (shift <= 58): two packed words per lane, element
// i = 32 r + lane in register r (k0, v0: element lane; k1, v1: element 32 +
// lane; n > 32, so lane 0 holds a key); 6 index bits.  Compare-exchanges
// across the two registers of a lane (stride 32) need no shuffle.
__device__ __forceinline__ void warp_sort64_core(uint64_t& k0, uint64_t& v0, uint64_t& k1, uint64_t& v1, bool in0,
                                                 bool in1, int lane, int shift) {
    const uint64_t low_mask = (1ull << shift) - 1ull;
    uint64_t p0 = in0 ? (((k0 & low_mask) << 6) | (uint64_t)lane) : ~0ull;
    uint64_t p1 = in1 ? (((k1 & low_mask) << 6) | (uint64_t)(32 + lane)) : ~0ull;
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride == 32) {  // size 64: element lane against element lane + 32, ascending
                const uint64_t a = p0 < p1 ? p0 : p1, b = p0 < p1 ? p1 : p0;
                p0 = a;
                p1 = b;
            } else {
                const uint64_t o0 = __shfl_xor_sync(0xffffffffu, p0, stride);
                const uint64_t o1 = __shfl_xor_sync(0xffffffffu, p1, stride);
                const bool lower = (lane & stride) == 0;
                const bool asc0 = (lane & size) == 0, asc1 = ((32 + lane) & size) == 0;
                const bool t0 = (lower == asc0) ? (o0 < p0) : (o0 > p0);
                const bool t1 = (lower == asc1) ? (o1 < p1) : (o1 > p1);
                p0 = t0 ? o0 : p0;
                p1 = t1 ? o1 : p1;
            }
        }
    }
    const int i0 = (int)(p0 & 63ull), i1 = (int)(p1 & 63ull);
    const uint64_t a0 = __shfl_sync(0xffffffffu, v0, i0 & 31), b0 = __shfl_sync(0xffffffffu, v1, i0 & 31);
    const uint64_t a1 = __shfl_sync(0xffffffffu, v0, i1 & 31), b1 = __shfl_sync(0xffffffffu, v1, i1 & 31);
    const uint64_t prefix = __shfl_sync(0xffffffffu, k0, 0) & ~low_mask;
    k0 = prefix | (p0 >> 6);
    v0 = (i0 >> 5) ? b0 : a0;
    k1 = prefix | (p1 >> 6);
    v1 = (i1 >> 5) ? b1 : a1;
}

__device__ __forceinline__ void warp_sort64_packed(uint64_t* __restrict__ keys, uint64_t* __restrict__ vals,
                                                   uint64_t lo, int n, int lane, int shift) {
    const bool in0 = lane < n, in1 = 32 + lane < n;
    uint64_t k0 = in0 ? keys[lo + lane] : 0ull, v0 = in0 ? vals[lo + lane] : 0ull;
    uint64_t k1 = in1 ? keys[lo + 32 + lane] : 0ull, v1 = in1 ? vals[lo + 32 + lane] : 0ull;
    warp_sort64_core(k0, v0, k1, v1, in0, in1, lane, shift);
    if (in0) {
        keys[lo + lane] = k0;
        vals[lo + lane] = v0;
    }
    if (in1) {
        keys[lo + 32 + lane] = k1;
        vals[lo + 32 + lane] = v1;
    }
}

constexpr int kProbeLimit = 64;  // shared-memory table probes before a partition falls back

// Shared-memory table of one partition: keys[T] hold the hashes h of the
// claimed keys themselves (h determines the key: key = unmixer64(h)), and an
// empty slot holds `empty`, a hash of another partition that no key of this
// one can equal.  Counts follow as n_samples uint32 per slot.  Returns 1 =
// claimed, 0 = present, -1 = no free slot within kProbeLimit probes; `slot`
// receives the key's slot unless -1 is returned.
__device__ __forceinline__ int smem_claim(unsigned long long* keys, uint32_t tmask, uint32_t s,
                                          unsigned long long h, unsigned long long empty, uint32_t& slot) {
    for (int i = 0; i < kProbeLimit; ++i) {
        const unsigned long long cur = keys[s];
        if (cur == h) {
            slot = s;
            return 0;
        }
        if (cur == empty) {
            const unsigned long long prev = atomicCAS(&keys[s], empty, h);
            if (prev == empty || prev == h) {
                slot = s;
                return prev == empty ? 1 : 0;
            }
        }
        s = (s + 1) & tmask;
    }
    return -1;
}

__device__ __forceinline__ int smem_find(const unsigned long long* keys, uint32_t tmask, uint32_t s,
                                         unsigned long long h, unsigned long long empty) {
    for (uint32_t i = 0; i <= tmask; ++i) {
        const unsigned long long cur = keys[s];
        if (cur == h) return (int)s;
        if (cur == empty) return -1;
        s = (s + 1) & tmask;
    }
    return -1;
}

// Filter pattern with the number of bits chosen at run time.
__device__ __forceinline__ uint64_t bloom_pattern_rt(uint64_t g, int n_hashes) {
    uint32_t lo = 0, hi = 0;
    for (int i = 0; i < n_hashes; ++i) {
        const uint32_t bit = (uint32_t)g & 63u;
        g >>= 6;
        const uint32_t m = 1u << (bit & 31u);
        if (bit & 32u) hi |= m;
        else lo |= m;
    }
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace kc

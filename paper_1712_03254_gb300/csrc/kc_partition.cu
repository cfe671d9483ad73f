// Partitioned counting path (sm_103a): hash-prefix buckets in HBM, one
// partition's filter slice and table in shared memory.
//
// The paper splits the k-mers of each chunk by the consumer thread that owns
// them with a counting-sort shuffle (histogram, prefix sum, broker copy;
// Section III-B) so that every consumer updates only its own structures
// (two-level partitioning, Section II-B).  Here the consumer is a CTA and its
// structures live in shared memory:
//
//   ingest (per kc_add_reads call)
//     k_bucket_pass<count>  per window: canonical key, h = mixer64(key),
//                           bucket = top a bits of h; per-CTA histogram in
//                           shared memory, written out CTA-major
//     k_bucket_offsets      per bucket: exclusive prefix over CTAs, totals
//     (scan)                bucket starts
//     k_bucket_base         absolute start of every (CTA, bucket) run
//     k_bucket_pass<scatter> the same windows again; each h is stored at the
//                           next position of its CTA's run of its bucket (or
//                           at a position from a global per-bucket cursor)
//   finalize (the consumer itself is k_consume_q in kc_batch.cu: one CTA per
//   partition holds the partition's filter words -- a contiguous slice, since
//   the filter word is also a prefix of h -- and an open-addressing table in
//   shared memory)
//     k_fb_*                fallback for partitions whose shared-memory table
//                           overflowed: the same steps with the partition's
//                           filter slice and a table in global memory.

#include <algorithm>

#include "kc_internal.h"

namespace kc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t warp_sum64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// L2 cache policy "evict last" for stores whose sectors are completed over
// time by later stores of the same CTA (sm_80+ createpolicy / cache_hint).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void st_u64_l2_hint(uint64_t* p, uint64_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

enum BucketMode { kCountPerCta = 0, kScatterCursor = 1, kScatterRegion = 2, kScatterStaged = 3 };

// Filler for the unused tail of a padded run: a hash whose partition prefix
// is that of the neighbouring partition, so that every reader of partition b
// (which checks the prefix) skips it.
__device__ __forceinline__ uint64_t pad_hash(uint32_t b, int a) { return (uint64_t)(b ^ 1u) << (64 - a); }

// Entries staged per bucket by the segment scatter: about 16K entries in all
// (128 KiB), never fewer than one sector's 4 per bucket.
__host__ __device__ __forceinline__ uint32_t stage_depth(int a) {
    const uint32_t d = (16384u >> a) & ~3u;
    return d < 4u ? 4u : d;
}

// kCountPerCta: per-CTA histogram of the windows' buckets in shared memory,
// written out CTA-major.  kScatterRegion: the same windows again; each CTA
// owns one run per bucket (exact offsets from the counts) and stores each h
// at the next position of its run, with an evict-last L2 policy so that the
// partly written sectors stay in L2 until later stores complete them.
// kScatterCursor: positions come from one global cursor per bucket instead.
template <int kMode>
__global__ void __launch_bounds__(512) k_bucket_pass(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                                     uint64_t n_units, uint64_t units_per_cta, PassParams p, int a,
                                                     uint32_t* __restrict__ counts,
                                                     const uint64_t* __restrict__ base,
                                                     unsigned long long* __restrict__ cursor,
                                                     uint64_t* __restrict__ out) {
    extern __shared__ uint32_t s_cnt[];
    const uint32_t P = 1u << a;
    if (kMode != kScatterCursor) {
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
    }
    const uint64_t pol = kMode == kScatterRegion ? l2_evict_last_policy() : 0ull;
    const uint64_t lo = (uint64_t)blockIdx.x * units_per_cta;
    const uint64_t hi = lo + units_per_cta < n_units ? lo + units_per_cta : n_units;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t* my_base = kMode == kScatterRegion ? base + (uint64_t)blockIdx.x * P : nullptr;
    for (uint64_t g = lo + (uint64_t)wid * 32; g < hi; g += (uint64_t)nwarps * 32) {
        const UnitWords uw = load_unit(pw, vw, g + lane, hi, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(kFull, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = mixer64(key);
                const uint32_t b = (uint32_t)(h >> (64 - a));
                if (h < p.h_lo || h > p.h_hi) {
                    // outside the kept hash range
                } else if (kMode == kScatterCursor) {
                    const unsigned long long pos = atomicAdd(cursor + b, 1ull);
                    out[pos] = h;
                } else {
                    const uint32_t r = atomicAdd(&s_cnt[b], 1u);
                    if (kMode == kScatterRegion) st_u64_l2_hint(out + __ldg(my_base + b) + r, h, pol);
                }
            }
            __syncwarp();
        }
    }
    if (kMode == kCountPerCta) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) counts[(uint64_t)blockIdx.x * P + i] = s_cnt[i];
    }
}

// Staged scatter: every CTA owns one run per partition whose start and length
// are multiples of 4 (padded counts), and stages up to 4 hashes per partition
// in shared memory; a full stage leaves as one aligned 32-byte sector, so
// DRAM only ever sees whole-sector writes.  Rounds are CTA-synchronous: each
// lane places at most one window per round, full stages are flushed after a
// barrier, and a window that found its stage full retries next round.
constexpr int kStagedThreads = 1024;

__global__ void __launch_bounds__(kStagedThreads) k_bucket_scatter_staged(
    const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw, uint64_t n_units, uint64_t units_per_cta,
    PassParams p, int a, const uint64_t* __restrict__ base, uint64_t* __restrict__ out) {
    extern __shared__ unsigned long long s_stage[];
    const uint32_t P = 1u << a;
    uint32_t* fill = reinterpret_cast<uint32_t*>(s_stage + 4 * (size_t)P);
    uint32_t* wpos = fill + P;
    __shared__ unsigned s_next;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        fill[i] = 0;
        wpos[i] = 0;
    }
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * units_per_cta;
    const uint64_t hi = lo + units_per_cta < n_units ? lo + units_per_cta : n_units;
    const uint64_t n_groups = (hi - lo + 31) / 32;
    const uint64_t* my_base = base + (uint64_t)blockIdx.x * P;
    const int lane = threadIdx.x & 31;
    UnitWords uw{0, 0, 0, 0};
    uint64_t vm = 0, ph = 0;
    uint32_t pb = 0;
    bool pend = false, warp_done = false;
    for (;;) {
        // a warp whose lanes have nothing left takes the next group of 32 units
        const bool need = __all_sync(kFull, vm == 0 && !pend);
        if (need && !warp_done) {
            unsigned g = 0;
            if (lane == 0) g = atomicAdd(&s_next, 1u);
            g = __shfl_sync(kFull, g, 0);
            if (g < n_groups) {
                uw = load_unit(pw, vw, lo + (uint64_t)g * 32 + lane, hi, lane);
                vm = uw.v;
            } else {
                warp_done = true;
            }
        }
        if (!pend && vm) {
            const int j = __clzll(vm);
            vm &= ~(0x8000000000000000ull >> j);
            const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
            ph = mixer64(key);
            pb = (uint32_t)(ph >> (64 - a));
            pend = ph >= p.h_lo && ph <= p.h_hi;  // only the kept hash range
        }
        if (pend) {
            const uint32_t pos = atomicAdd(&fill[pb], 1u);
            if (pos < 4) {
                s_stage[(size_t)pb * 4 + pos] = ph;
                pend = false;
            }
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
            if (fill[b] >= 4) {
                const ulonglong2* src = reinterpret_cast<const ulonglong2*>(s_stage + (size_t)b * 4);
                ulonglong2* dst = reinterpret_cast<ulonglong2*>(out + __ldg(my_base + b) + wpos[b]);
                dst[0] = src[0];
                dst[1] = src[1];
                wpos[b] += 4;
                fill[b] = 0;  // windows beyond the 4 staged ones retry next round
            }
        }
        if (!__syncthreads_or(!warp_done || vm != 0 || pend)) break;
    }
    // partly filled stages: pad to a whole sector
    for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
        const uint32_t f = fill[b];
        if (f) {
            uint64_t* dst = out + __ldg(my_base + b) + wpos[b];
            for (uint32_t i = 0; i < 4; ++i) dst[i] = i < f ? (uint64_t)s_stage[(size_t)b * 4 + i] : pad_hash(b, a);
        }
    }
}

// Extraction pass: every window's h is written once, CTA by CTA, into one
// contiguous segment per CTA of a linear array (warp-aggregated positions, so
// the stores are coalesced), and the CTA's histogram over partitions goes to
// counts[cta][*].  seg[cta] = {segment start, its length}.
//
// kRange: only windows with p.h_lo <= h <= p.h_hi are kept (a handle owning
// a hash range, or one range of an out-of-core job).  The CTA still reserves
// room for all its windows, but a warp claims positions step by step for the
// windows it keeps, so the segment holds the kept hashes contiguously and its
// length is set at the end; the kept total goes to ctr->kept.
constexpr int kExtractThreads = 1024;

// Units [lo, hi) by one CTA: its histogram row goes to counts[0 .. 2^a)
// (added to it with accumulate: a later piece of the same segment) and its
// segment (piece) descriptor to *seg.  K > 0: k = K known at compile time
// (every shift of the rolling codes a constant); K = 0: k from p.
template <bool kRange, int K>
__device__ __forceinline__ void extract_range(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                              uint64_t lo, uint64_t hi, const PassParams& p, int a,
                                              uint32_t* __restrict__ counts, unsigned long long* __restrict__ g_cursor,
                                              SegDesc* __restrict__ seg, uint64_t* __restrict__ lin,
                                              DevCounters* __restrict__ ctr, bool accumulate = false) {
    extern __shared__ uint32_t s_cnt[];
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_pos;
    __shared__ unsigned long long s_warp_tot[kExtractThreads / 32];
    const uint32_t P = 1u << a;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_cnt[i] = 0;
    // the CTA's window count, from the valid-window bits
    unsigned long long mine = 0;
    for (uint64_t u = lo + threadIdx.x; u < hi; u += blockDim.x) mine += __popcll(__ldg(vw + u));
    mine = warp_sum64(mine);
    if (lane == 0) s_warp_tot[wid] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < nwarps; ++w) tot += s_warp_tot[w];
        s_base = atomicAdd(g_cursor, tot);
        s_pos = 0;
        *seg = SegDesc{s_base, tot, 0ull, 0ull};
    }
    __syncthreads();
    const uint64_t base = s_base;
    const int hist_shift = 32 - a;  // a <= 20: the partition is the top a bits of h's high word
    const unsigned lt = (1u << lane) - 1u;
    for (uint64_t g = lo + (uint64_t)wid * 32; g < hi; g += (uint64_t)nwarps * 32) {
        const UnitWords uw = load_unit(pw, vw, g + lane, hi, lane);
        const uint64_t vm = uw.v;
        const unsigned nv = (unsigned)__popcll(vm);
        // the warp's windows of these 32 units get consecutive positions,
        // claimed once; each step's stores are coalesced
        const unsigned tot = __reduce_add_sync(kFull, nv);
        if (tot == 0) continue;
        unsigned wb = 0;
        if (!kRange) {
            if (lane == 0) wb = atomicAdd(&s_pos, tot);
            wb = __shfl_sync(kFull, wb, 0);
        }
        // every lane walks the 64 window starts of its unit with rolling codes
        RollingWindow rw = rolling_start(uw.w0, uw.w1, uw.w2, p);
        uint64_t vbits = vm;  // window start j's bit at the top at step j
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            bool has = (int64_t)vbits < 0;
            vbits <<= 1;
            uint64_t h = 0;
            if (has) {
                h = mixer64(rw.fwd < rw.rc ? rw.fwd : rw.rc);
                if (kRange) has = h >= p.h_lo && h <= p.h_hi;
                if (has) atomicAdd(&s_cnt[(uint32_t)(h >> 32) >> hist_shift], 1u);
            }
            const unsigned ballot = __ballot_sync(kFull, has);
            if (kRange && ballot) {  // warp-uniform: positions for this step's kept windows
                if (lane == 0) wb = atomicAdd(&s_pos, (unsigned)__popc(ballot));
                wb = __shfl_sync(kFull, wb, 0);
            }
            if (has) lin[base + wb + __popc(ballot & lt)] = h;
            if (!kRange) wb += __popc(ballot);
            if (K > 0) rolling_step_k<(K > 0 ? K : 1)>(rw);
            else rolling_step(rw, p);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) counts[i] = (accumulate ? counts[i] : 0u) + s_cnt[i];
    if (kRange && threadIdx.x == 0) {
        seg->len = s_pos;
        if (s_pos) atomicAdd(&ctr->kept, (unsigned long long)s_pos);
    }
}

template <bool kRange, int K>
__global__ void __launch_bounds__(kExtractThreads) k_extract_count(const uint64_t* __restrict__ pw,
                                                       const uint64_t* __restrict__ vw, uint64_t n_units,
                                                       uint64_t units_per_cta, PassParams p, int a,
                                                       uint32_t* __restrict__ counts,
                                                       unsigned long long* __restrict__ g_cursor,
                                                       SegDesc* __restrict__ seg, uint64_t* __restrict__ lin,
                                                       DevCounters* __restrict__ ctr, int accumulate) {
    uint64_t lo = (uint64_t)blockIdx.x * units_per_cta;
    if (lo > n_units) lo = n_units;  // a CTA past the end: an empty piece
    const uint64_t hi = lo + units_per_cta < n_units ? lo + units_per_cta : n_units;
    extract_range<kRange, K>(pw, vw, lo, hi, p, a, counts + ((uint64_t)blockIdx.x << a), g_cursor, seg + blockIdx.x, lin,
                          ctr, accumulate != 0);
}

constexpr int kLinThreads = 1024;
constexpr int kLinPerThread = 4;
constexpr uint32_t kRetryCap = 2048;  // hashes one retry list holds
constexpr uint32_t kPieceMax = 1u << 31;  // hashes a scatter loop indexes with 32 bits

// Staged scatter of hashes already in memory.  CTA c moves segment c
// (seg[c] = {offset into src, length, group}) into its padded runs, 4 hashes
// per thread per round; full 4-entry stages leave as aligned 32-byte sectors.
// A hash goes to bucket (h >> (64 - a1 - a2)) & (2^a2 - 1); with a1 > 0 the
// segment belongs to level-1 group `group`, hashes of another group (the
// level-1 run padding) are skipped, and the run padding written here carries
// the prefix of another level-2 partition.
//
// A hash whose stage is full goes to a retry list in shared memory and is
// staged again, first thing, in the next round, so the warp that held it
// takes its next rows at once (a warp loads new rows only when all its lanes
// are free, which keeps the loads coalesced).  Two lists alternate between
// rounds.  Hashes failing again go to the front of the other list (at most as
// many as the list held), new failures to its back, as long as the space the
// front may still need is left; beyond that a hash stays with its thread.
// Segment sd of src into its runs, one per bucket, starting at base[0 .. 2^a2).
// The segment may come in pieces (pieces[0], pieces[stride], ... of the same
// group), taken one after the other into the same runs.
__device__ __forceinline__ void scatter_segment(const uint64_t* __restrict__ src, const SegDesc* __restrict__ pieces,
                                                int n_pieces, size_t stride, int a1, int a2,
                                                const uint64_t* __restrict__ base, uint64_t* __restrict__ out) {
    extern __shared__ unsigned long long s_stage[];
    __shared__ unsigned s_front[2], s_back[2];  // entries at the front / back of each retry list
    const uint32_t P = 1u << a2;
    const uint32_t D = stage_depth(a2);  // entries staged per bucket, a multiple of 4
    uint32_t* fill = reinterpret_cast<uint32_t*>(s_stage + (size_t)D * P);
    uint64_t* cursor = reinterpret_cast<uint64_t*>(fill + P);  // next output position of each run
    uint64_t* retry = cursor + P;                              // two lists of kRetryCap hashes
    const uint64_t* my_base = base;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        fill[i] = 0;
        cursor[i] = __ldg(my_base + i);
    }
    if (threadIdx.x == 0) s_front[0] = s_back[0] = s_front[1] = s_back[1] = 0;
    __syncthreads();
    const uint32_t group = (uint32_t)pieces[0].group;
    // a1 + a2 <= 20: bucket and group are bits of h's high word
    const int shift = 32 - a1 - a2, gshift = 32 - a1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int par = 0;  // retry list read this round
    for (int pc = 0; pc < n_pieces; ++pc)
    for (uint64_t c0 = 0; c0 < pieces[(size_t)pc * stride].len; c0 += kPieceMax) {
        // a piece (at most kPieceMax hashes of it, 32-bit indices) ends with
        // every hash staged or flushed: the stages go on
        const SegDesc sd = pieces[(size_t)pc * stride];
        const uint64_t* __restrict__ in = src + sd.off + c0;
        const uint32_t len = (uint32_t)min(sd.len - c0, (uint64_t)kPieceMax);
        // thread t owns elements t, t + nt, t + 2 nt, ... of the segment, in order;
        // the next rows are always in flight while the current ones are staged
        uint32_t next = threadIdx.x;
        uint64_t ph[kLinPerThread], nx[kLinPerThread];
        uint32_t pend = 0;  // bit e: ph[e] still to be staged
        uint32_t nval = 0;  // bit e: nx[e] loaded, not yet taken
#pragma unroll
        for (int e = 0; e < kLinPerThread; ++e) {
            if (next < len) {
                nx[e] = __ldcg(in + next);
                nval |= 1u << e;
            }
            next += blockDim.x;
        }
        for (;;) {
            const unsigned n_front = min(s_front[par], kRetryCap), n_back = min(s_back[par], kRetryCap);
            const unsigned n_in = n_front + n_back;
            const uint64_t* rin = retry + (size_t)par * kRetryCap;
            uint64_t* rout = retry + (size_t)(par ^ 1) * kRetryCap;
            // the retry list first: a failure goes to the front of the other list
            for (unsigned i = threadIdx.x; i < n_in; i += blockDim.x) {
                const uint64_t h = rin[i < n_front ? i : kRetryCap - 1 - (i - n_front)];
                const uint32_t b = ((uint32_t)(h >> 32) >> shift) & (P - 1);
                const uint32_t pos = atomicAdd(&fill[b], 1u);
                if (pos < D) s_stage[(size_t)b * D + pos] = h;
                else rout[atomicAdd(&s_front[par ^ 1], 1u)] = h;  // at most n_in of these
            }
            // Warp-uniform: a warp takes its next rows only when none of its lanes
            // still holds a pending hash, so every load stays coalesced.
            if (__all_sync(kFull, pend == 0)) {
#pragma unroll
                for (int e = 0; e < kLinPerThread; ++e) {
                    ph[e] = nx[e];
                    if (((nval >> e) & 1u) && (a1 == 0 || ((uint32_t)(ph[e] >> 32) >> gshift) == group)) pend |= 1u << e;
                }
                nval = 0;
#pragma unroll
                for (int e = 0; e < kLinPerThread; ++e) {
                    if (next < len) {
                        nx[e] = __ldcg(in + next);
                        nval |= 1u << e;
                    }
                    // the rows after these start their way into L2 now
                    const uint32_t ahead = next + kLinPerThread * blockDim.x;
                    if (ahead < len) asm volatile("prefetch.global.L2 [%0];" ::"l"(in + ahead));
                    next += blockDim.x;
                }
            }
#pragma unroll
            for (int e = 0; e < kLinPerThread; ++e) {
                if (pend & (1u << e)) {
                    const uint64_t h = ph[e];
                    const uint32_t b = ((uint32_t)(h >> 32) >> shift) & (P - 1);
                    const uint32_t pos = atomicAdd(&fill[b], 1u);
                    if (pos < D) {
                        s_stage[(size_t)b * D + pos] = h;
                        pend &= ~(1u << e);
                    } else {
                        // the back of the other list, leaving the n_in entries the
                        // front may take; past that the hash stays and retries
                        const unsigned k = atomicAdd(&s_back[par ^ 1], 1u);
                        if (k < kRetryCap - n_in) {
                            rout[kRetryCap - 1 - k] = h;
                            pend &= ~(1u << e);
                        } else {
                            atomicSub(&s_back[par ^ 1], 1u);
                        }
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_front[par] = s_back[par] = 0;  // read by every thread above
            if (D == 4) {
                // shallow stages (many buckets): a thread per bucket, one sector
                for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
                    if (fill[b] >= 4) {
                        const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(s_stage + (size_t)b * 4);
                        ulonglong2* dst = reinterpret_cast<ulonglong2*>(out + cursor[b]);
                        dst[0] = sp[0];
                        dst[1] = sp[1];
                        cursor[b] += 4;
                        fill[b] = 0;
                    }
                }
            } else {
                // deep stages (few buckets): a warp per bucket writes its whole
                // sectors, then keeps the 0..3 entries left over at the front
                for (uint32_t b = wid; b < P; b += nwarps) {
                    const uint32_t f = min(fill[b], D);
                    const uint32_t whole = f & ~3u;
                    unsigned long long* st = s_stage + (size_t)b * D;
                    uint64_t* dst = out + cursor[b];
                    for (uint32_t i = lane * 2; i < whole; i += 64)
                        *reinterpret_cast<ulonglong2*>(dst + i) = *reinterpret_cast<const ulonglong2*>(st + i);
                    __syncwarp();
                    if (lane == 0) {
                        for (uint32_t i = whole; i < f; ++i) st[i - whole] = st[i];
                        cursor[b] += whole;
                        fill[b] = f - whole;  // hashes beyond D went to the retry list
                    }
                    __syncwarp();
                }
            }
            par ^= 1;
            if (!__syncthreads_or(pend != 0 || nval != 0 || s_front[par] != 0 || s_back[par] != 0)) break;
        }
    }
    for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
        const uint32_t f = min(fill[b], D);
        const uint32_t whole = f & ~3u;
        uint64_t* dst = out + cursor[b];
        for (uint32_t i = 0; i < whole; ++i) dst[i] = s_stage[(size_t)b * D + i];
        if (f > whole) {
            const uint64_t pad = pad_hash((group << a2) | b, a1 + a2);
            for (uint32_t i = whole; i < whole + 4; ++i) dst[i] = i < f ? (uint64_t)s_stage[(size_t)b * D + i] : pad;
        }
    }
}

// CTA c: segment c, in n_pieces pieces segs[c], segs[c + gridDim.x], ...
__global__ void __launch_bounds__(kLinThreads) k_scatter_staged_seg(const uint64_t* __restrict__ src,
                                                                    const SegDesc* __restrict__ segs, int n_pieces,
                                                                    int a1, int a2,
                                                                    const uint64_t* __restrict__ base,
                                                                    uint64_t* __restrict__ out) {
    scatter_segment(src, segs + blockIdx.x, n_pieces, gridDim.x, a1, a2, base + ((uint64_t)blockIdx.x << a2), out);
}

// Per-segment histogram over the level-2 buckets of a level-1 group's
// hashes (hashes of another group -- padding -- are skipped).
__global__ void __launch_bounds__(1024) k_count_seg(const uint64_t* __restrict__ src, const SegDesc* __restrict__ segs,
                                                    int a1, int a2, uint32_t* __restrict__ counts) {
    extern __shared__ uint32_t s_cnt[];
    const uint32_t P = 1u << a2;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const SegDesc sd = segs[blockIdx.x];
    const uint32_t group = (uint32_t)sd.group;
    const int shift = 64 - a1 - a2;
    for (uint64_t i = threadIdx.x; i < sd.len; i += blockDim.x) {
        const uint64_t h = __ldcg(src + sd.off + i);
        if ((uint32_t)(h >> (64 - a1)) == group) atomicAdd(&s_cnt[(uint32_t)(h >> shift) & (P - 1)], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) counts[(uint64_t)blockIdx.x * P + i] = s_cnt[i];
}

// Level-2 offsets: for partition (g, s), the prefix over the segments of
// group g (segments vlo[g] .. vlo[g+1]-1) of their padded counts; totals into
// the flat (g, s) order.  One thread per (g, s).
__global__ void k_regroup_offsets(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ vlo, int a1, int a2,
                                  uint64_t* __restrict__ rel, uint32_t* __restrict__ total) {
    const uint32_t P2 = 1u << a2;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ((uint64_t)1 << (a1 + a2))) return;
    const uint32_t g = (uint32_t)(t >> a2), sb = (uint32_t)(t & (P2 - 1));
    uint64_t run = 0;
    for (uint32_t v = vlo[g]; v < vlo[g + 1]; ++v) {
        uint32_t x = counts[(uint64_t)v * P2 + sb];
        x = (x + 3u) & ~3u;
        rel[(uint64_t)v * P2 + sb] = run;
        run += x;
    }
    total[t] = (uint32_t)run;
}

// rel[v][s] += starts[(group of v, s)]
__global__ void k_regroup_base(uint64_t* __restrict__ rel, const uint64_t* __restrict__ starts,
                               const SegDesc* __restrict__ segs, uint64_t n_segs, int a2) {
    const uint32_t P2 = 1u << a2;
    const uint64_t n = n_segs * P2;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t v = i >> a2;
        rel[i] += starts[((uint64_t)segs[v].group << a2) + (i & (P2 - 1))];
    }
}

// rel[c][b] = sum of counts[c'][b] over c' < c; total[b] = sum over all CTAs.
// One thread per bucket; the column is read 16 CTAs at a time so that the
// loads are independent and in flight together.
// With pad4, every count is rounded up to a multiple of 4 first.
__global__ void k_bucket_offsets(const uint32_t* __restrict__ counts, int n_ctas, uint32_t P, int pad4,
                                 uint64_t* __restrict__ rel, uint32_t* __restrict__ total) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= P) return;
    uint64_t run = 0;
    for (int c0 = 0; c0 < n_ctas; c0 += 16) {
        uint32_t x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            x[j] = c0 + j < n_ctas ? __ldg(counts + (uint64_t)(c0 + j) * P + b) : 0u;
            if (pad4) x[j] = (x[j] + 3u) & ~3u;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (c0 + j < n_ctas) rel[(uint64_t)(c0 + j) * P + b] = run;
            run += x[j];
        }
    }
    total[b] = (uint32_t)run;
}

__global__ void k_bucket_base(uint64_t* __restrict__ rel, const uint64_t* __restrict__ starts, int n_ctas,
                              uint32_t P) {
    const uint64_t n = (uint64_t)n_ctas * P;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) rel[i] += starts[i % P];
}

// ---- fallback for partitions whose shared-memory table overflowed ----------

__global__ void k_fb_claim(FallbackArgs F, int bt) {
    const uint64_t* __restrict__ d = F.data[bt];
    const uint64_t lo = F.starts[bt][F.part], hi = F.starts[bt][F.part + 1];
    const uint64_t low_mask = (1ull << (64 - F.part_bits)) - 1ull;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t cand = 0, claimed = 0;
    for (uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) {
        const uint64_t h = d[i];
        if ((uint32_t)(h >> (64 - F.part_bits)) != F.part || h < F.h_lo) continue;  // padding, done
        const uint64_t pat = bloom_pattern(mixer64(h), F.n_hashes);
        const unsigned long long old = atomicOr(F.bloom + (h >> F.bloom_shift), (unsigned long long)pat);
        if (F.all_candidates || (old & pat) == pat) {
            ++cand;
            claimed += table_claim(F.table, F.table_mask, (h & low_mask) & F.table_mask, (h & low_mask) + 1ull,
                                   F.ctr);
        }
    }
    cand = warp_sum64(cand);
    claimed = warp_sum64(claimed);
    if ((threadIdx.x & 31) == 0) {
        if (cand) atomicAdd(&F.ctr->candidates, (unsigned long long)cand);
        if (claimed) atomicAdd(&F.ctr->claimed, (unsigned long long)claimed);
    }
}

__global__ void k_fb_recount(FallbackArgs F, int bt) {
    const uint64_t* __restrict__ d = F.data[bt];
    const uint64_t lo = F.starts[bt][F.part], hi = F.starts[bt][F.part + 1];
    const uint64_t low_mask = (1ull << (64 - F.part_bits)) - 1ull;
    const int smp = F.samples[bt];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) {
        const uint64_t h = d[i];
        if ((uint32_t)(h >> (64 - F.part_bits)) != F.part || h < F.h_lo) continue;
        table_count(F.table, F.table_mask, (h & low_mask) & F.table_mask, (h & low_mask) + 1ull, smp, F.ctr);
    }
}

__global__ void k_fb_compact(FallbackArgs F) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint64_t n = F.table_mask + 1;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t hpre = (uint64_t)F.part << (64 - F.part_bits);
    for (uint64_t b0 = warp * 32; b0 < n; b0 += n_warps * 32) {
        const uint64_t i = b0 + lane;
        bool keep = false;
        ulonglong2 v = make_ulonglong2(0, 0);
        if (i < n) {
            v = *reinterpret_cast<const ulonglong2*>(F.table + i);
            if (v.x != 0ull) {
                uint64_t sum = (uint32_t)v.y;
                if (F.n_samples == 2) sum += (uint32_t)(v.y >> 32);
                keep = sum >= F.min_count;
            }
        }
        const unsigned ballot = __ballot_sync(kFull, keep);
        if (!ballot) continue;
        const int leader = __ffs(ballot) - 1;
        unsigned long long pos0 = 0;
        if (lane == leader) pos0 = atomicAdd(F.n_out, (unsigned long long)__popc(ballot));
        pos0 = __shfl_sync(kFull, pos0, leader);
        if (keep) {
            const uint64_t pos = pos0 + __popc(ballot & lt);
            if (pos < F.out_cap) {
                F.out_keys[pos] = unmixer64(hpre | (v.x - 1ull));
                F.out_vals[pos] = v.y;
            }
        }
    }
}

__global__ void k_prefix_hist(const uint64_t* __restrict__ keys, DevCounters* __restrict__ ctr, uint64_t cap,
                              int shift, uint64_t n_buckets, uint32_t* __restrict__ hist) {
    const uint64_t n = ctr->survivors < cap ? ctr->survivors : cap;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t b = keys[i] >> shift;
        if (b < n_buckets) atomicAdd(hist + b, 1u);
        else atomicOr(&ctr->err, DERR_INTERNAL);
    }
}

// ---- batched ingest: the phases over every job's batches -------------------

// Batch of (batch, bucket) index f, of (item, bucket) index r: binary search
// over the batches' first indices.
__device__ __forceinline__ uint32_t batch_of_bucket(const IngestPlan* P, uint64_t f) {
    uint32_t lo = 0, hi = P->n_batches;  // invariant: batches[lo].bucket_off <= f
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P->batches[mid].bucket_off <= f) lo = mid;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t batch_of_rel(const IngestPlan* P, uint64_t r) {
    uint32_t lo = 0, hi = P->n_batches;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P->batches[mid].rel_off <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Extraction over the item queue: each CTA takes the next item (a unit range
// of one batch) and extracts it as a CTA of k_extract_count would.
template <bool kRange, int K>
__global__ void __launch_bounds__(kExtractThreads) k_ingest_extract(const IngestPlan* __restrict__ P) {
    __shared__ unsigned s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&P->head[0], 1u);
        __syncthreads();
        const unsigned item = s_item;
        if (item >= P->n_items) break;
        const IngestBatch& B = P->batches[P->item_batch[item]];
        const uint32_t i = item - B.item0;
        const uint64_t lo = (uint64_t)i * B.upi;
        const uint64_t hi = lo + B.upi < B.n_units ? lo + B.upi : B.n_units;
        extract_range<kRange, K>(B.pw, B.vw, lo, hi, B.p, B.a, B.counts + ((uint64_t)i << B.a), B.g_cursor, B.seg + i,
                              B.lin, B.ctr);
        __syncthreads();  // the shared counters are reset by the next item
    }
}

// Per (batch, bucket): run starts of the batch's items relative to the
// bucket's start (counts padded to 4), and the bucket's total.
__global__ void k_ingest_offsets(const IngestPlan* __restrict__ P) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < P->n_buckets; f += stride) {
        const IngestBatch& B = P->batches[batch_of_bucket(P, f)];
        const uint64_t b = f - B.bucket_off;
        uint64_t run = 0;
        for (uint32_t i = 0; i < B.n_items; ++i) {
            const uint64_t r = ((uint64_t)i << B.a) + b;
            B.rel[r] = run;
            run += (B.counts[r] + 3u) & ~3u;
        }
        B.total[b] = (uint32_t)run;
    }
}

// One CTA per batch: bucket starts = exclusive scan of the totals (2^a <= 4096
// buckets, four per thread), the sum at starts[2^a].
__global__ void __launch_bounds__(1024) k_ingest_starts(const IngestPlan* __restrict__ P) {
    __shared__ unsigned long long s_w[32];
    for (uint32_t t = blockIdx.x; t < P->n_batches; t += gridDim.x) {
        const IngestBatch& B = P->batches[t];
        const uint32_t n = 1u << B.a;
        const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
        const uint32_t b0 = threadIdx.x * per;
        unsigned long long mine = 0;
        for (uint32_t k = 0; k < per; ++k)
            if (b0 + k < n) mine += B.total[b0 + k];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        unsigned long long incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const unsigned long long v = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0ull;
            unsigned long long vi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, vi, o);
                if (lane >= o) vi += y;
            }
            s_w[lane] = vi - v;
        }
        __syncthreads();
        unsigned long long run = s_w[wid] + incl - mine;
        for (uint32_t k = 0; k < per; ++k) {
            if (b0 + k < n) {
                B.starts[b0 + k] = run;
                run += B.total[b0 + k];
            }
        }
        if (b0 < n && b0 + per >= n) B.starts[n] = run;
        __syncthreads();  // s_w is reused by the next batch
    }
}

// Per (item, bucket): the run's absolute start.
__global__ void k_ingest_bases(const IngestPlan* __restrict__ P) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < P->n_rel; r += stride) {
        const IngestBatch& B = P->batches[batch_of_rel(P, r)];
        const uint64_t x = r - B.rel_off;
        B.rel[x] += B.starts[x & ((1ull << B.a) - 1ull)];
    }
}

// Staged scatter over the item queue: each CTA takes the next item's segment.
__global__ void __launch_bounds__(kLinThreads) k_ingest_scatter(const IngestPlan* __restrict__ P) {
    __shared__ unsigned s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&P->head[1], 1u);
        __syncthreads();
        const unsigned item = s_item;
        if (item >= P->n_items) break;
        const IngestBatch& B = P->batches[P->item_batch[item]];
        const uint32_t i = item - B.item0;
        scatter_segment(B.lin, B.seg + i, 1, 0, 0, B.a, B.rel + ((uint64_t)i << B.a), B.out);
        __syncthreads();  // the stages are reset by the next item
    }
}

}  // namespace

size_t bucket_pass_smem(int a) { return sizeof(uint32_t) << a; }
size_t staged_scatter_smem(int a) {
    return ((size_t)stage_depth(a) * sizeof(uint64_t) + 2 * sizeof(uint32_t)) << a;
}

void launch_bucket_count(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                         int n_ctas, const PassParams& p, int a, uint32_t* counts, cudaStream_t st) {
    const size_t smem = bucket_pass_smem(a);
    allow_max_dynamic_smem(k_bucket_pass<kCountPerCta>);
    k_bucket_pass<kCountPerCta><<<n_ctas, 512, smem, st>>>(pw, vw, n_units, units_per_cta, p, a, counts, nullptr,
                                                           nullptr, nullptr);
}

// k = 31 (the longest k, the one the paper's configurations use) gets the
// kernel with constant shifts
template <bool kRange>
static void extract_count_k(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                            int n_ctas, const PassParams& p, int a, uint32_t* counts, unsigned long long* cur,
                            SegDesc* seg, uint64_t* lin, DevCounters* ctr, cudaStream_t st, bool accumulate) {
    const size_t smem = bucket_pass_smem(a);
    if (p.k == 31) {
        allow_max_dynamic_smem(k_extract_count<kRange, 31>);
        k_extract_count<kRange, 31><<<n_ctas, kExtractThreads, smem, st>>>(pw, vw, n_units, units_per_cta, p, a,
                                                                           counts, cur, seg, lin, ctr, accumulate);
    } else {
        allow_max_dynamic_smem(k_extract_count<kRange, 0>);
        k_extract_count<kRange, 0><<<n_ctas, kExtractThreads, smem, st>>>(pw, vw, n_units, units_per_cta, p, a, counts,
                                                                          cur, seg, lin, ctr, accumulate);
    }
}

void launch_extract_count(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                          int n_ctas, const PassParams& p, int a, uint32_t* counts, uint64_t* g_cursor, SegDesc* seg,
                          uint64_t* lin, DevCounters* ctr, cudaStream_t st, bool accumulate) {
    unsigned long long* cur = reinterpret_cast<unsigned long long*>(g_cursor);
    if (p.h_lo == 0ull && p.h_hi == ~0ull)
        extract_count_k<false>(pw, vw, n_units, units_per_cta, n_ctas, p, a, counts, cur, seg, lin, ctr, st, accumulate);
    else
        extract_count_k<true>(pw, vw, n_units, units_per_cta, n_ctas, p, a, counts, cur, seg, lin, ctr, st, accumulate);
}

// stage, fill count and 64-bit output cursor per bucket, then the two retry lists
size_t staged_seg_smem(int a) {
    return (((size_t)stage_depth(a) * sizeof(uint64_t) + sizeof(uint32_t) + sizeof(uint64_t)) << a) +
           2 * kRetryCap * sizeof(uint64_t);
}

void launch_scatter_staged_seg(const uint64_t* src, const SegDesc* segs, int n_segs, int n_pieces, int a1, int a2,
                               const uint64_t* base, uint64_t* out, cudaStream_t st) {
    const size_t smem = staged_seg_smem(a2);
    allow_max_dynamic_smem(k_scatter_staged_seg);
    k_scatter_staged_seg<<<n_segs, kLinThreads, smem, st>>>(src, segs, n_pieces, a1, a2, base, out);
}

void launch_count_seg(const uint64_t* src, const SegDesc* segs, int n_segs, int a1, int a2, uint32_t* counts,
                      cudaStream_t st) {
    const size_t smem = bucket_pass_smem(a2);
    allow_max_dynamic_smem(k_count_seg);
    k_count_seg<<<n_segs, 1024, smem, st>>>(src, segs, a1, a2, counts);
}

void launch_regroup_offsets(const uint32_t* counts, const uint32_t* vlo, int a1, int a2, uint64_t* rel,
                            uint32_t* total, cudaStream_t st) {
    const uint64_t n = 1ull << (a1 + a2);
    k_regroup_offsets<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(counts, vlo, a1, a2, rel, total);
}

void launch_regroup_base(uint64_t* rel, const uint64_t* starts, const SegDesc* segs, uint64_t n_segs, int a2,
                         cudaStream_t st) {
    const uint64_t n = n_segs << a2;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_regroup_base<<<grid, 256, 0, st>>>(rel, starts, segs, n_segs, a2);
}

void launch_bucket_offsets(const uint32_t* counts, int n_ctas, int a, int pad4, uint64_t* rel, uint32_t* total,
                           cudaStream_t st) {
    const uint32_t P = 1u << a;
    k_bucket_offsets<<<(P + 63) / 64, 64, 0, st>>>(counts, n_ctas, P, pad4, rel, total);
}

void launch_bucket_base(uint64_t* rel, const uint64_t* starts, int n_ctas, int a, cudaStream_t st) {
    const uint64_t n = (uint64_t)n_ctas << a;
    unsigned grid = (unsigned)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_bucket_base<<<grid, 256, 0, st>>>(rel, starts, n_ctas, 1u << a);
}

void launch_bucket_scatter(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, uint64_t units_per_cta,
                           int n_ctas, const PassParams& p, int a, int mode, const uint64_t* base, uint64_t* cursor,
                           uint64_t* out, cudaStream_t st) {
    if (mode == kScatterStaged) {
        const size_t smem = staged_scatter_smem(a);
        allow_max_dynamic_smem(k_bucket_scatter_staged);
        k_bucket_scatter_staged<<<n_ctas, kStagedThreads, smem, st>>>(pw, vw, n_units, units_per_cta, p, a, base, out);
    } else if (mode == kScatterCursor) {
        k_bucket_pass<kScatterCursor><<<n_ctas, 512, 0, st>>>(pw, vw, n_units, units_per_cta, p, a, nullptr, nullptr,
                                                             reinterpret_cast<unsigned long long*>(cursor), out);
    } else {
        const size_t smem = bucket_pass_smem(a);
        allow_max_dynamic_smem(k_bucket_pass<kScatterRegion>);
        k_bucket_pass<kScatterRegion><<<n_ctas, 512, smem, st>>>(pw, vw, n_units, units_per_cta, p, a, nullptr, base,
                                                                 nullptr, out);
    }
}

size_t ingest_scatter_smem(int max_a) { return staged_seg_smem(max_a); }

void launch_ingest(const IngestPlan* plan, const IngestPlan& hp, bool ranged, bool all_k31, int sm_count,
                   cudaStream_t st) {
    const size_t esmem = bucket_pass_smem(hp.max_a);
    const unsigned n_ext = (unsigned)std::min<uint64_t>(hp.n_items, (uint64_t)sm_count * 2);
    const auto ext = [&](auto kern) {
        allow_max_dynamic_smem(kern);
        kern<<<n_ext, kExtractThreads, esmem, st>>>(plan);
    };
    if (ranged) {
        if (all_k31) ext(k_ingest_extract<true, 31>);
        else ext(k_ingest_extract<true, 0>);
    } else {
        if (all_k31) ext(k_ingest_extract<false, 31>);
        else ext(k_ingest_extract<false, 0>);
    }
    const auto grid_of = [&](uint64_t n) { return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, 4096)); };
    k_ingest_offsets<<<grid_of(hp.n_buckets), 256, 0, st>>>(plan);
    k_ingest_starts<<<(unsigned)std::min<uint32_t>(hp.n_batches, 1024), 1024, 0, st>>>(plan);
    k_ingest_bases<<<grid_of(hp.n_rel), 256, 0, st>>>(plan);
    const size_t ssmem = ingest_scatter_smem(hp.max_a);
    allow_max_dynamic_smem(k_ingest_scatter);
    k_ingest_scatter<<<(unsigned)std::min<uint64_t>(hp.n_items, (uint64_t)sm_count), kLinThreads, ssmem, st>>>(plan);
}

size_t consume_smem(int slice_log2, int table_log2, int n_samples) {
    return (sizeof(uint64_t) << slice_log2) + (sizeof(uint64_t) << table_log2) +
           ((sizeof(uint32_t) * (size_t)n_samples) << table_log2);
}

void launch_fb_claim(const FallbackArgs& F, int bt, cudaStream_t st) { k_fb_claim<<<1024, 256, 0, st>>>(F, bt); }
void launch_fb_recount(const FallbackArgs& F, int bt, cudaStream_t st) {
    k_fb_recount<<<1024, 256, 0, st>>>(F, bt);
}
void launch_fb_compact(const FallbackArgs& F, cudaStream_t st) { k_fb_compact<<<1024, 256, 0, st>>>(F); }

void launch_prefix_hist(const uint64_t* keys, DevCounters* ctr, uint64_t cap, int shift, uint64_t n_buckets,
                        uint32_t* hist, const Grid& g, cudaStream_t st) {
    k_prefix_hist<<<g.sm_count * 4, 256, 0, st>>>(keys, ctr, cap, shift, n_buckets, hist);
}

}  // namespace kc

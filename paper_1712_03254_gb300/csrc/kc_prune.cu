// The paper's two-filter Prune chain (Section III, Prune and Count units) on
// the direct strategy's resident reads (sm_103a).
//
// Prune  every valid window ORs its bit pattern into the first filter; a
//        window whose bits were all set already (the key was seen before, or
//        the filter answers with a false positive) ORs the same pattern into
//        the second filter, at the same word.  The second filter then holds
//        every key seen at least twice, plus some false positives.
// Count  every valid window whose key is in the second filter is claimed in
//        the table and counted there in the same step: the second filter is
//        complete before counting starts, so one pass gives exact counts, and
//        the compaction (count >= min_count) removes the false positives, as
//        the paper's Unify unit does.
// With min_count <= 1 every window is counted.

#include "kc_ctx.h"

namespace kc {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__global__ void __launch_bounds__(256) k_prune(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                               uint64_t n_units, PassParams p, unsigned long long* __restrict__ bf1,
                                               unsigned long long* __restrict__ bf2, DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long promoted = 0;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const UnitWords uw = load_unit(pw, vw, base + lane, n_units, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(kFullMask, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = mixer64(key);
                const unsigned long long pat = bloom_pattern(mixer64(h), p.n_hashes);
                const uint64_t w = h >> p.bloom_shift;
                const unsigned long long old = atomicOr(bf1 + w, pat);
                if ((old & pat) == pat) {
                    atomicOr(bf2 + w, pat);
                    ++promoted;
                }
            }
            __syncwarp();
        }
    }
    promoted = warp_sum(promoted);
    if (lane == 0 && promoted) atomicAdd(&ctr->candidates, promoted);
}

__global__ void __launch_bounds__(256) k_count_chain(const uint64_t* __restrict__ pw,
                                                     const uint64_t* __restrict__ vw, uint64_t n_units, PassParams p,
                                                     const unsigned long long* __restrict__ bf2,
                                                     Slot* __restrict__ table, DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long claimed = 0;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const UnitWords uw = load_unit(pw, vw, base + lane, n_units, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(kFullMask, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = canonical_key(window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = mixer64(key);
                const unsigned long long pat = bloom_pattern(mixer64(h), p.n_hashes);
                if (p.all_candidates || (__ldg(bf2 + (h >> p.bloom_shift)) & pat) == pat) {
                    const uint64_t home = h >> p.table_shift;
                    claimed += table_claim(table, p.table_mask, home, key + 1, ctr);
                    table_count(table, p.table_mask, home, key + 1, p.sample, ctr);
                }
            }
            __syncwarp();
        }
    }
    claimed = warp_sum(claimed);
    if (lane == 0 && claimed) atomicAdd(&ctr->claimed, claimed);
}

unsigned grid_for_units(uint64_t n_units, const Grid& g) {
    uint64_t blocks = (n_units + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > (uint64_t)g.ctas()) blocks = (uint64_t)g.ctas();
    return (unsigned)blocks;
}

}  // namespace

void launch_prune(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, uint64_t* bf1,
                  uint64_t* bf2, DevCounters* ctr, const Grid& g, cudaStream_t st) {
    k_prune<<<grid_for_units(n_units, g), 256, 0, st>>>(pw, vw, n_units, p,
                                                         reinterpret_cast<unsigned long long*>(bf1),
                                                         reinterpret_cast<unsigned long long*>(bf2), ctr);
}

void launch_count_chain(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p,
                        const uint64_t* bf2, Slot* table, DevCounters* ctr, const Grid& g, cudaStream_t st) {
    k_count_chain<<<grid_for_units(n_units, g), 256, 0, st>>>(
        pw, vw, n_units, p, reinterpret_cast<const unsigned long long*>(bf2), table, ctr);
}

}  // namespace kc

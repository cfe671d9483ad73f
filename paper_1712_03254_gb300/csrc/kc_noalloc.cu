// kc_bloom_build_noalloc: the Bloom filter of a read set, with no memory
// allocation at all.
//
// Some callers cannot allocate device memory when they want the filter: an
// application whose own allocator has already reserved the device's memory, a
// latency-critical loop that must not pay for (or synchronise on) cudaMalloc,
// or code that is only allowed to touch buffers it was handed.  For them this
// entry point works entirely in caller-provided inputs and outputs plus one
// fixed scratch array that is part of the library image.
//
// Scratch: g_noalloc_scratch, a file-scope __device__ array of
// kNoallocScratchWords 64-bit words (4 MiB + a few words), holding a padded
// copy of the packed reads, the read-start bits, the valid-window bits and the
// job counters.  Every GPU that loads the library keeps it until the process
// exits.  Every call uses the same array, so calls whose device work overlaps
// (different streams, or different host threads) race on it; the caller must
// order them.  The parts that must start at zero (read-start bits, counters)
// are cleared by each call.
//
// Host code cannot use the symbol's name as a device address: the device
// address is looked up with cudaGetSymbolAddress once per device, with that
// device current, on the first call made on that device (so that first call
// should come before any stream capture).

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/kc.h"
#include "kc_internal.h"

namespace {

constexpr uint64_t kMaxBases = KC_NOALLOC_MAX_BASES;
constexpr uint64_t kMaxUnits = kMaxBases / 64;
// packed copy (2 words per unit + 2), read-start bits, valid bits, counters
constexpr uint64_t kPackedWords = 2 * kMaxUnits + 2;
constexpr uint64_t kCounterWords = sizeof(kc::DevCounters) / 8;
constexpr uint64_t kNoallocScratchWords = kPackedWords + 2 * kMaxUnits + kCounterWords;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

kc_status noalloc_fail(kc_status s, const std::string& msg) {
    kc::set_last_error(msg);  // reported by kc_last_error()
    return s;
}

// Filter-only variant of the first counting pass: every valid window sets
// its key's bits in its filter word; nothing is claimed or counted.
__global__ void __launch_bounds__(256) k_bloom_only(const uint64_t* __restrict__ pw, const uint64_t* __restrict__ vw,
                                                    uint64_t n_units, kc::PassParams p,
                                                    unsigned long long* __restrict__ bloom) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < n_units; base += n_warps * 32) {
        const kc::UnitWords uw = kc::load_unit(pw, vw, base + lane, n_units, lane);
        uint64_t vm = uw.v;
        const int n_iter = __reduce_max_sync(0xffffffffu, (unsigned)__popcll(vm));
        for (int it = 0; it < n_iter; ++it) {
            if (vm) {
                const int j = __clzll(vm);
                vm &= ~(0x8000000000000000ull >> j);
                const uint64_t key = kc::canonical_key(kc::window_code(uw.w0, uw.w1, uw.w2, j, p.rc_shift), p);
                const uint64_t h = kc::mixer64(key);
                atomicOr(bloom + (h >> p.bloom_shift), (unsigned long long)kc::bloom_pattern(kc::mixer64(h), p.n_hashes));
            }
            __syncwarp();
        }
    }
}

// Memory this call's kernels may read and write directly: device memory of
// the current device, or managed memory.  Device memory of another GPU is
// refused (peer access may be off, and nothing here copies it first).
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch array on the current device.
kc_status scratch_address(uint64_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(KC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(KC_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return noalloc_fail(KC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<uint64_t*>(g_scratch_ptr[dev]);
    return KC_OK;
}

#define NA_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return noalloc_fail(KC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" kc_status kc_bloom_build_noalloc(int k, uint64_t bloom_bits, int n_hashes, const uint64_t* packed_reads,
                                            const uint64_t* offsets, const uint64_t* n_mask, uint64_t n_reads,
                                            uint64_t* bloom_out, void* stream) {
    kc::set_last_error("");
    if (k < 1 || k > 31) return noalloc_fail(KC_ERR_ARG, "k must be in 1..31");
    if (bloom_bits < 4096 || (bloom_bits & (bloom_bits - 1))) return noalloc_fail(KC_ERR_ARG, "bloom_bits must be a power of two >= 4096");
    if (n_hashes < 1 || n_hashes > 10) return noalloc_fail(KC_ERR_ARG, "n_hashes must be in 1..10");
    if (!bloom_out || !on_device(bloom_out))
        return noalloc_fail(KC_ERR_ARG, "bloom_out must be device memory of the current device");
    if (n_reads && (!offsets || !on_device(offsets)))
        return noalloc_fail(KC_ERR_ARG, "offsets must be device memory of the current device");
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* scratch = nullptr;
    kc_status s = scratch_address(&scratch);
    if (s != KC_OK) return s;

    NA_CUDA(cudaMemsetAsync(bloom_out, 0, bloom_bits / 8, st));
    if (n_reads == 0) return KC_OK;
    uint64_t ends[2];
    NA_CUDA(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_reads, 8, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    const uint64_t b0 = ends[0], b1 = ends[1];
    if (b1 < b0) return noalloc_fail(KC_ERR_ARG, "read offsets decrease");
    if (b1 == b0) return KC_OK;
    if (!packed_reads || !n_mask || !on_device(packed_reads) || !on_device(n_mask))
        return noalloc_fail(KC_ERR_ARG, "packed_reads and n_mask must be device memory of the current device");
    const uint64_t B = (b0 / 64) * 64;
    const uint64_t n_local = b1 - B;
    if (n_local > kMaxBases)
        return noalloc_fail(KC_ERR_CAPACITY, "read set larger than the fixed scratch (KC_NOALLOC_MAX_BASES bases)");
    const uint64_t n_units = (n_local + 63) / 64;
    const uint64_t n_pwords_src = (n_local + 31) / 32;
    uint64_t* pw = scratch;
    uint64_t* bd = scratch + kPackedWords;
    uint64_t* vw = bd + kMaxUnits;
    kc::DevCounters* ctr = reinterpret_cast<kc::DevCounters*>(vw + kMaxUnits);

    NA_CUDA(cudaMemcpyAsync(pw, packed_reads + B / 32, n_pwords_src * 8, cudaMemcpyDeviceToDevice, st));
    NA_CUDA(cudaMemsetAsync(pw + n_pwords_src, 0, (2 * n_units + 2 - n_pwords_src) * 8, st));
    NA_CUDA(cudaMemsetAsync(bd, 0, n_units * 8, st));
    NA_CUDA(cudaMemsetAsync(ctr, 0, sizeof(kc::DevCounters), st));
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    kc::Grid g;
    g.sm_count = sms > 0 ? sms : 152;
    kc::launch_mark_read_starts(offsets, n_reads, B, n_local, bd, ctr, st);
    kc::launch_build_valid(n_mask + B / 64, bd, n_units, b0 - B, n_local, k, vw, ctr, g, st);
    kc::PassParams p{};
    p.k = k;
    p.rc_shift = 64 - 2 * k;
    p.kmask = (1ull << (2 * k)) - 1ull;
    int lw = 0;
    while ((1ull << lw) < bloom_bits / 64) ++lw;
    p.bloom_shift = 64 - lw;
    p.n_hashes = n_hashes;
    uint64_t grid = (n_units + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > (uint64_t)g.sm_count * 8) grid = (uint64_t)g.sm_count * 8;
    k_bloom_only<<<(unsigned)grid, 256, 0, st>>>(pw, vw, n_units, p, reinterpret_cast<unsigned long long*>(bloom_out));
    NA_CUDA(cudaGetLastError());
    kc::DevCounters hc;
    NA_CUDA(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (hc.err & kc::DERR_OFFSETS) return noalloc_fail(KC_ERR_ARG, "read offsets decrease");
    return KC_OK;
}

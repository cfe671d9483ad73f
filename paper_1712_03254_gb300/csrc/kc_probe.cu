// kc_atomic_ceilings: measured rates of the random atomic updates the
// counting kernels are built from.
//
// The paper finds the random updates of its Bloom filters and hash tables to
// be what bounds counting (Section IV-C: the filters' random accesses, not
// bandwidth, limit the Prune-to-Unify phase).  The counting path here issues,
// per window, random 32-bit adds to shared-memory histograms (extraction and
// scatter), one random 64-bit OR into a shared-memory filter slice and one
// random 32-bit add into a shared-memory count table (the partition consumer),
// or, in the direct strategy, one random 64-bit OR into the filter in global
// memory.  Each probe below issues one kind of update at random addresses, as
// fast as the GPU takes them, and reports updates per second:
//
//   smem_or64   64-bit atomicOr into a 4096-word shared array per CTA
//   smem_add32  32-bit atomicAdd into 4096 shared counters per CTA
//   l2_or64     64-bit atomicOr into a 16 MiB global array (held in L2)
//   hbm_or64    64-bit atomicOr into a 4 GiB global array (beyond L2)
//
// Addresses come from a per-thread xorshift generator; each thread keeps
// several updates in flight.  Every kernel runs a fixed number of iterations
// and has no waits.

#include <cuda_runtime.h>

#include <string>

#include "../../include/kc.h"
#include "kc_internal.h"

namespace {

constexpr int kSmemWords = 4096;
constexpr int kProbeThreads = 512;
constexpr int kInFlight = 4;

__device__ __forceinline__ uint64_t xorshift(uint64_t& x) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return x;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_smem_or64(int iters, unsigned long long* sink) {
    __shared__ unsigned long long s[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) s[i] = 0ull;
    __syncthreads();
    uint64_t x = 0x9e3779b97f4a7c15ull * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) {
            const uint64_t r = xorshift(x);
            atomicOr(&s[(uint32_t)r & (kSmemWords - 1)], 1ull << (r >> 58));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicXor(sink, s[blockIdx.x & (kSmemWords - 1)]);
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_smem_add32(int iters, unsigned long long* sink) {
    __shared__ unsigned int s[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) s[i] = 0u;
    __syncthreads();
    uint64_t x = 0x9e3779b97f4a7c15ull * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) {
            const uint64_t r = xorshift(x);
            atomicAdd(&s[(uint32_t)r & (kSmemWords - 1)], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicXor(sink, (unsigned long long)s[blockIdx.x & (kSmemWords - 1)]);
}

// words: a power of two; every address is inside [0, words)
__global__ void __launch_bounds__(kProbeThreads) k_probe_global_or64(unsigned long long* a, uint64_t words, int iters) {
    uint64_t x = 0x9e3779b97f4a7c15ull * (blockIdx.x * blockDim.x + threadIdx.x + 1);
    const uint64_t mask = words - 1;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kInFlight; ++j) {
            const uint64_t r = xorshift(x);
            atomicOr(&a[r & mask], 1ull << (r >> 58));
        }
    }
}

kc_status probe_fail(kc_status s, const std::string& msg) {
    kc::set_last_error(msg);
    return s;
}

#define PR_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            cleanup();                                                                                 \
            return probe_fail(e_ == cudaErrorMemoryAllocation ? KC_ERR_OOM_DEVICE : KC_ERR_CUDA,       \
                              std::string(#call ": ") + cudaGetErrorString(e_));                       \
        }                                                                                              \
    } while (0)

}  // namespace

extern "C" kc_status kc_atomic_ceilings(kc_atomic_rates* out, void* stream) {
    kc::set_last_error("");
    if (!out) return probe_fail(KC_ERR_ARG, "out is null");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    unsigned long long *sink = nullptr, *l2 = nullptr, *hbm = nullptr;
    auto cleanup = [&]() {
        if (st) cudaStreamSynchronize(st);
        else cudaDeviceSynchronize();
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
        if (sink) cudaFree(sink);
        if (l2) cudaFree(l2);
        if (hbm) cudaFree(hbm);
    };
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    const uint64_t l2_words = (16ull << 20) / 8, hbm_words = (4ull << 30) / 8;
    cudaError_t me = cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(kc::sync_api_mutex());
        if ((me = cudaMalloc(&sink, 8)) == cudaSuccess && (me = cudaMalloc(&l2, l2_words * 8)) == cudaSuccess)
            me = cudaMalloc(&hbm, hbm_words * 8);
    }
    PR_CUDA(me);  // after the lock: cleanup takes it again
    PR_CUDA(cudaMemsetAsync(l2, 0, l2_words * 8, st));
    PR_CUDA(cudaMemsetAsync(hbm, 0, hbm_words * 8, st));
    // timed launch after one warm-up launch; updates per second
    auto time_it = [&](auto launch, double updates, double* rate) -> cudaError_t {
        launch();
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return e;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return e;
        *rate = ms > 0.f ? updates / (ms * 1e-3) : 0.0;
        return cudaSuccess;
    };
    const int smem_ctas = sms * 4, smem_iters = 4096;
    const double smem_updates = (double)smem_ctas * kProbeThreads * smem_iters * kInFlight;
    PR_CUDA(time_it([&] { k_probe_smem_or64<<<smem_ctas, kProbeThreads, 0, st>>>(smem_iters, sink); }, smem_updates,
                    &out->smem_or64_per_s));
    PR_CUDA(time_it([&] { k_probe_smem_add32<<<smem_ctas, kProbeThreads, 0, st>>>(smem_iters, sink); },
                    smem_updates, &out->smem_add32_per_s));
    const int g_ctas = sms * 4, g_iters = 256;
    const double g_updates = (double)g_ctas * kProbeThreads * g_iters * kInFlight;
    PR_CUDA(time_it([&] { k_probe_global_or64<<<g_ctas, kProbeThreads, 0, st>>>(l2, l2_words, g_iters); }, g_updates,
                    &out->l2_or64_per_s));
    PR_CUDA(time_it([&] { k_probe_global_or64<<<g_ctas, kProbeThreads, 0, st>>>(hbm, hbm_words, g_iters); },
                    g_updates, &out->hbm_or64_per_s));
    cleanup();
    return KC_OK;
}

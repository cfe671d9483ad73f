// Handle state shared by the C-ABI layer (kc_api.cu) and the batched
// finalize engine (kc_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/kc.h"
#include "kc_internal.h"

struct kc_batch_ctx;

namespace kc {
// The Prune chain (kc_prune.cu): filter and second-filter update over the
// resident reads, then the exact count of the second filter's keys.
void launch_prune(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p, uint64_t* bf1,
                  uint64_t* bf2, DevCounters* ctr, const Grid& g, cudaStream_t st);
void launch_count_chain(const uint64_t* pw, const uint64_t* vw, uint64_t n_units, const PassParams& p,
                        const uint64_t* bf2, Slot* table, DevCounters* ctr, const Grid& g, cudaStream_t st);
}  // namespace kc

namespace kcapi {

struct Batch {
    int sample = 0;
    // direct strategy: the resident reads, rescanned by the recount
    uint64_t* pw = nullptr;  // packed words, 2 * n_units + 2
    uint64_t* vw = nullptr;  // valid-window-start words, n_units
    uint64_t n_units = 0;
    // partitioned strategy: window hashes grouped by partition
    uint64_t* hdata = nullptr;    // capacity: one per base of the batch
    uint64_t* hstarts = nullptr;  // partition starts, 2^part_bits + 1
    uint64_t hcap = 0;
    // partitioned, over the device budget: the reads are kept (pw, vw) and
    // extracted again at kc_finalize, one hash range at a time
    bool deferred = false;
    // partitioned, kc_config.batched_ingest: the reads are kept (pw, vw) until
    // kc_finalize extracts and groups them with the other batches of its batch
    bool pending = false;
    uint64_t n_local = 0;  // bases spanned by the batch's units, from its first unit
};

enum class State { Open, Finalized, Poisoned };

// Windows per partition the library's own choice of partition bits aims at:
// the partition consumer's threads (512) times the 64 iterations of each
// thread whose windows it counts in its filter pass.
constexpr uint64_t kWindowsPerPartition = 32768;

// Host reads copied in chunks by kc_add_reads: chunk c covers units
// [u[c], u[c + 1]); its packed words (and the next unit's first word) and
// N-mask words (and the next one) are on the device once ev[c] has completed
// on the copy stream.  The grouping builds a chunk's valid-window bits and
// extracts its windows as soon as it lands, so the copies of the later chunks
// overlap the extraction of the earlier ones (the double-buffered transfer
// and GPU cycles of Section III-A).
constexpr int kMaxChunks = 4;
constexpr uint64_t kChunkUnits = 1ull << 15;  // units per chunk at least (2 Mbases)
struct ChunkedReads {
    int n = 0;
    uint64_t u[kMaxChunks + 1] = {};
    cudaEvent_t ev[kMaxChunks] = {};
    const uint64_t* nm = nullptr;  // N-mask words of the batch
    const uint64_t* bd = nullptr;  // read-start bits of the batch
    uint64_t start_local = 0, n_local = 0;
};

// One spilled group of partitions: its sorted survivors in pinned host
// memory (keys, then packed counts), the swap metadata of the paper's Count
// unit (partition range, location, number of items).
struct SpillRun {
    uint32_t first_part = 0, n_parts = 0;
    uint64_t* host = nullptr;  // n_items keys followed by n_items packed counts (inside a pinned chunk)
    uint64_t n_items = 0;
};

// Pinned host memory the spilled runs are placed in; kept across kc_reset so
// a repeated out-of-core job does not pin memory again.
struct PinnedChunk {
    uint64_t* p = nullptr;
    uint64_t words = 0, used = 0;
};

kc_status fail(kc_status s, const std::string& msg);
kc_status cuda_fail(cudaError_t e, const char* what);

#define KC_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return kcapi::cuda_fail(e_, #call); \
    } while (0)

// After kernel launches: the launch error, named by where it happened.
#define KC_LAUNCHED(where)                                          \
    do {                                                            \
        cudaError_t e_ = cudaGetLastError();                        \
        if (e_ != cudaSuccess) return kcapi::cuda_fail(e_, where);  \
    } while (0)

}  // namespace kcapi

struct kc_ctx {
    int k = 0, n_samples = 0, n_hashes = 0;
    uint64_t bloom_bits = 0;
    uint32_t min_count = 0;
    kc_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr, copy_stream = nullptr;
    bool own_stream = false;
    cudaEvent_t ev_copy = nullptr, ev_main = nullptr;
    // chunked host copies (kc_add_reads): the offsets check, then one event
    // per chunk; a device word for the check's error bits and its pinned copy
    cudaEvent_t ev_chunk[kcapi::kMaxChunks + 1] = {};
    kc::DevCounters* chk_ctr = nullptr;
    // pinned host words small readbacks land in ([0] the offsets check's
    // error bits, [1..2] the first and last offset of device offsets)
    uint64_t* pinned = nullptr;
    kc::Grid grid;
    int log2_words = 0, log2_slots = 0;
    uint64_t n_slots = 0;
    int strategy = KC_STRATEGY_DIRECT;
    int part_bits = 0;   // partitioned: 2^part_bits partitions
    int l1_bits = 0;     // partitioned: bits of the first grouping at ingest (= part_bits up to 12)
    int slice_log2 = 0;  // partitioned: filter words per partition
    // partitioned, kc_config.part_bits = 0: the partition bits of the filter
    // alone (slices of 4096 words), raised at the first kc_add_reads after
    // create / reset for the windows it brings (kcapi::choose_partitions)
    bool auto_part = false;
    int base_part_bits = 0;

    uint64_t* bloom = nullptr;
    uint64_t* bloom2 = nullptr;  // the Prune chain's second filter (kc_config.prune_chain)
    kc::Slot* table = nullptr;
    kc::DevCounters* ctr = nullptr;
    std::vector<kcapi::Batch> batches;
    uint64_t bases = 0;
    uint64_t reads = 0;  // reads added since create / reset

    uint64_t* res_keys = nullptr;
    uint64_t* res_vals = nullptr;
    uint64_t n_result = 0;
    uint64_t res_cap = 0;

    kc::DevCounters host_ctr{};
    kcapi::State state = kcapi::State::Open;
    size_t fixed_bytes = 0;

    // Phase timing (kc_config.timing): event pairs recorded on the stream,
    // turned into milliseconds after the next synchronisation.
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> ev_pool;
    std::vector<Mark> marks;
    double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t launches = 0;
    uint32_t fallback_partitions = 0;

    // out-of-core results (kc_config.spill)
    bool spilled = false;
    std::vector<kcapi::SpillRun> spill_dir;
    std::vector<kcapi::PinnedChunk> spill_chunks;
    uint64_t spilled_bytes = 0;

    // Filter unit (kc_filter.cu): the selected result keys in key order and
    // their lookup table (2^sel_buckets_log2 buckets of four slots: 32-bit
    // fingerprints, then the slots' 64-bit codes)
    uint64_t* sel_keys = nullptr;
    uint64_t* sel_vals = nullptr;
    uint64_t* sel_table = nullptr;
    uint64_t n_sel = 0;
    int sel_buckets_log2 = 0;
    bool sel_pre = false;  // a shared-memory prefilter follows the table
    bool has_selection = false;
    uint64_t filter_windows = 0, filter_hits = 0;  // summed over kc_filter_reads calls

    // stem-grouped items of the result (kc_export_stems), built on first use
    kc_stem_item* stem_items = nullptr;
    uint64_t n_stems = 0;
    bool has_stems = false;


    // hash-range ownership (kc_config.own_bits): keys with own_h_lo <= h <=
    // own_h_hi, i.e. partitions own_plo .. own_phi - 1
    uint64_t own_h_lo = 0, own_h_hi = ~0ull;
    uint32_t own_plo = 0, own_phi = 0;
    bool owner = false;
    // device budget (kc_config.device_budget) and the batches kept as reads
    uint32_t deferred = 0, scan_groups = 0;

    kc::PassParams params(int sample) const {
        kc::PassParams p{};
        p.h_lo = own_h_lo;
        p.h_hi = own_h_hi;
        p.k = k;
        p.rc_shift = 64 - 2 * k;
        p.kmask = (1ull << (2 * k)) - 1ull;
        p.bloom_shift = 64 - log2_words;
        p.n_hashes = n_hashes;
        p.table_shift = 64 - log2_slots;
        p.table_mask = n_slots - 1;
        p.all_candidates = min_count <= 1 ? 1 : 0;
        p.sample = sample;
        return p;
    }
};

namespace kcapi {

enum Phase {
    kIngest = 0,
    kPass1 = 1,
    kPass2 = 2,
    kCompact = 3,
    kSort = 4,
    kFilterSelect = 5,
    kFilterReads = 6,
    kStems = 7
};

// Phase timing events, recorded on stream st (the handle's stream if null).
cudaEvent_t phase_begin(kc_handle h, cudaStream_t st = nullptr);
void phase_end(kc_handle h, int phase, cudaEvent_t a, cudaStream_t st = nullptr);
void phase_collect(kc_handle h);
kc_status read_counters(kc_handle h);
kc_status device_errors(kc_handle h);
void free_result(kc_handle h);
void release_spill(kc_handle h);
void free_spill_chunks(kc_handle h);
uint64_t* spill_alloc(kc_handle h, uint64_t words);  // nullptr when pinning fails
kc_status check_open(kc_handle h);                   // KC_ERR_ARG / KC_ERR_STATE for null or poisoned
bool is_device_ptr(const void* p);
// Copy a spilled result back to the device and sort it there
// (KC_ERR_OOM_DEVICE, nothing changed, when it does not fit).
kc_status resort_spilled(kc_handle h);
void free_selection(kc_handle h);
void free_stems(kc_handle h);
// Group a batch's window hashes (those in [p.h_lo, p.h_hi]) by partition
// into b.hdata / b.hstarts; exact: size b.hdata after one read-back.
kc_status bucket_batch(kc_handle h, Batch& b, uint64_t n_local, cudaStream_t st, const kc::PassParams& p,
                       bool exact, const ChunkedReads* chunks = nullptr);
// The ingest scatter mode bucket_batch uses for the handle (kc_config.scatter_mode
// resolved against the grouping levels and the shared memory).
int scatter_mode_of(kc_handle h);
uint64_t held_bytes(kc_handle h);
// Extract and group every pending batch (kc_config.batched_ingest) of the
// handles on stream st, ordered after each handle's stream by the caller.
kc_status ingest_pending(kc_handle* hs, int n, cudaStream_t st, int sm_count);
uint64_t room_bytes(kc_handle h);
// Sort n (key, value) pairs (keys below 2^key_bits) from tk/tv into out_k/out_v;
// ctr->survivors holds n on the device; synchronises the stream.
kc_status sort_pairs(kc_handle h, const uint64_t* tk, const uint64_t* tv, uint64_t n, int key_bits,
                     kc::DevCounters* ctr, uint64_t* out_k, uint64_t* out_v, int phase);

}  // namespace kcapi

// Batched finalize of partitioned handles (kc_batch.cu).
kc_status kc_batch_finalize_internal(kc_batch_ctx* b, kc_handle* hs, int n);
kc_status kc_batch_create_internal(cudaStream_t st, kc_batch_ctx** out);
void kc_batch_destroy_internal(kc_batch_ctx* b);

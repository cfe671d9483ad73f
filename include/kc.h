/*
 * kc.h -- C ABI of libkc, a GB300 (sm_103a) k-mer frequency counter.
 *
 * The library counts canonical k-mers of DNA reads per sample, drops k-mers
 * that occur once with a Bloom filter, and returns the exact counts of the
 * survivors in ascending key order.  This is the counting step of the
 * reference-free variant caller described in "Accelerating K-mer Frequency
 * Counting with GPU and Non-Volatile Memory" (Cadenelli, Polo, Carrera):
 *   - k-mers of a read: its M-k+1 substrings of length k (Section II-A);
 *   - 2-bit, 64-bit encoding of a k-mer (Section II-A);
 *   - singleton removal through a Bloom filter that answers "seen before"
 *     (Section III, Prune unit), exact counts per sample (Section II-B, Count
 *     unit; Section III-D, 16-byte k-mer items), false positives removed
 *     before output (Section III, Unify unit).
 *
 * Definitions used throughout (the exact result; readings of the paper that
 * it leaves open are marked "library"):
 *   base codes      A=0 C=1 G=2 T=3; a window over any other character is
 *                   skipped (library reading of the reads' quality check).
 *   key             min(forward, reverse complement), each the 2k-bit number
 *                   whose most significant 2 bits are the window's first base
 *                   (library: canonical keys), so 1 <= k <= 31 fits a uint64.
 *   result          keys whose count summed over samples is >= min_count,
 *                   ascending, with one uint32 count per sample.  A count
 *                   that would pass 2^32-1 is an error, never a wrapped or
 *                   clamped number: kc_finalize returns KC_ERR_CAPACITY (it
 *                   takes more than 4.29e9 copies of one k-mer in one sample).
 *   Bloom filter    bloom_bits / 64 words; key sets n_hashes bits of ONE word
 *                   (library: word-blocked, so a single atomic decides whether
 *                   a key was seen before):
 *                     h = mixer64(key), g = mixer64(h)
 *                     word = h >> (64 - log2(bloom_bits / 64))
 *                     bit i = (g >> 6i) & 63, i < n_hashes
 *                   mixer64 = SplitMix64 output function (Steele, Lea &
 *                   Flood, OOPSLA 2014).
 *
 * Packed read format (what kc_add_reads consumes):
 *   packed_reads  base i of the caller's base stream is bits
 *                 [63-2(i%32) .. 62-2(i%32)] of packed_reads[i/32] (first base
 *                 in the most significant bits).  An N base may hold any code.
 *   n_mask        bit 63-(i%64) of n_mask[i/64] is 1 iff base i is unknown
 *                 (any character other than A, C, G, T).
 *   offsets       n_reads+1 non-decreasing base indices; read r covers bases
 *                 [offsets[r], offsets[r+1]).  offsets[0] may be > 0; only the
 *                 words that cover [offsets[0], offsets[n_reads]) are read.
 *
 * Pointers: every array argument may be host memory (pageable or pinned) or
 * device memory of the handle's device; the library detects which.  The caller
 * owns its arrays; the library owns the filter, the table, its copy of the
 * reads and the result.  All functions return a kc_status; none aborts, exits
 * or traps.  After an error the handle stays valid; if device state may be
 * inconsistent it is poisoned and every later call except kc_destroy,
 * kc_reset and kc_last_error returns KC_ERR_STATE.
 *
 * Threading: a handle is used by one thread at a time.  kc_last_error is
 * per thread.
 */
#ifndef KC_H
#define KC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kc_ctx* kc_handle;

typedef enum kc_status {
    KC_OK = 0,
    KC_ERR_ARG = 1,        /* invalid argument (range, format, offsets)          */
    KC_ERR_STATE = 2,      /* call not allowed now, or handle poisoned           */
    KC_ERR_OOM_DEVICE = 3, /* device allocation failed                          */
    KC_ERR_OOM_HOST = 4,   /* host allocation failed                            */
    KC_ERR_CUDA = 5,       /* CUDA runtime error (message in kc_last_error)      */
    KC_ERR_TIMEOUT = 6,    /* a bounded device wait gave up                      */
    KC_ERR_CAPACITY = 7,   /* table full, count overflow or output too small     */
    KC_ERR_INTERNAL = 8    /* library bug detected by a self-check               */
} kc_status;

/* Tuning and resource knobs; zero means "library default" everywhere. */
typedef struct kc_config {
    uint32_t struct_size;         /* sizeof(kc_config), for ABI growth             */
    uint32_t block_threads;       /* threads per CTA of the streaming kernels       */
    uint32_t ctas_per_sm;         /* resident CTAs per SM for grid sizing (<= 64);
                                     partitioned: extraction CTAs per SM, i.e. the
                                     reads each extraction CTA takes               */
    uint32_t part_bits;           /* partitioned: log2 of the number of hash-prefix
                                     partitions (1..20; above 12 the hashes are
                                     grouped in two levels).  0: chosen by the
                                     library -- filter slices of 4096 words, or
                                     more partitions (at most 2^12, slices of at
                                     least 8 words) when the first kc_add_reads
                                     after create / reset brings more than 32768
                                     windows (bases - reads * (k - 1)) per
                                     partition                                  */
    uint64_t table_slots;         /* direct: open-addressing slots (power of two)
                                     of the global table                            */
    uint32_t spill;               /* partitioned: kc_finalize takes 64 groups of
                                     partitions in turn and copies each group's
                                     sorted result to pinned host memory on a side
                                     stream.  1: kc_dump copies the runs back and
                                     sorts them on the device when it has room
                                     (else as 2); 2: kc_dump merges the runs on
                                     the host                                       */
    uint32_t timing;              /* 1: record CUDA events around every phase on
                                     the handle's stream (see kc_stats.ms_*)        */
    uint32_t strategy;            /* KC_STRATEGY_*                                  */
    uint32_t smem_table_log2;     /* partitioned: log2 shared-memory table slots of
                                     one partition (10..13)                         */
    uint32_t scatter_mode;        /* partitioned ingest: 1 = one global cursor per
                                     partition, 2 = one exact run per (CTA,
                                     partition), 3 = runs padded to whole 32-byte
                                     sectors, staged in shared memory, 4 = as 3,
                                     from hashes first written per CTA to a linear
                                     array (default)                                */
    uint32_t split_max;           /* partitioned: a partition whose candidates
                                     overflow its shared-memory table is counted
                                     again as 2, 4, ... 2^split_max sub-ranges of
                                     its filter slice before it falls back to a
                                     global table (0 = 6; at most the slice's
                                     log2 words; KC_SPLIT_NONE = never split)       */
    uint32_t prune_chain;         /* 1: the paper's two-filter Prune chain (direct
                                     strategy; KC_ERR_ARG with the partitioned one):
                                     kc_add_reads puts every window into the filter
                                     and a window whose bits were all set already
                                     into a second filter of the same size;
                                     kc_finalize counts, in one exact pass, the
                                     windows whose key is in the second filter (see
                                     kc_export_bloom2).  The result is the same.    */
    uint32_t own_bits;            /* partitioned: hash-range ownership.  0: the
                                     handle counts every key.  Else the keys are
                                     split into 2^own_bits shards by the top
                                     own_bits bits of h = mixer64(key) and the
                                     handle counts only the shards own_lo ..
                                     own_hi - 1: its result, filter words and
                                     kc_stats.owned_windows cover those keys alone
                                     (a contiguous slice of the filter; the other
                                     words stay 0).  Handles owning disjoint
                                     ranges of the same reads give disjoint
                                     results whose union, merged by key
                                     (kc_merge_results), is the whole job's, and
                                     whose filters OR to the whole filter: the
                                     second level of partitioning of Section
                                     II-B, one owner per range with its own
                                     structures and no synchronisation.  Needs
                                     own_bits <= the partition bits (1..20)       */
    uint32_t own_lo;              /* first owned shard                              */
    uint32_t own_hi;              /* one past the last owned shard (0 = 2^own_bits) */
    uint64_t device_budget;       /* partitioned: device bytes the job may hold
                                     (filter, resident batches, result).  0: the
                                     device's free memory when the call runs.  A
                                     kc_add_reads whose window hashes would pass
                                     the budget keeps the batch's packed reads
                                     instead (about 0.4 byte per base rather than
                                     8 per window); kc_finalize then extracts and
                                     groups those reads again, one hash range at a
                                     time, and spills the sorted result of every
                                     range to pinned host memory as with spill = 1
                                     (Section III-D: tables swapped out when they
                                     outgrow memory).  A job whose result would
                                     not fit is spilled the same way.            */
    uint32_t batched_ingest;      /* partitioned: 1 = kc_add_reads stores the reads
                                     only, and kc_finalize / kc_batch_finalize
                                     extract and group the windows of every job
                                     of the batch together: one persistent launch
                                     over a queue of (batch, unit range) items per
                                     phase (extraction, bucket offsets, starts,
                                     run bases, staged scatter) instead of a set
                                     of launches per kc_add_reads call.  The
                                     result is the same.                          */
    uint32_t reserved32;
} kc_config;

#define KC_SPLIT_NONE 0xffffffffu

/*
 * Strategies.  Both compute the same result and filter bit for bit.
 *   DIRECT       kc_add_reads updates the global filter with one 64-bit
 *                atomicOr per window and claims candidates in a global
 *                open-addressing table; kc_finalize recounts every window
 *                against that table.
 *   PARTITIONED  kc_add_reads stores each window's 64-bit hash grouped by
 *                2^part_bits hash-prefix partitions (counting-sort shuffle, as
 *                the paper's Encode / Prefix-sum / Broker kernels group k-mers
 *                by consumer, Section III-B); kc_finalize gives each partition
 *                to one CTA that keeps the partition's filter words and table
 *                in shared memory (filter update, candidate claims, exact
 *                recount, compaction).  The filter is built at kc_finalize.
 *   AUTO         PARTITIONED when the filter slices fit shared memory, else
 *                DIRECT.
 */
enum { KC_STRATEGY_AUTO = 0, KC_STRATEGY_DIRECT = 1, KC_STRATEGY_PARTITIONED = 2 };

/* Counters of one job (valid after kc_finalize unless noted). */
typedef struct kc_stats {
    uint64_t windows;         /* valid windows added so far, all samples         */
    uint64_t bases;           /* bases added so far                              */
    uint64_t candidates;      /* windows the filter reported as seen before      */
    uint64_t table_keys;      /* distinct keys held in the table (all partitions) */
    uint64_t result_keys;     /* keys in the result                              */
    uint64_t spilled_bytes;   /* result bytes copied to pinned host memory       */
    uint32_t partitions;      /* hash-prefix partitions used                     */
    uint32_t table_log2;      /* log2 of table slots per partition               */
    uint64_t device_bytes;    /* device memory held by the handle                */
    uint64_t launches;        /* kernels launched since create / reset           */
    /* Device time per phase since create / reset, from CUDA events on the
     * handle's stream (zero unless kc_config.timing = 1; complete after
     * kc_finalize): ingest = read-start and valid-window bits (host reads
     * copied in chunks: their valid bits are built with each chunk's
     * extraction, inside pass1); sort = key-prefix bucketing and bucket sorts.  DIRECT: pass1 = filter update and
     * candidate claims, pass2 = exact recount, compact = survivor compaction.
     * PARTITIONED: pass1 = hash bucketing (count and scatter), pass2 = the
     * shared-memory partition consumer (filter, claims, recount, compaction),
     * compact = fallback partitions. */
    double ms_ingest, ms_pass1, ms_pass2, ms_compact, ms_sort;
    uint32_t strategy;              /* KC_STRATEGY_DIRECT or KC_STRATEGY_PARTITIONED */
    uint32_t fallback_partitions;   /* partitions whose table left shared memory    */
    uint32_t split_partitions;      /* partitions counted as sub-ranges (split_max) */
    uint32_t split_level;           /* finest split level any partition needed      */
    /* Filter unit (kc_filter_*; timing as above): time on the handle's
     * stream of all selections (compaction and lookup table, from the first
     * kernel to the last, host gaps included) and of the rescan kernels of
     * all kc_filter_reads calls since create / reset; keys of the current
     * selection, valid windows rescanned and windows whose key was selected. */
    double ms_filter_select, ms_filter_reads;
    uint64_t filter_selected, filter_windows, filter_hits;
    /* Stem table (kc_export_stems; timing as above): device time of building
     * it, and its number of items. */
    double ms_stems;
    uint64_t stem_items;
    /* Windows whose key the handle owns (= windows without own_bits; complete
     * after kc_finalize), batches kept as packed reads because their hashes
     * would have passed the device budget, and the hash ranges kc_finalize
     * extracted those batches in (0 when none was kept). */
    uint64_t owned_windows;
    uint32_t deferred_batches;
    uint32_t scan_groups;
} kc_stats;

/*
 * Batched finalize (partitioned strategy): many handles finalized together.
 * Their partitions form one work queue served by one persistent launch (each
 * CTA takes the next (job, partition) item); their survivors are sorted by a
 * CUDA graph captured once per batch object and replayed for every batch.
 * Results are the same as finalizing each handle alone.
 */
typedef struct kc_batch_ctx* kc_batch;

/* Create a batch object whose work is ordered on stream (a cudaStream_t as
 * void*; NULL = its own stream). */
kc_status kc_batch_create(void* stream, kc_batch* out);

/* Finalize n open handles (all partitioned, distinct) together.  Work queued
 * on each handle's stream is finished first; afterwards each handle is
 * finalized as by kc_finalize and its stream is ordered after the batch. */
kc_status kc_batch_finalize(kc_batch b, kc_handle* handles, int n);

/* Batched ingest (kc_config.batched_ingest; Section III-A's pipeline of
 * transfer and GPU cycles, its kernels over every job of the batch): extract
 * and group the reads that the n handles' kc_add_reads calls kept, all
 * together on the batch's stream -- a persistent extraction launch over a
 * queue of (read batch, unit range) items of every job, one launch each for
 * the bucket offsets, starts and run bases of all of them, and a persistent
 * staged-scatter launch over the same items.  Handles without kept reads, or
 * not partitioned or open, are left alone.  The call does not wait for the
 * device: each handle's stream is ordered after the work, so a later
 * kc_finalize / kc_batch_finalize (which runs this step itself for reads
 * still kept) sees the grouped hashes.  KC_ERR_ARG for a null batch or
 * handle list, or a handle listed twice. */
kc_status kc_batch_ingest(kc_batch b, kc_handle* handles, int n);

void kc_batch_destroy(kc_batch b);

/*
 * Job server with continuous batching (host-submitted jobs).  Two ingest
 * threads admit queued jobs in arrival order as soon as their estimated
 * device footprint fits device_budget_bytes and copy their reads to the
 * device on their own streams (kc_config.batched_ingest); an extract thread
 * takes every job copied so far and extracts and groups them together
 * (kc_batch_ingest, one launch per phase); two finalize threads, each with
 * its own batch object, repeatedly
 * take every job ingested so far (at most max_batch) as one batch
 * (kc_batch_finalize), copy the results into pinned host blocks (one pool
 * per process, reused across jobs and servers and kept until the process
 * exits, up to 8 GiB; ordinary host memory past that) and release the jobs'
 * device memory.  Jobs that arrive while a batch runs are ingested at
 * once and join a next batch.  Each job's result is the one kc_finalize would
 * give it alone.  All kc_server_* calls are thread-safe.
 */
typedef struct kc_server_ctx* kc_server;

typedef struct kc_job_spec {
    int k, n_samples, n_hashes;
    uint32_t min_count;
    uint64_t bloom_bits;
    /* per sample, in the packed format above, HOST memory that must stay
     * valid until kc_server_wait has returned for the job */
    const uint64_t* packed[2];
    const uint64_t* offsets[2];
    const uint64_t* n_mask[2];
    uint64_t n_reads[2];
} kc_job_spec;

typedef struct kc_server_stats {
    uint64_t submitted, completed, failed, batches;
    double mean_batch;        /* jobs per finalized batch                      */
    double p50_ms, p99_ms, mean_ms;  /* submit -> result in host memory        */
    double jobs_per_s;        /* completed jobs / (last completion - first submit) */
    uint64_t peak_bytes;      /* largest admitted footprint sum                */
    uint64_t budget_bytes;
    /* mean stage times of completed jobs: submit -> admitted, admitted ->
     * reads on the device, -> its batch starts, batch start -> result in host
     * memory */
    double mean_queue_ms, mean_ingest_ms, mean_batch_wait_ms, mean_finalize_ms;
    /* where a finalize thread's time goes, mean per batch: the batched
     * finalize call, then copying the batch's results to host memory, then
     * releasing its jobs' handles */
    double mean_batch_finalize_ms, mean_batch_copy_ms, mean_batch_release_ms;
    /* jobs that ran on a finished job's handle (reset and kept for the next
     * job with the same parameters) instead of a new one */
    uint64_t reused_handles;
    /* mean per job of the ingest stage's two parts: getting a handle (a
     * reused one, or kc_create_ex) and adding its reads (kc_add_reads) */
    double mean_ingest_handle_ms, mean_ingest_add_ms;
} kc_server_stats;

/* Create a server on the current device (max_batch >= 1). */
kc_status kc_server_create(uint64_t device_budget_bytes, int max_batch, kc_server* out);
/* As kc_server_create; flags KC_SERVER_TUNED: every job takes the partitioned
 * knobs of its class from the tuning cache (kc_tune_lookup) when there is an
 * entry, the defaults otherwise. */
#define KC_SERVER_TUNED 1u
kc_status kc_server_create_ex(uint64_t device_budget_bytes, int max_batch, uint32_t flags, kc_server* out);
/* Queue a job; *job_id identifies it.  KC_ERR_ARG for device pointers. */
kc_status kc_server_submit(kc_server s, const kc_job_spec* spec, uint64_t* job_id);
/* Wait for a job (timeout_s < 0: no limit; KC_ERR_TIMEOUT when it runs out);
 * returns the job's status, its result size and its latency. */
kc_status kc_server_wait(kc_server s, uint64_t job_id, double timeout_s, uint64_t* n_keys, double* latency_ms);
/* Copy a finished job's result (as kc_dump) and forget the job; keys == NULL
 * only reports the size and keeps the job. */
kc_status kc_server_result(kc_server s, uint64_t job_id, uint64_t* keys, uint32_t* counts, uint64_t capacity,
                           uint64_t* n_out);
kc_status kc_server_stats_get(kc_server s, kc_server_stats* out);
/* Stop the threads; jobs not finished are dropped. */
void kc_server_destroy(kc_server s);

/* Fill *cfg with the defaults (struct_size set). */
void kc_default_config(kc_config* cfg);

/*
 * Autotuning.  The paper sizes its work units by hand and notes that the
 * chunk sizes have to be chosen with care (Section III-B, the Orchestrator's
 * cycles); here the library measures instead.  kc_autotune runs the caller's
 * own job (the same reads, k, filter, hashes, min_count) once per candidate
 * configuration and keeps the fastest:
 *   PARTITIONED  partition bits (filter slices of 2^13 down to 2^8 words),
 *                then the shared-memory table size (2^10..2^13 slots), then
 *                extraction CTAs per SM (the reads each CTA takes: 1, 2, 3)
 *   DIRECT       grid CTAs per SM (4, 8, 16)
 * Each candidate is timed as the median, over `reps` runs after one warm-up
 * run, of the CUDA-event time from before kc_add_reads to after kc_finalize
 * on the tuner's stream (allocation in kc_create_ex is outside the timing).
 * Block sizes are fixed per kernel and are not searched.
 *
 *   inputs    n_inputs read batches, each added with kc_add_reads (host or
 *             device pointers, as there; device inputs time the counting alone)
 *   best      the fastest configuration
 *   trials    if not NULL, up to max_trials timed candidates in the order
 *             tried (ms < 0: the candidate was rejected or failed); *n_trials
 *             receives the number written
 *
 * The best configuration is also stored in a process-wide cache under the
 * job's class (k, n_samples, bloom_bits, n_hashes, min_count > 1, the bases
 * rounded up to a power of two, the device's SM count), where kc_tune_lookup
 * finds it; kc_tune_cache_save / kc_tune_cache_load keep the cache in a text
 * file, one class per line.
 */
typedef struct kc_tune_input {
    int sample;
    const uint64_t* packed_reads;
    const uint64_t* offsets;
    const uint64_t* n_mask;
    uint64_t n_reads;
} kc_tune_input;

typedef struct kc_tune_trial {
    kc_config config;
    double ms;
} kc_tune_trial;

kc_status kc_autotune(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                      const kc_tune_input* inputs, int n_inputs, int reps, kc_config* best,
                      kc_tune_trial* trials, int max_trials, int* n_trials);

/* The cached configuration of the job class of (k, n_samples, bloom_bits,
 * n_hashes, min_count, n_bases) on the current device: *found = 1 and *out
 * filled, or *found = 0 and *out left alone. */
kc_status kc_tune_lookup(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                         uint64_t n_bases, kc_config* out, int* found);

/* Write the cache to path (replacing the file) / merge the entries of path
 * into the cache (KC_ERR_ARG for a malformed file, which changes nothing). */
kc_status kc_tune_cache_save(const char* path);
kc_status kc_tune_cache_load(const char* path);
/* Drop every cached entry. */
void kc_tune_cache_clear(void);

/*
 * Create a counting job on the current CUDA device.
 *   k          window length, 1..31
 *   n_samples  1 or 2 (2: joint normal/tumour table, Section III-D layout of
 *              one key with two counts)
 *   bloom_bits power of two, >= 4096
 *   n_hashes   bits per key in its filter word, 1..10
 *   min_count  keys whose count summed over samples is below this are dropped
 *              (2 drops the k-mers that occur once; 1 keeps every key)
 * Returns KC_ERR_ARG on out-of-range arguments.
 */
kc_status kc_create(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                    kc_handle* out);

/*
 * As kc_create, with tuning knobs (cfg may be NULL) and a CUDA stream
 * (a cudaStream_t passed as void*; NULL = the library creates its own) on
 * which every device operation of the handle is ordered.
 */
kc_status kc_create_ex(int k, int n_samples, uint64_t bloom_bits, int n_hashes, uint32_t min_count,
                       const kc_config* cfg, void* stream, kc_handle* out);

/*
 * Add n_reads reads of one sample (0 <= sample < n_samples) in the packed
 * format above.  The library copies what it needs: host arrays before
 * returning, so the caller may reuse them at once; device arrays on the
 * handle's stream, in order after the work already queued there, so the
 * caller may reuse them once its own work is ordered after that stream
 * (kc_finalize returns after it).  Device work continues asynchronously on
 * the handle's stream.  Host reads of at least 2 x 2^15 units (64 bases
 * each) are copied in up to four chunks, each extracted as it lands (Section
 * III-A's overlapped transfer and GPU cycles).  Reads shorter than k add no
 * windows.  Offsets that decrease give KC_ERR_ARG (checked before the call
 * returns for host reads -- on the host, or for the chunked copies on the
 * device -- and on the device for device reads, where the error surfaces at
 * kc_finalize).  Not allowed after kc_finalize (KC_ERR_STATE).
 */
kc_status kc_add_reads(kc_handle h, int sample, const uint64_t* packed_reads, const uint64_t* offsets,
                       const uint64_t* n_mask, uint64_t n_reads);

/* Finish the job: exact recount, singleton and false-positive removal, sort.
 * Blocks until the result is ready on the device. */
kc_status kc_finalize(kc_handle h);

/*
 * Copy the result: keys[i] ascending, counts[i * n_samples + s].  With
 * keys == NULL only *n_out is written (size query).  capacity is in keys;
 * a smaller capacity than the result gives KC_ERR_CAPACITY and *n_out = size.
 */
kc_status kc_dump(kc_handle h, uint64_t* keys, uint32_t* counts, uint64_t capacity, uint64_t* n_out);

/* Copy filter words [first_word, first_word + n_words) (for parity checks and
 * checkpoints).  Blocks until pending work is done.  With the partitioned
 * strategy the filter is built by kc_finalize (all zero before). */
kc_status kc_export_bloom(kc_handle h, uint64_t* words, uint64_t first_word, uint64_t n_words);

/* Copy words [first_word, first_word + n_words) of the Prune chain's second
 * filter (kc_config.prune_chain = 1; KC_ERR_STATE otherwise).  Its content
 * depends on the order in which concurrent windows reach the first filter: it
 * holds every key seen at least twice, and a key seen once only if other keys
 * had set all of its bits before it. */
kc_status kc_export_bloom2(kc_handle h, uint64_t* words, uint64_t first_word, uint64_t n_words);

kc_status kc_stats_get(kc_handle h, kc_stats* out);

/*
 * Downstream of the count: the result in the paper's item form, its joint
 * count spectrum, and the Filter unit.  All need a finalized handle; a result
 * spilled to host memory (kc_config.spill) is first copied back and sorted on
 * the device (KC_ERR_OOM_DEVICE if it does not fit).  Output arrays may be
 * host or device memory; every call blocks until its output is written.
 */

/* One k-mer item of the joint table in the 16-byte form of Section III-D:
 * 8 bytes of k-mer, the two samples' counts in 4 bytes, 4 bytes of padding.
 * count[s] = min(count of sample s, 65535); count[1] = 0 for one sample;
 * pad = 0. */
typedef struct kc_item16 {
    uint64_t key;
    uint16_t count[2];
    uint32_t pad;
} kc_item16;

/* Write the result as items, ascending keys (same order and keys as kc_dump).
 * items == NULL: size query (*n_out).  capacity in items; a smaller capacity
 * than the result gives KC_ERR_CAPACITY.  Device items must be 16-byte
 * aligned (KC_ERR_ARG otherwise). */
kc_status kc_export_items(kc_handle h, kc_item16* items, uint64_t capacity, uint64_t* n_out);

/* Joint count spectrum of the result: with two samples
 * hist[min(c0, cap) * (cap + 1) + min(c1, cap)] = number of result keys with
 * those clamped counts ((cap + 1)^2 entries); with one sample hist[min(c0,
 * cap)] (cap + 1 entries).  hist is overwritten.  1 <= cap <=
 * KC_SPECTRUM_MAX_CAP. */
#define KC_SPECTRUM_MAX_CAP 1023u
kc_status kc_spectrum(kc_handle h, uint32_t cap, uint64_t* hist);

/* One item of the stem-grouped table (Section II-A: a stem is the middle k-2
 * bases of a k-mer; Section III-D: a 72-byte item of 8 bytes of stem and a
 * 2-byte count per sample for each of the 16 k-mers that extend the stem by
 * one base on each side).  With canonical keys: one item per canonical stem
 * c (the smaller of a stem and its reverse complement, as a 2(k-2)-bit code)
 * with at least one non-zero entry; count[s][4 * code(x) + code(y)] =
 * min(count of sample s of the canonical key of the k-mer x c y, 65535), 0
 * if that key is not in the result; count[1][*] = 0 for one sample. */
typedef struct kc_stem_item {
    uint64_t stem;
    uint16_t count[2][16];
} kc_stem_item;

/* Write the stem-grouped table, ascending stems.  Built on the device at the
 * first call after kc_finalize and kept until kc_reset.  items == NULL: size
 * query.  KC_ERR_STATE for k < 3; KC_ERR_CAPACITY when capacity (in items) is
 * smaller than the table. */
kc_status kc_export_stems(kc_handle h, kc_stem_item* items, uint64_t capacity, uint64_t* n_out);

/*
 * Filter unit (Section II-B): select the k-mers whose counts differ between
 * the normal and the tumoral sample, then read the input again and look every
 * k-mer up among the selected ones, which finds the reads that carry them.
 * The paper gives no threshold; a result key is selected iff, with t = tumor
 * and n = the other sample,
 *     count[t] >= min_tumor  and  count[n] <= max_normal  and
 *     count[t] >= ratio * count[n]          (ratio 0: no ratio test)
 * Only keys of the result (count summed over samples >= min_count) can be
 * selected.  Two-sample handles only (KC_ERR_STATE otherwise).
 */
typedef struct kc_filter_spec {
    int tumor;            /* sample holding the tumoral reads: 0 or 1        */
    uint32_t min_tumor;
    uint32_t max_normal;
    uint32_t ratio;
} kc_filter_spec;

/* Select the keys (replacing an earlier selection); *n_selected = how many.
 * KC_ERR_ARG for tumor outside 0..1. */
kc_status kc_filter_select(kc_handle h, const kc_filter_spec* spec, uint64_t* n_selected);

/* Copy the selected keys, ascending, with their counts (counts[i * 2 + s]),
 * as kc_dump does for the result.  KC_ERR_STATE before kc_filter_select. */
kc_status kc_filter_keys(kc_handle h, uint64_t* keys, uint32_t* counts, uint64_t capacity, uint64_t* n_out);

/*
 * Rescan n_reads reads (packed format above, any sample or any other read
 * set; the arrays are not kept) against the selection:
 *   hits        n_reads uint32, overwritten: hits[r] = number of valid
 *               windows of read r whose canonical key is selected
 *   candidates  NULL, or room for n_reads uint64: the indices r (0-based in
 *               this call) with hits[r] > 0, ascending
 *   n_candidates  number of reads with hits[r] > 0
 * KC_ERR_STATE before kc_filter_select; KC_ERR_ARG for decreasing offsets.
 */
kc_status kc_filter_reads(kc_handle h, const uint64_t* packed_reads, const uint64_t* offsets, const uint64_t* n_mask,
                          uint64_t n_reads, uint32_t* hits, uint64_t* candidates, uint64_t* n_candidates);

/* Forget all reads and results but keep the allocations, for a new job with
 * the same parameters. */
kc_status kc_reset(kc_handle h);

void kc_destroy(kc_handle h);

/*
 * kc_merge_results -- merge n_runs results, each sorted by key with keys
 * unique across runs (as handles owning disjoint hash ranges of one job give
 * them), into one ascending result.  Host memory only; no GPU is used.
 *   keys[r], counts[r]  run r: n[r] keys and n[r] x n_samples counts (row-major)
 *   out_keys, out_counts  sum of n[r] entries each; out_counts may be NULL
 * KC_ERR_ARG for null arrays, n_samples outside 1..2 or a run that is not
 * strictly ascending; KC_ERR_ARG also when two runs hold the same key (the
 * ranges were not disjoint).  Runs of more than 2^20 keys in all are merged on
 * several host threads.
 */
kc_status kc_merge_results(int n_runs, const uint64_t* const* keys, const uint32_t* const* counts, const uint64_t* n,
                           int n_samples, uint64_t* out_keys, uint32_t* out_counts);

/*
 * kc_atomic_ceilings -- measured ceilings of the random atomic updates the
 * counting kernels are made of (the paper finds random updates of its filters
 * and tables to bound counting, Section IV-C).  Each field is updates per
 * second over the whole GPU, one kind of update at random addresses:
 *   smem_or64_per_s   64-bit atomicOr into a 4096-word shared-memory array
 *                     per CTA (the partition consumer's filter slice)
 *   smem_add32_per_s  32-bit atomicAdd into 4096 shared-memory counters per
 *                     CTA (the extraction and scatter histograms, the
 *                     consumer's counts)
 *   l2_or64_per_s     64-bit atomicOr into a 16 MiB global array (held in L2)
 *   hbm_or64_per_s    64-bit atomicOr into a 4 GiB global array (beyond L2:
 *                     the direct strategy's filter update)
 * Allocates about 4 GiB of device memory for the call; work is ordered on
 * stream (cudaStream_t as void*, NULL = the legacy default stream) and the
 * call returns when it is done.  A measurement aid, not a step of the path.
 */
typedef struct kc_atomic_rates {
    double smem_or64_per_s, smem_add32_per_s, l2_or64_per_s, hbm_or64_per_s;
} kc_atomic_rates;
kc_status kc_atomic_ceilings(kc_atomic_rates* out, void* stream);

/* Message of the last error on this thread ("" if none). */
const char* kc_last_error(void);

/* Name of a status code. */
const char* kc_status_string(kc_status s);

/*
 * kc_bloom_build_noalloc -- the Bloom filter of one read set (the filter
 * kc_export_bloom returns after counting the same reads with the same k,
 * bloom_bits and n_hashes), computed without allocating any memory.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory when they need the filter -- an application whose
 * own allocator already holds the device's memory, a latency-critical loop
 * that must not wait on cudaMalloc, or code restricted to the buffers it was
 * given.
 *
 *   packed_reads, offsets, n_mask  inputs in the packed format above; all in
 *                  device memory of the current device, or managed memory
 *                  (KC_ERR_ARG otherwise: host memory and another GPU's memory
 *                  are refused, since nothing is copied first)
 *   bloom_out      bloom_bits / 64 words of such memory, overwritten
 *   stream         cudaStream_t as void*, NULL for the default stream; the call
 *                  synchronises this stream twice (it reads the read range
 *                  back before its launches and the error bits after them) and
 *                  returns after its work on the stream is done
 *
 * Everything intermediate lives in one fixed scratch array inside the library
 * (a file-scope __device__ array of about 4 MiB that every GPU loading the
 * library keeps until the process exits), so a read set may span at most
 * KC_NOALLOC_MAX_BASES bases from offsets[0] rounded down to a multiple of 64
 * to offsets[n_reads]; larger sets give KC_ERR_CAPACITY.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current).  All calls share the array and each clears the parts that
 * must start at zero, so calls whose device work overlaps (other streams or
 * host threads) race: order them.
 * Errors are reported by the status and kc_last_error().
 */
#define KC_NOALLOC_MAX_BASES (1ull << 23)
kc_status kc_bloom_build_noalloc(int k, uint64_t bloom_bits, int n_hashes, const uint64_t* packed_reads,
                                 const uint64_t* offsets, const uint64_t* n_mask, uint64_t n_reads,
                                 uint64_t* bloom_out, void* stream);

/*
 * Host helper: pack n_bases ASCII characters into the packed format above
 * (packed: ceil(n_bases/32) words, n_mask: ceil(n_bases/64) words, both
 * written in full, unused tail bits zero).  Any byte other than 'A','C','G','T'
 * is an unknown base.
 */
kc_status kc_pack_ascii(const char* ascii, uint64_t n_bases, uint64_t* packed, uint64_t* n_mask);

#ifdef __cplusplus
}
#endif

#endif /* KC_H */

/*
 * pcfsort.h -- C ABI of the GB300 (sm_103a) PCF Learned Sort library.
 *
 * The library sorts 64-bit keys on one GPU with PCF Learned Sort
 * (Sato & Matsui, "PCF Learned Sort: a Learning Augmented Sort Algorithm
 * with O(n log log n) Expected Complexity", TMLR 2025):
 *   Algorithm 1 (Learned-Sort): inputs shorter than tau go to a standard
 *   sort; otherwise a CDF model is trained, every key is appended to bucket
 *   floor(F(x) gamma) + 1 of gamma + 1 buckets, buckets of size >= delta are
 *   sorted by the standard sort and the others recursively, and the sorted
 *   buckets are concatenated.
 *   Sec. 3.3 (PCF model): alpha sampled keys are counted into beta
 *   equal-width bins i(x) = floor((x - x_min) beta / (x_max - x_min)) + 1,
 *   b_i = |{j : i(a_j) <= i}| and F(x) = b_{i(x)} / alpha.
 *   Theorem pcf-nlogn / Sec. 4: alpha = beta = gamma = delta = floor(n^{3/4}),
 *   tau = 100 (the default policy).
 *
 * The output is the unique ascending order of the keys (IEEE-754 total
 * order for binary64 keys, so -0 sorts before +0; unsigned order for u64
 * keys); the pair sorts are stable (equal keys keep their input order).
 * Results do not depend on the seed, the policy or the tuning.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers of the context's device; h_*
 *     pointers are HOST pointers.  The caller owns all key and value buffers.
 *     d_in may equal d_out (in-place sort); otherwise the ranges must not
 *     overlap.  Keys are 8-byte aligned, values 4-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Calls are issued on `stream`, ordered after the work already queued
 *     there, and return when the sort is complete on the device, except
 *     where stated.  They block because Algorithm 1's recursion is
 *     data-dependent: each global level ends with the host reading back the
 *     level's record (how many buckets go on to the next level, to the
 *     standard sort, or are finished on chip), which sizes the next level's
 *     launches.  A replayed sort graph (pcf_graph_*) runs the whole sort with
 *     no such read-back.  pcf_ctx_sync returns the last sort's status.
 *     A context serialises its own calls; use one context per host thread.
 *   - Errors are returned, never raised: no call aborts, traps or exits.
 *     On PCF_ERR_INVALID_KEY (a NaN key) the output buffers are not written.
 *     n = 0 and n = 1 succeed without device work other than a copy.
 *   - Maximum n per array (and per batched call in total): 2^32 - 1 keys.
 */
#ifndef PCFSORT_H
#define PCFSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCF_KEY_F64 = 0, /* IEEE-754 binary64, ordered by the total order, NaN rejected */
  PCF_KEY_U64 = 1  /* unsigned 64-bit integers                                     */
} pcf_key_type;

typedef enum {
  PCF_OK = 0,
  PCF_ERR_INVALID_ARG = 1, /* bad pointer, size, key type, policy or tuning            */
  PCF_ERR_INVALID_KEY = 2, /* a NaN key (the paper's keys are real numbers)            */
  PCF_ERR_OOM = 3,         /* device or pinned-host allocation failed                  */
  PCF_ERR_CUDA = 4,        /* a CUDA runtime call failed (see pcf_last_cuda_error)     */
  PCF_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (no trap is used)     */
  PCF_ERR_INTERNAL = 6     /* an internal consistency check failed                     */
} pcf_status;

/* CDF model of every bucketing step: the piecewise-constant PCF of Sec. 3.3
 * (F(x) = b_k / alpha in bin k), or the piecewise-linear spline through the
 * same counts of Spline Learned Sort (App. A.5: F(x) = (b_{k-1} + f (b_k -
 * b_{k-1})) / alpha, f the key's position in its bin).  Binary64 evaluation,
 * the order of operations stated in the library's design notes. */
typedef enum { PCF_MODEL_PCF = 0, PCF_MODEL_SPLINE = 1 } pcf_model;

/* Range the bins span in every bucketing step: the (sub)array's own minimum
 * and maximum (Sec. 3.3: one full pass per step), or the alpha sampled keys'
 * (no full pass; keys outside that range take the end bins; where the
 * samples are all equal or their range is degenerate, the array's range is
 * used).  The output is the same either way. */
typedef enum { PCF_RANGE_ARRAY = 0, PCF_RANGE_SAMPLE = 1 } pcf_range;

/* Parameters of Algorithm 1: alpha = floor(n^(a_num/den)), beta = ...(b_num),
 * gamma = ...(c_num), delta = ...(d_num), recomputed for every (sub)array
 * from its own n; tau is the small-input threshold; model a pcf_model;
 * range_mode a pcf_range.  Supported: den in 1..4, 1 <= a_num, b_num, c_num
 * <= den, 1 <= d_num < den (0 < d < 1, as Lemma nlogn requires),
 * 16 <= tau <= 65535.  Default: {3,3,3,3,4,PCF_MODEL_PCF,100,PCF_RANGE_ARRAY}. */
typedef struct {
  uint32_t a_num, b_num, c_num, d_num, den;
  uint32_t model;
  uint64_t tau;
  uint32_t range_mode;
} pcf_policy;

/* Implementation knobs.  They change speed only, never the result or the
 * model: max_digit_bits = widest bucket-id digit scattered per global pass
 * (4..12); tile_log2 = log2 of keys per count tile of pass 1 (12..18; pass 2
 * uses tiles 4x larger);
 * leaf_cap = the largest bucket finished on chip (64..8192, power of two; key-
 * value sorts use at most 1024, and a smaller one where the policy's tables
 * would not fit shared memory);
 * leaf_mode = how keys-only sorts finish a bucket on chip: 1 = a block-local
 * Standard-Sort of the whole bucket (one equal-width MSD split of its range,
 * then ranks within the parts), 2 = the remaining Learned-Sort steps of
 * Algorithm 1 run in shared memory.  Key-value sorts always take 2.
 * Zero fields keep the current value.  Default: {11, 14, 8192, 1}. */
typedef struct {
  uint32_t max_digit_bits;
  uint32_t tile_log2;
  uint32_t leaf_cap;
  uint32_t leaf_mode;
} pcf_tuning;

typedef struct pcf_ctx pcf_ctx;

/* Per-call counters (filled by the last sort on the context). */
typedef struct {
  uint64_t levels;           /* global bucketing levels run                     */
  uint64_t global_passes;    /* digit scatter passes over device memory         */
  uint64_t leaf_buckets;     /* buckets finished in shared memory               */
  uint64_t fallback_buckets; /* buckets sent to the standard sort (|c| >= delta or degenerate) */
  uint64_t fallback_keys;
  uint64_t bytes_moved;      /* bytes read + written by all passes (a model: range 8,
                                histogram 12, scatter 22 and 18, on-chip 16, fallback 16
                                per merge pass, per key; + values)                */
  uint64_t kernel_launches;  /* this library's kernel launches in the call       */
  uint64_t fallback_splits;  /* fallback items split three ways around a value that
                                dominates them (below / equal / above)          */
  /* Alg. 1's decisions, for comparison with a sequential PCF Learned Sort:
   * buckets whose size reached the failure guard |c_j| >= delta (at any
   * level, on chip included) and their keys, and Learned-Sort calls that
   * bucketed their input (a model built and every key appended).  Key-value
   * sorts append stably and take every step of Alg. 1, so these equal a
   * sequential run's; keys-only sorts may append equal-bucket keys in another
   * order and finish on-chip buckets by a block-local sort (tuning leaf_mode). */
  uint64_t guard_buckets;
  uint64_t guard_keys;
  uint64_t bucketings;
} pcf_call_stats;

/* Creates a context on `device`.  The context owns its workspace (grown on
 * demand, kept until destroy), a status word and a pinned host staging area. */
pcf_status pcf_ctx_create(pcf_ctx** out, int device);
/* Frees everything the context owns.  NULL is accepted. */
pcf_status pcf_ctx_destroy(pcf_ctx* ctx);
/* Replaces the policy (copied).  PCF_ERR_INVALID_ARG if unsupported. */
pcf_status pcf_ctx_set_policy(pcf_ctx* ctx, const pcf_policy* policy);
/* Replaces non-zero tuning fields (copied). */
pcf_status pcf_ctx_set_tuning(pcf_ctx* ctx, const pcf_tuning* tuning);
pcf_status pcf_ctx_get_tuning(const pcf_ctx* ctx, pcf_tuning* out);
/* Pre-allocates workspace for sorts of up to n_total keys (pairs != 0: with
 * values) so that later calls allocate nothing. */
pcf_status pcf_ctx_reserve(pcf_ctx* ctx, uint64_t n_total, int pairs);
/* Counters of the last sort on this context. */
pcf_status pcf_ctx_last_stats(const pcf_ctx* ctx, pcf_call_stats* out);
/* Waits for the work queued on `stream` and returns the status of the
 * context's last sort (PCF_OK before any).  Sorts already return their
 * status when they finish; this is the stream-ordered way to read it. */
pcf_status pcf_ctx_sync(pcf_ctx* ctx, void* stream);

/* Device workspace for sorting n_total keys in S arrays (pairs != 0: with
 * u32 values) with the policy and tuning of ctx (NULL: the defaults): an
 * upper bound, in bytes, on what a context grows to for such a sort (the
 * key-sized scratch of 14 bytes per key, 18 with values, plus the level
 * tables, sized for S arrays of equal length at level 0 and for every key
 * reaching a deeper level).  The context allocates on demand; this figure
 * lets a caller budget device memory before the call (or reserve it with
 * pcf_ctx_reserve, which pre-allocates the key-sized part).  *out = 0 for
 * n_total = 0.  PCF_ERR_INVALID_ARG: n_total > 2^32 - 1, or S = 0 with keys. */
pcf_status pcf_workspace_bytes(const pcf_ctx* ctx, uint64_t n_total, uint32_t S,
                               pcf_key_type kt, int pairs, uint64_t* out);
/* Device bytes the context holds now (the sum of its workspace buffers). */
pcf_status pcf_ctx_workspace_held(const pcf_ctx* ctx, uint64_t* out);

/* Sorts n keys (Algorithm 1, PCF model of Sec. 3.3) from d_in into d_out. */
pcf_status pcf_sort_keys(pcf_ctx* ctx, const void* d_in, void* d_out, uint64_t n,
                         pcf_key_type kt, uint64_t seed, void* stream);

/* Stable key-value sort: d_vals_out[i] is the value that travelled with
 * d_keys_out[i]; equal keys keep their input order. */
pcf_status pcf_sort_pairs(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                          void* d_keys_out, uint32_t* d_vals_out, uint64_t n,
                          pcf_key_type kt, uint64_t seed, void* stream);

/* Sorts S independent arrays in one batched pass.  Segment s is keys
 * [h_offsets[s], h_offsets[s+1]) of the key buffers (h_offsets: S+1
 * non-decreasing HOST values, h_offsets[0] = 0) and is sorted exactly as
 * pcf_sort_keys / pcf_sort_pairs would sort it with seed + s.  d_vals_* may
 * be NULL (keys only).  In-place when d_keys_in == d_keys_out. */
pcf_status pcf_sort_segmented(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                              void* d_keys_out, uint32_t* d_vals_out,
                              const uint64_t* h_offsets, uint32_t S, pcf_key_type kt,
                              uint64_t seed, void* stream);

/* pcf_sort_segmented with the S+1 offsets in DEVICE memory (u64, 8-byte
 * aligned; the rules of h_offsets apply) and n_cap the number of keys the
 * key (and value) buffers hold.  The offsets are read on `stream`, after
 * the work queued there (a kernel that produced them on that stream need
 * not be waited for), through the context's pinned staging buffer; offsets
 * that break the rules, or end beyond n_cap, return PCF_ERR_INVALID_ARG with
 * nothing written. */
pcf_status pcf_sort_segmented_dev(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                                  void* d_keys_out, uint32_t* d_vals_out,
                                  const uint64_t* d_offsets, uint32_t S, uint64_t n_cap,
                                  pcf_key_type kt, uint64_t seed, void* stream);

/* Allocation-free batched sort of small arrays (keys only; the paper has no
 * counterpart: it is an interface for callers that must not allocate device
 * memory during a call -- cudaMalloc/cudaFree synchronise the whole device,
 * and memory held by a caching allocator or an engine may be exhausted).
 *
 * Sorts S arrays of at most PCF_STATIC_MAX_ARRAY_KEYS keys each, exactly as
 * pcf_sort_segmented would with the default policy and seed + s for array s.
 * d_offsets: S+1 non-decreasing u64 DEVICE values, d_offsets[0] = 0,
 * d_offsets[S] = n_total (checked on the device).  In-place when
 * d_keys_in == d_keys_out.  Runs on the calling thread's current device.
 *
 * Scratch: one fixed device array of the library (about 2.9 MB per device),
 * its address resolved by cudaGetSymbolAddress on the first call on each
 * device; make that first call before any stream capture on the device.
 * The address is kept for the life of the process: after cudaDeviceReset
 * on a device, do not call this entry point on that device again.
 * `stream` must belong to the current device (else PCF_ERR_INVALID_ARG).
 * Calls no allocating CUDA or library function.  All calls on a device share
 * the scratch: calls in flight at the same time on one device race and give
 * undefined results -- serialise them.
 *
 * Errors: PCF_ERR_INVALID_ARG when S > PCF_STATIC_MAX_ARRAYS, n_total >
 * PCF_STATIC_MAX_KEYS, an array longer than PCF_STATIC_MAX_ARRAY_KEYS or
 * offsets that break the rules above (nothing written); PCF_ERR_INVALID_KEY
 * on a NaN key (nothing written).  Returns when the sort is complete. */
#define PCF_STATIC_MAX_ARRAY_KEYS 1024u
#define PCF_STATIC_MAX_ARRAYS 65536u
#define PCF_STATIC_MAX_KEYS (1u << 22)
pcf_status pcf_sort_segmented_static(const void* d_keys_in, void* d_keys_out,
                                     const uint64_t* d_offsets, uint32_t S, uint64_t n_total,
                                     pcf_key_type kt, uint64_t seed, void* stream);

/* A batched sort captured in a CUDA graph (the batched form: one graph
 * launch runs the whole sort of pcf_sort_segmented -- every level's kernels,
 * copies and memsets -- with no host round trip inside).
 *
 * pcf_graph_create sorts the buffers once as pcf_sort_segmented would
 * (d_keys_in -> d_keys_out, segments h_offsets, seed + s for segment s,
 * the policy and tuning of `like`, copied), keeping the host's decision at
 * the end of each global level: the next level's plan and the buckets sent
 * to the standard sort.  It then captures the same sort into a graph.  The
 * graph keeps the buffer addresses and the segments; its own context owns
 * the scratch (about what pcf_sort_segmented would use; `like` is not
 * used after the call).  Out of place only: the key (and value) buffers in
 * and out must not overlap, and the graph never writes the input.
 *
 * pcf_graph_launch sorts the CURRENT contents of d_keys_in into d_keys_out
 * and returns when they are sorted.  It replays the graph; a guard kernel
 * at each level's end compares the device's own plan with the recorded one,
 * and on a difference every later kernel of the graph returns at once and
 * the call sorts the input again without the graph (*replayed = 0).  The
 * graph keeps its capture, unless the plan of this input is the one the
 * previous miss met too: then it captures that plan instead.  After a miss
 * the next launch sorts without the graph first and replays again once an
 * input takes the captured plan, so inputs whose plans keep changing cost
 * one plain sort each.  The output is the same either way (the unique
 * sorted order).  A sort whose recording sent buckets to the
 * standard sort (duplicate-heavy input; its rounds are planned on the host)
 * is not captured: its launches sort without the graph.
 *
 * Errors as pcf_sort_segmented (a NaN key: PCF_ERR_INVALID_KEY, output not
 * written).  One graph must not be launched from two threads at once. */
typedef struct pcf_graph pcf_graph;
pcf_status pcf_graph_create(pcf_graph** out, const pcf_ctx* like, const void* d_keys_in,
                            const uint32_t* d_vals_in, void* d_keys_out, uint32_t* d_vals_out,
                            const uint64_t* h_offsets, uint32_t S, pcf_key_type kt,
                            uint64_t seed, void* stream);
/* replayed (may be NULL): 1 when the graph did the sort, 0 when it ran
 * without the graph */
pcf_status pcf_graph_launch(pcf_graph* g, void* stream, int* replayed);
/* captured: whether the graph holds a capture; replays / eager_runs: the
 * launches it replayed, the sorts it ran without the graph (creation
 * included).  Any output pointer may be NULL. */
pcf_status pcf_graph_info(const pcf_graph* g, int* captured, uint64_t* replays,
                          uint64_t* eager_runs);
/* Frees the graph and its context.  NULL is accepted. */
pcf_status pcf_graph_destroy(pcf_graph* g);

/* End-to-end form on HOST buffers: copies h_keys (n keys, ideally pinned)
 * to the device, sorts, and copies the result back into h_keys. */
pcf_status pcf_sort_keys_host(pcf_ctx* ctx, void* h_keys, uint64_t n, pcf_key_type kt,
                              uint64_t seed, void* stream);

/* Several arrays on HOST buffers: array i (ns[i] keys at h_keys[i], sorted in
 * place, ideally pinned) is sorted exactly as pcf_sort_keys_host would sort
 * it with seed + i.  The library uploads array i + 1 and downloads array
 * i - 1 on two copy streams of its own while array i is sorted on `stream`
 * (three device slots of max ns[i] keys, kept by the context).  Returns when
 * every array is back on the host; on an error no copy is left in flight and
 * the arrays after the failing one are unspecified. */
pcf_status pcf_sort_keys_host_batch(pcf_ctx* ctx, void* const* h_keys, const uint64_t* ns,
                                    uint32_t count, pcf_key_type kt, uint64_t seed,
                                    void* stream);

/* Level-0 model-based bucketing only (Alg. 1's bucketing step with the PCF
 * model of Sec. 3.3), with alpha, beta, gamma given instead of the policy's:
 * the experiment of Sec. 4.2 that checks Lemma pcf-divide-success-prob
 * (bucketing fails when some bucket holds more than delta keys).  Array s is
 * keys [h_offsets[s], h_offsets[s+1]) of d_keys (S+1 non-decreasing HOST
 * offsets, h_offsets[0] = 0, every array at least 2 keys), sampled exactly
 * as pcf_sort_segmented samples its level 0 (seed + s).
 *   h_max[s]  (HOST, S entries): max_j |c_j| over its gamma + 1 buckets; n_s
 *             when the array is not bucketed (one value, or a degenerate
 *             range: Alg. 1 sends it to Standard-Sort whole).
 *   d_counts  (DEVICE, optional, S x (gamma + 1) u32, array-major): the bucket
 *             sizes |c_0| .. |c_gamma| of each bucketed array (zeros for the
 *             others); NULL uses context scratch.
 * Limits: 1 <= alpha < 2^32, 1 <= beta < 2^32 - 1, 1 <= gamma < 2^24.  Keys
 * are only read.  PCF_ERR_INVALID_KEY on a NaN key. */
pcf_status pcf_bucket_sizes(pcf_ctx* ctx, const void* d_keys, const uint64_t* h_offsets,
                            uint32_t S, pcf_key_type kt, uint64_t seed, uint64_t alpha,
                            uint64_t beta, uint64_t gamma, uint32_t* d_counts, uint64_t* h_max,
                            void* stream);

/* Device copy bandwidth with the passes' access pattern (16-byte loads and
 * stores, grid-stride, each byte read and written once): one untimed copy,
 * then `reps` copies of `bytes` from d_src to d_dst (device buffers, 16-byte
 * aligned, not overlapping; bytes a non-zero multiple of 16), timed with CUDA
 * events on `stream`.  *gb_per_s = 2 * bytes * reps / time.  A reference for
 * the passes' roofline measured in the same run. */
pcf_status pcf_copy_bandwidth(pcf_ctx* ctx, const void* d_src, void* d_dst, uint64_t bytes,
                              uint32_t reps, void* stream, double* gb_per_s);

/* Stage timing of the last sort (milliseconds between CUDA events recorded
 * on the sort's stream) when enabled with pcf_ctx_enable_timing(ctx, 1):
 * [0] range (k_range + k_model), [1] sample + PCF table (k_sample),
 * [2] pass-1 histogram + scan, [3] pass-1 scatter (k_scatter1),
 * [4] pass-2 groups + histogram + scans, [5] pass-2 scatter (k_scatter2),
 * [6] buckets finished on chip (k_buckets + k_leaf), [7] standard-sort
 * fallback.  Events only; the call synchronises at its end either way. */
pcf_status pcf_ctx_enable_timing(pcf_ctx* ctx, int on);
pcf_status pcf_ctx_stage_ms(const pcf_ctx* ctx, float out[8]);

/* Text of a status code (static storage). */
const char* pcf_status_string(pcf_status s);
/* The last CUDA error string seen by this context ("" if none). */
const char* pcf_last_cuda_error(const pcf_ctx* ctx);

/* Library version: major * 10000 + minor * 100 + patch. */
uint32_t pcf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PCFSORT_H */

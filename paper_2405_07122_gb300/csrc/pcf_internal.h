// pcf_internal.h -- work descriptors shared by the kernels and the host
// driver of the PCF Learned Sort library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pcf_common.cuh"

namespace pcf {

// Status bits written by kernels into the context's device status word.
enum : uint32_t {
  STATUS_NAN = 1u,       // a NaN key was seen (binary64 keys)
  STATUS_TIMEOUT = 2u,   // a bounded wait gave up
  STATUS_INTERNAL = 4u,  // an internal capacity check failed
  STATUS_BOUNDS = 8u,    // a checked build caught an index out of bounds
  STATUS_REPLAN = 16u,   // a replayed sort graph met a plan other than its recording
  STATUS_ABORT = STATUS_NAN | STATUS_TIMEOUT | STATUS_INTERNAL | STATUS_BOUNDS | STATUS_REPLAN,
};

// The device-side gate of a sort: each kernel of a level returns before any
// other access once the status word holds an abort bit (a NaN key, a failed
// wait or check, a replayed graph whose plan no longer holds).  Nothing is
// written after the sort has failed, with no host round trip between the
// range pass that finds a NaN and the kernels that write the output.  The
// word changes only between launches (or, for NaN and timeouts, inside the
// launch that finds them), and kernel boundaries order it.
__device__ __forceinline__ bool pcf_aborted(const uint32_t* status) {
  return status && (*reinterpret_cast<const volatile uint32_t*>(status) & STATUS_ABORT) != 0;
}

// The status buffer of a sort (64 bytes, zeroed at the call's start):
//   [0]  u32 status word (STATUS_*)
//   [8]  u64 key-buffer length for the checked build's index checks
//   [16] u64 x 3 counters of Alg. 1's decisions (DecisionCounters)
// The counters record what the sort decided, for comparison with the
// oracle: every bucket whose size reached the failure guard |c| >= delta
// (any level, on chip included) and its keys, and every Learned-Sort call
// that bucketed its input (a model was built and the keys were appended).
struct DecisionCounters {
  unsigned long long guard_buckets, guard_keys, bucketings;
};
__device__ __forceinline__ DecisionCounters* pcf_counters(const uint32_t* status) {
  return reinterpret_cast<DecisionCounters*>(const_cast<uint32_t*>(status) + 4);
}

// SEG_NEEDRANGE: the samples' range (R14) was equal or degenerate; the
// array's own range decides
enum : uint32_t { SEG_BUCKET = 0, SEG_SINGLE = 1, SEG_DEGEN = 2, SEG_NEEDRANGE = 3 };

// One (sub)array bucketed by a global level (Algorithm 1, one call of
// Learned-Sort with its own model).  Host-planned fields first.
struct Seg {
  uint64_t off;     // offset of its first key in the key buffers
  uint64_t n;       // number of keys
  uint64_t start;   // offset inside the caller's array (keys the sample stream)
  uint64_t seed;    // the caller's seed for this array
  uint32_t depth;   // recursion depth (0 = the caller's array)
  uint32_t status;  // SEG_* (set on the device from the range)
  uint32_t alpha, beta, gamma, delta;
  uint32_t b1, b2;  // bucket-id bits scattered by pass 1 / pass 2 (b1 + b2 = bits of gamma)
  uint64_t T_off;   // its table (beta + 1 u32) in the table pool
  uint64_t cbase1;  // its pass-1 count block (2^b1 x tiles1) in the pass-1 matrix
  uint64_t key_prefix;  // sum of n over the earlier segments of the level
  uint32_t tiles1;      // count tiles of pass 1
  uint32_t tbase;       // inclusive scan of the table pool before this segment
  uint64_t group_base;  // index of its first pass-1 group
  uint64_t bucket_base; // index of its first bucket (gamma + 1 of them)
  uint64_t ord_lo, ord_hi;  // range (total-order keys), reduced on the device
  BinModel bm;
};

// A pass-2 segment: the keys of one pass-1 digit of one Seg.
struct Group {
  uint64_t off;         // key offset of its first key
  uint64_t key_prefix;  // compacted offset (sum of sizes of earlier groups)
  uint64_t cbase;       // its count block (2^b2 x tiles) in the pass-2 matrix
  uint32_t n;
  uint32_t tiles;
  uint32_t seg;
  uint32_t pad;
};

// Every bucket of a level, in memory order (bucket index order): written by
// k_buckets, read by the on-chip kernels and the next level's planning.
enum : uint32_t {
  BK_LEAF = 1u,  // finished on chip
  BK_STD = 2u,   // ... by Standard-Sort (|c| >= delta or |c| < tau)
};
struct BRec {
  uint32_t off;    // absolute offset of its first key
  uint32_t n;      // size
  uint32_t kind;   // BK_* (0: empty, already finished, or handled elsewhere)
  uint32_t depth;  // recursion depth of the Learned-Sort call on this bucket
  uint64_t start;  // offset inside the caller's array
  uint64_t seed;
};

// A bucket for the standard sort (failure guard |c| >= delta, or a
// degenerate range).
struct FbItem {
  uint64_t off;
  uint64_t n;
};

// Device-side plan of the next level: one row per (sub)array, these count
// columns, scanned into bases.
enum : uint32_t {
  PC_RANGE = 0,  // range tiles
  PC_K1,         // sample CTAs
  PC_TILES1,     // pass-1 count tiles
  PC_GROUPS,     // pass-1 groups
  PC_BUCKETS,    // gamma + 1
  PC_TPOOL,      // beta + 1
  PC_CMAT1,      // pass-1 count entries
  PC_CMAT2,      // pass-2 count entries (bound)
  PC_TILES2,     // pass-2 tiles (bound)
  PC_NCOL
};

struct PlanTotals {
  uint64_t col[PC_NCOL];  // column totals
  uint64_t n_keys;        // sum of n
  uint64_t lo, hi;        // smallest offset, largest end
  uint32_t S;             // (sub)arrays
  uint32_t dmax1, dmax2, two_pass;
};

// Where a level's plan lives on the device.
struct DevPlan {
  Seg* segs;
  uint32_t* rb;  // range tile bases [S+1]
  uint32_t* k1;  // sample CTA bases [S+1]
  uint32_t* t1;  // pass-1 tile bases [S+1]
  uint64_t* gb;  // group bases [S+1]
  uint64_t* bb;  // bucket bases [S+1]
};

// Counters written by k_buckets.
struct LevelOut {
  uint32_t n_leaf;
  uint32_t n_next;
  uint32_t n_fb;
  uint32_t n_flag;    // buckets flagged for the next global level
  uint64_t flag_n;    // length of the flag scan: the buckets when any is flagged, else 0
  uint32_t max_fb_n;  // largest standard-sort bucket (sizes the merge passes)
  uint32_t leaf_cursor; // work counter of the leaf kernel
  uint64_t mid_keys;  // keys finished by k_mid (their own Learned-Sort call on chip)
  PlanTotals plan;    // the next level's plan (device-built)
};

struct KeyBufs {
  const uint64_t* src;  // where the level reads
  uint64_t* tmp;        // pass-1 target
  uint64_t* out;        // pass-2 target
  const uint32_t* src_v;
  uint32_t* tmp_v;
  uint32_t* out_v;
  uint16_t* tmp_aux;    // low bucket-id digit carried from pass 1 to pass 2
  const uint32_t* jbuf; // bucket id of every key of the level (written by k_hist1)
};


// ---- bulk (1-D tensor-memory-accelerator) copies into shared memory ----
// A CTA stages a run of keys by one cp.async.bulk that completes on an
// mbarrier; the consumers wait on the barrier's phase.  Every wait is
// bounded by the global timer, so a copy that never lands ends the kernel
// with STATUS_TIMEOUT instead of hanging it.
// bounded waits on the staging barrier: about two seconds of the global
// timer (each try_wait suspends for a hardware-chosen while)
constexpr uint64_t kBulkWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  // make the initialised barrier visible to the bulk-copy (async) proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// one arrival that also expects `bytes` of bulk-copy transactions
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// waits (bounded) for the barrier's phase `parity` to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it >= (1u << 30)) return false;
    if ((it & 63u) == 0) {
      const uint64_t t = global_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > kBulkWaitNs) return false;
    }
  }
}


// ---- checked builds (-DPCF_CHECKED) ----
// Index checks in place of a memory checker: a computed index is tested
// against its buffer before the access; one out of bounds sets STATUS_BOUNDS
// and the access is skipped (no trap, no fault).  The key buffers' length
// is read from the status buffer (u64 at byte 8, written at each call's
// start).  In normal builds every check is `true`.
#ifdef PCF_CHECKED
__device__ __forceinline__ bool pcf_in_bounds(uint64_t i, uint64_t n, uint32_t* status) {
  if (i < n) return true;
  if (status) atomicOr(status, (uint32_t)STATUS_BOUNDS);
  return false;
}
__device__ __forceinline__ uint64_t pcf_key_limit(const uint32_t* status) {
  const uint64_t lim = status ? *reinterpret_cast<const volatile uint64_t*>(status + 2) : 0ull;
  return lim ? lim : ~0ull;  // 0: not set by this entry point
}
#define PCF_IN(i, n, st) pcf_in_bounds((uint64_t)(i), (uint64_t)(n), (st))
#define PCF_IN_KEYS(i, st) pcf_in_bounds((uint64_t)(i), pcf_key_limit(st), (st))
#else
#define PCF_IN(i, n, st) true
#define PCF_IN_KEYS(i, st) true
#endif

// ---- kernel launchers ----
struct LaunchCfg {
  cudaStream_t stream;
  uint32_t kt;
  uint32_t model = MODEL_PCF;  // the policy's CDF model
  uint32_t range_mode = RANGE_ARRAY;  // ... and range
  bool pairs;
  // keys-only leaf buckets: finished by the block-local Standard-Sort
  // (k_leaf_sort) rather than by further Learned-Sort steps on chip
  bool leaf_sort = false;
  uint32_t* status;  // device status word
  uint64_t* launches;  // host counter of kernel launches (may be null)
};

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, once per device and kernel.  The limit only ever grows, so
// callers on several host threads (each with its own context) never lower
// it under one another's launches; a launch then needs only its own size.
cudaError_t allow_max_smem(const void* kernel);

inline void count_launch(const LaunchCfg& c, uint64_t k = 1) {
  if (c.launches) *c.launches += k;
}

// Tile sizes (keys).
constexpr uint32_t kRangeTile = 16384;
constexpr uint32_t kSamplesPerCta = 4096;
constexpr uint32_t kScatterSub = 4096;  // keys staged in shared memory at once
constexpr uint32_t kScanTile = 4096;    // entries per decoupled-lookback tile
constexpr uint32_t kMergeTile = 2048;   // keys per block-sorted run
constexpr uint32_t kMaxDigitBits = 12;

// a replayed graph's end-of-level check against its recording (STATUS_REPLAN)
cudaError_t launch_guard(const LaunchCfg& c, const LevelOut* dev, const LevelOut* rec);
cudaError_t launch_guard_list(const LaunchCfg& c, const FbItem* dev, const FbItem* rec,
                              uint32_t n);
cudaError_t launch_guard_words(const LaunchCfg& c, const void* dev, const void* rec,
                               uint64_t n_words);
// only_status: reduce only the segments in that status (~0u: all)
cudaError_t launch_range(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* range_base,
                         uint32_t n_tiles, const uint64_t* keys, bool check_nan,
                         uint32_t only_status = ~0u);
// pass 0: the range reduced by launch_range; 1: the samples' range (R14),
// SEG_NEEDRANGE where it is equal or degenerate; 2: those segments again,
// from their array range
cudaError_t launch_model(const LaunchCfg& c, Seg* segs, uint32_t S, uint32_t pass = 0);
// min and max of every segment's alpha samples into its range fields
cudaError_t launch_sample_range(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* k1_base,
                                uint32_t n_ctas, const uint64_t* keys);
cudaError_t launch_sample(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* k1_base,
                          uint32_t n_ctas, const uint64_t* keys, uint32_t* tpool);
// cumulative counts b (inclusive scan of the whole pool) + per-segment bases
cudaError_t launch_table(const LaunchCfg& c, Seg* segs, uint32_t S, uint32_t* tpool,
                         uint64_t pool_n, uint64_t* status_words, uint32_t* tile_counter,
                         uint64_t spin_limit);
// check_nan: flag NaN keys (a sample range has no full range pass to do it)
cudaError_t launch_hist1(const LaunchCfg& c, const Seg* segs, uint32_t S, const uint32_t* tile_base,
                         uint32_t n_tiles, uint32_t tile_keys, const uint64_t* keys,
                         const uint32_t* tpool, uint32_t* cmat, uint32_t dmax, uint32_t* jout,
                         bool check_nan = false);
// Level-0 bucket sizes of every segment (ids from k_hist1's jbuf): counts
// (zeroed by the caller) at bucket_base, and out_max[s] = max_j |c_j| (n
// for a segment that was not bucketed).
cudaError_t launch_bucket_sizes(const LaunchCfg& c, const Seg* segs, uint32_t S,
                                const uint32_t* tile_base, uint32_t n_tiles, uint32_t tile_keys,
                                const uint32_t* jbuf, uint32_t* counts, uint64_t* out_max);
// 16-byte device-to-device copy of n16 words (the copy bandwidth probe)
cudaError_t launch_copy128(cudaStream_t st, const void* src, void* dst, uint64_t n16,
                           uint32_t grid);
// Small host <-> device transfers of a sort, copied by the SMs through the
// device view of pinned host memory.  A copy-engine transfer would queue
// behind any large copy in the same direction already issued on another
// stream (a caller's bulk upload or download), stalling the sort for its
// whole duration.
cudaError_t launch_xfer(cudaStream_t st, void* dst, const void* src, size_t bytes);
cudaError_t launch_scan(const LaunchCfg& c, uint32_t* data, uint64_t n, const uint64_t* n_dev,
                        uint64_t* status_words, uint32_t* tile_counter, uint32_t withhold,
                        uint64_t spin_limit, uint64_t* total_out, bool inclusive = false);
cudaError_t launch_scatter1(const LaunchCfg& c, const Seg* segs, uint32_t S,
                            const uint32_t* tile_base, uint32_t n_tiles, uint32_t tile_keys,
                            const KeyBufs& kb, const uint32_t* tpool, const uint32_t* cmat,
                            uint32_t dmax);
cudaError_t launch_groups(const LaunchCfg& c, const Seg* segs, uint32_t S,
                          const uint64_t* group_base_dev, uint64_t n_groups, const uint32_t* cmat1,
                          uint32_t tile_keys, Group* groups, uint32_t* g_tiles,
                          uint32_t* g_centries);
cudaError_t launch_group_bases(const LaunchCfg& c, Group* groups, uint64_t n_groups,
                               const uint32_t* g_centries_scan);
cudaError_t launch_hist2(const LaunchCfg& c, const Group* groups, uint32_t n_groups,
                         const Seg* segs, const uint32_t* g_tile_scan, const uint64_t* total_tiles,
                         uint32_t n_tiles_bound, uint32_t tile_keys, const uint16_t* aux,
                         uint32_t* cmat2, uint32_t dmax);
cudaError_t launch_scatter2(const LaunchCfg& c, const Group* groups, uint32_t n_groups,
                            const Seg* segs, const uint32_t* g_tile_scan,
                            const uint64_t* total_tiles, uint32_t n_tiles_bound,
                            uint32_t tile_keys, const KeyBufs& kb, const uint32_t* cmat2,
                            uint32_t dmax);
cudaError_t launch_buckets(const LaunchCfg& c, const Seg* segs, uint32_t S, uint64_t n_buckets,
                           const uint64_t* bucket_base, const Group* groups,
                           const uint32_t* cmat1, const uint32_t* cmat2, bool two_pass,
                           uint32_t leaf_cap, uint32_t tau, const uint64_t* X, const uint32_t* Xv,
                           uint64_t* out_k, uint32_t* out_v, BRec* brec, uint32_t* next_flag,
                           FbItem* fb, LevelOut* lo, uint32_t max_items,
                           uint2* leaf_lists = nullptr, uint32_t* leaf_counts = nullptr,
                           uint32_t leaf_classes = 0, uint32_t* mid_list = nullptr,
                           uint32_t* mid_count = nullptr);
// builds the next level's plan from the flagged buckets (next_flag[B] = 1
// for a bucket of the next level; scanned in place), s_max rows at most;
// n_flagged receives the number of (sub)arrays
cudaError_t launch_plan_next(const LaunchCfg& c, const BRec* brec, uint32_t* next_flag,
                             uint64_t n_buckets, uint32_t s_max, Policy P, uint32_t dbits,
                             uint32_t tile_keys, const DevPlan& out, uint32_t* cols,
                             uint32_t* block_sums, LevelOut* lo, uint64_t* sw,
                             uint32_t* tile_counter, uint64_t spin_limit, uint64_t* n_flagged);
cudaError_t launch_seg_status_lists(const LaunchCfg& c, const Seg* segs, uint32_t S,
                                    FbItem* fb, LevelOut* lo, uint32_t max_items);
// copies the segments whose status is in status_mask (bit per SEG_*), or,
// with kCopyOneDigit, the bucketed segments whose bucket id has one digit
constexpr uint32_t kCopyOneDigit = 0x100u;
cudaError_t launch_copy_segs(const LaunchCfg& c, const Seg* segs, uint32_t S,
                             const uint32_t* range_base, uint32_t n_tiles, const uint64_t* src,
                             uint64_t* dst, const uint32_t* src_v, uint32_t* dst_v,
                             uint32_t status_mask);
// on-chip finish, one warp per bucket: every BK_LEAF record of br[0..nb)
// (any order), keys X -> out at the record's offset
struct OnchipGeo {
  uint32_t capw;   // keys of a warp's slice (the largest bucket it takes)
  uint32_t tmax;   // beta + 1 bound
  uint32_t kmax;   // gamma + 1 bound
  uint32_t smax;   // pending calls per warp
  uint32_t bytes;  // shared memory of one warp's slice
};
OnchipGeo onchip_geometry(uint32_t capw, const Policy& P, bool pairs);
// Size classes of the on-chip finish: (0, 256], (256, 512], ..., up to
// 8192 keys; onchip_classes(cap) of them are used below leaf_cap = cap.
constexpr uint32_t kMaxClasses = 6;
uint32_t onchip_classes(uint32_t leaf_cap);
// A failure-guard bucket (|c| >= delta) is finished on chip only up to this
// many keys when one warp runs its Standard-Sort (the Learned-Sort steps on
// chip); larger ones go to the fallback, where the whole device sorts them.
// The block-local leaf sort takes failure-guard buckets up to leaf_cap
// (Standard-Sort is any sort, Sec. 3.1).
constexpr uint32_t kStdLeafMax = 1024;
__host__ __device__ inline uint32_t guard_leaf_max(uint32_t leaf_cap, bool block_local) {
  return block_local ? leaf_cap : (leaf_cap < kStdLeafMax ? leaf_cap : kStdLeafMax);
}
// Runs of 32 adjacent leaf buckets of at most this many keys each are
// listed as one leaf record (buckets are ordered, so the run sorted as one
// piece is the buckets sorted one after another).
constexpr uint32_t kRunBucket = 64;
// Mid-size (sub)arrays (leaf_cap, kMidCap]: one Learned-Sort call per CTA
// (k_mid) instead of a further global level; kMidTab bounds beta + 1 and
// gamma + 1 (kMidCap^(3/4) + 1 under the paper's policy).
constexpr uint32_t kMidCap = 32768;
constexpr uint32_t kMidTab = 2056;
// upper bound on the leaf records k_mid lists for a level of n_level keys:
// per class (q >= 1: records of more than 2^(q+5) keys; q = 0: at most one
// record per bucket of the mid (sub)arrays, each more than leaf_cap keys)
inline uint64_t mid_class_cap(uint32_t q, uint64_t n_level, uint32_t leaf_cap) {
  if (q > 0) return (n_level >> (q + 5)) + 1;
  const uint64_t g = (n_level / ((uint64_t)leaf_cap + 1) + 1) * kMidTab;
  return (g < n_level ? g : n_level) + 1;
}
// The block-local sort's classes (0, 64], (64, 128], (128, 256], (256, 512],
// ... up to leaf_cap: leaf_sort_classes(cap) of them, at most kMaxLeafClasses.
constexpr uint32_t kMaxLeafClasses = 8;
uint32_t leaf_sort_classes(uint32_t leaf_cap);
__device__ __forceinline__ uint32_t leaf_size_class(uint32_t n) {
  return n <= 64 ? 0u : (uint32_t)(32 - __clz((int)(n - 1))) - 6u;
}
// Mid-size buckets mid_list[0 .. *mid_count) (bucket indices into brec,
// keys in X): each one Learned-Sort call by one CTA; its buckets appended
// in Y and listed for the block-local sort (lists: class q at
// class_base[q], counts[q]); next_flag[B] = 1 where the call leaves the
// bucket to the next global level.  The default policy only (PCF model,
// array range).
struct MidLists {
  uint64_t base[kMaxLeafClasses];
  uint64_t cap[kMaxLeafClasses];
};
cudaError_t launch_mid(const LaunchCfg& c, const uint32_t* mid_list, const uint32_t* mid_count,
                       const BRec* brec, const uint64_t* X, uint64_t* Y, uint64_t* out,
                       uint32_t* next_flag, uint2* lists, const MidLists& ml,
                       uint32_t* list_counts, uint32_t leaf_classes, uint32_t leaf_cap,
                       const Policy& P, LevelOut* lo);
// The largest bucket finished on chip: leaf_cap (key-value sorts at most
// 1024), halved until the policy's slice fits one block's shared memory.
uint32_t onchip_cap(uint32_t leaf_cap, const Policy& P, bool pairs);
// lists: (block-local sort: leaf_sort_classes, else onchip_classes)(leaf_cap)
// x nb x 8 bytes of scratch (u32 record indices, or (offset, size) pairs
// for the block-local sort); counts: kMaxLeafClasses u32
// prelisted: the block-local sort's class lists and counts were already
// written (by k_buckets), so they are not built from the records again
// class_base: the block-local sort's class lists at these record offsets
// (prelisted lists only; nullptr: class q at q * nb); class_stream: the
// stream of each class's launch (block-local sort; nullptr: c.stream)
cudaError_t launch_onchip(const LaunchCfg& c, const BRec* br, uint32_t nb, uint32_t leaf_cap,
                          const uint64_t* X, const uint32_t* Xv, uint64_t* out, uint32_t* out_v,
                          Policy P, const uint16_t* ptab, uint32_t* lists, uint32_t* counts,
                          bool prelisted = false, const uint64_t* class_base = nullptr,
                          const cudaStream_t* class_stream = nullptr);
cudaError_t launch_fb_range(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                            const uint32_t* tile_base, uint32_t n_tiles, const uint64_t* keys,
                            uint64_t* ord_lohi);
// Duplicate-heavy items: a value that holds at least a quarter of a sample
// of kModeSample keys marks the item dominant (pivot[i] = that total-order
// value, dom[i] = 1; items with one value are never dominant).
constexpr uint32_t kModeSample = 256;
cudaError_t launch_fb_mode(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint64_t* keys, const uint64_t* ord_lohi, uint64_t* pivot,
                           uint32_t* dom);
// Stable three-way split of every item around its pivot (below, equal,
// above), keys -> dst at the item's own offsets, in kMergeTile tiles:
// counting writes cnt[3][n_tiles + 1] (the last column zero), the caller
// scans the rows (exclusive; one scan of all three rows in a row serves, as
// only differences within a row are used), then the scatter places every
// key.  item_cnt[3 i + p] (zeroed by the caller) receives item i's part sizes.
cudaError_t launch_fb_part_count(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                                 const uint32_t* mtile_base, uint32_t n_mtiles,
                                 const uint64_t* keys, const uint64_t* pivot, uint32_t* cnt,
                                 uint64_t* item_cnt);
cudaError_t launch_fb_part_scatter(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                                   const uint32_t* mtile_base, uint32_t n_mtiles,
                                   const uint64_t* keys, const uint32_t* vals,
                                   const uint64_t* pivot, const uint32_t* cnt_ex, uint64_t* dst,
                                   uint32_t* dst_v);
// copies every item's keys (and values) src -> dst
cudaError_t launch_fb_move(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint32_t* mtile_base, uint32_t n_mtiles, const uint64_t* src,
                           uint64_t* dst, const uint32_t* src_v, uint32_t* dst_v);
// sorts the items in `keys` (scratch `tmp`), leaving the result in `final`
cudaError_t launch_fb_sort(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint32_t* mtile_base, uint32_t n_mtiles, uint64_t max_n,
                           const uint64_t* ord_lohi, uint64_t* keys, uint64_t* tmp,
                           uint32_t* vals, uint32_t* tmp_v, uint64_t* final_k,
                           uint32_t* final_v);

}  // namespace pcf

// pcf_host.cu -- host driver and C ABI of the PCF Learned Sort library.
//
// Algorithm 1 of Sato & Matsui (TMLR 2025) is run level by level: every
// (sub)array too large for one warp's shared memory is bucketed by a global
// level (range -> PCF model -> bucket ids -> two stable digit scatters), its
// buckets are finished on chip when they fit, recursed at the next level
// when they do not, and sent to the standard sort when |c| >= delta.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>
#include <map>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pcfsort.h"
#include "../../include/pcfsort_debug.h"
#include "pcf_internal.h"


using namespace pcf;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

struct HostBuf {  // pinned staging
  void* p = nullptr;
  void* dp = nullptr;  // its device view
  size_t cap = 0;
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
};

// Side streams that run beside the caller's within one level (the mid-size
// Learned-Sort calls and their leaf sort; the level's leaf classes above 512
// keys), all on disjoint keys, forked and joined by events (created on first
// use, on the context's device; a capture takes them into the graph).
struct SideStream {
  cudaStream_t st = nullptr, st2 = nullptr;  // the mid calls; the larger leaf classes
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
  bool ready = false;
  cudaError_t init() {
    if (ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&join2, cudaEventDisableTiming);
    ready = !e;
    return e;
  }
  ~SideStream() {
    if (!ready) return;
    cudaStreamDestroy(st);
    cudaStreamDestroy(st2);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    cudaEventDestroy(join2);
  }
};

// Copy streams and events of the pipelined host-buffer entry point (created
// on first use, on the context's device).
constexpr int kPipeSlots = 3;
struct CopyPipe {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t loaded[kPipeSlots], sorted[kPipeSlots], stored[kPipeSlots];
  bool ready = false;
  cudaError_t init() {
    if (ready) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking);
    for (int i = 0; i < kPipeSlots && !e; ++i) {
      e = cudaEventCreateWithFlags(&loaded[i], cudaEventDisableTiming);
      if (!e) e = cudaEventCreateWithFlags(&sorted[i], cudaEventDisableTiming);
      if (!e) e = cudaEventCreateWithFlags(&stored[i], cudaEventDisableTiming);
    }
    ready = !e;
    return e;
  }
  ~CopyPipe() {
    if (!ready) return;
    cudaStreamDestroy(in);
    cudaStreamDestroy(out);
    for (int i = 0; i < kPipeSlots; ++i) {
      cudaEventDestroy(loaded[i]);
      cudaEventDestroy(sorted[i]);
      cudaEventDestroy(stored[i]);
    }
  }
};

}  // namespace

namespace {
// alpha..delta of a (sub)array, cached for n < 2^16 (levels can hold tens of
// thousands of segments)
struct ParamCache {
  uint64_t key = ~0ull;
  std::vector<Params> small;
  const Params& get(const Policy& P, uint64_t n, Params& tmp) {
    const uint64_t k = ((uint64_t)P.a_num << 32) ^ ((uint64_t)P.b_num << 24) ^
                       ((uint64_t)P.c_num << 16) ^ ((uint64_t)P.d_num << 8) ^ P.den;
    if (k != key) {
      key = k;
      small.assign(1u << 16, Params{0, 0, 0, 0});
    }
    if (n < (1u << 16)) {
      Params& c = small[n];
      if (c.alpha == 0) c = params_of(P, n);
      return c;
    }
    tmp = params_of(P, n);
    return tmp;
  }
};

}  // namespace

struct pcf_ctx {
  int device = 0;
  int num_sms = 0;
  Policy policy{3, 3, 3, 3, 4, MODEL_PCF, 100, RANGE_ARRAY, 0};
  pcf_tuning tuning{11, 14, 8192, 1};
  std::string last_err;
  pcf_call_stats stats{};
  bool timing = false;
  float stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // workspace
  DevBuf tmp_k, tmp_v, tmp_aux, host_keys;
  DevBuf segs, bases, tpool, done, cmat1, cmat2, sw, groups, gtiles, gcent, gtot;
  DevBuf leaf, next, fb, lout, status, misc, fb_items, fb_bases, fb_lohi, small_items;
  DevBuf segs_b, pcols, pbsums;  // the other level's plan, its count columns
  DevBuf olist;                  // on-chip buckets listed by size class
  DevBuf mid;                    // k_mid's work list and its leaf records
  DevBuf jbuf;                   // bucket id of every key of a level
  DevBuf small_segs;             // range records of the on-chip arrays (level 0)
  DevBuf fb_cnt;                 // per-tile part counts of the three-way splits
  DevBuf bcounts, bmax;          // bucket sizes of the bucketing-only entry point
  HostBuf h_stage, h_lout, h_status, h_items;
  HostBuf h_stage_small;  // range records of the on-chip arrays (level 0)
  HostBuf h_fb;           // fallback items and their tables, both ways
  HostBuf h_offs;         // device offsets of pcf_sort_segmented_dev, read back
  pcf_status last_status = PCF_OK;  // of the last sort (pcf_ctx_sync)
  DevBuf ptab;            // alpha..delta for n = 0..leaf_cap (u16 x 4)
  uint64_t ptab_key = 0;  // policy/cap the table was built for
  ParamCache pcache;
  DevBuf pipe_keys;  // kPipeSlots arrays of the pipelined host entry point
  CopyPipe pipe;
  SideStream side;   // the mid calls beside the level's leaf sort
};

cudaError_t pcf::allow_max_smem(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({kernel, dev});
  if (it != done.end()) return it->second;
  int optin = 0;
  cudaFuncAttributes fa;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (!e) e = cudaFuncGetAttributes(&fa, kernel);
  // the limit covers the dynamic part; the kernel's static shared memory
  // takes the rest of the block's opt-in maximum
  if (!e)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  done[{kernel, dev}] = e;
  return e;
}

namespace {

pcf_status cuda_fail(pcf_ctx* c, cudaError_t e) {
  c->last_err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PCF_ERR_OOM : PCF_ERR_CUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_); \
  } while (0)

// NVTX range over a scope (a profiler's timeline shows the sort's levels
// and stages; without a tool attached it costs a few nanoseconds)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Test hook: the allocation that many device allocations from now fails
// (host side, as cudaMalloc would report exhausted memory); -1: never.
thread_local int64_t g_fail_alloc_after = -1;

// Set while this thread captures a sort graph: the capture reuses the
// buffers of the run it replays, and a buffer that would have to grow
// fails the capture instead (an allocation is not a stream operation).
thread_local bool g_capturing = false;

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
  if (g_capturing) return cudaErrorStreamCaptureUnsupported;
  if (g_fail_alloc_after >= 0 && g_fail_alloc_after-- == 0) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    return cudaErrorMemoryAllocation;
  }
  if (b.p) {
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return e;
    }
    want = bytes;
  }
  b.cap = want;
  return cudaSuccess;
}

cudaError_t ensure_host(HostBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return cudaSuccess;
  if (g_capturing) return cudaErrorStreamCaptureUnsupported;
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.cap = 0;
  b.dp = nullptr;
  size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMallocHost(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  e = cudaHostGetDevicePointer(&b.dp, b.p, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(b.p);
    b.p = b.dp = nullptr;
    return e;
  }
  b.cap = want;
  return cudaSuccess;
}

// Device view of a pointer into a pinned staging buffer.
void* dview(const HostBuf& b, const void* hp) {
  return (char*)b.dp + ((const char*)hp - (const char*)b.p);
}

template <typename T>
T* as(DevBuf& b) {
  return (T*)b.p;
}

bool policy_ok(const Policy& P) {
  if (P.den < 1 || P.den > 4) return false;
  if (P.a_num < 1 || P.a_num > P.den || P.b_num < 1 || P.b_num > P.den) return false;
  if (P.c_num < 1 || P.c_num > P.den) return false;
  if (P.d_num < 1 || P.d_num >= P.den) return false;
  if (P.tau < 16 || P.tau > 65535) return false;
  if (P.model != MODEL_PCF && P.model != MODEL_SPLINE) return false;
  if (P.range_mode != RANGE_ARRAY && P.range_mode != RANGE_SAMPLE) return false;
  return true;
}

uint32_t bits_of(uint32_t v) {  // number of bits to hold values 0..v
  uint32_t b = 0;
  while (b < 32 && (v >> b) != 0) ++b;
  return b;
}

struct InSeg {
  uint64_t off, n, start, seed;
  uint32_t depth;
};

struct Plan {
  std::vector<Seg> segs;
  std::vector<uint32_t> range_base, k1_base, tile1_base;
  std::vector<uint64_t> group_base, bucket_base;
  uint64_t tpool = 0, cmat1 = 0, cmat2_bound = 0, tiles2_bound = 0, n_groups = 0, n_buckets = 0;
  uint32_t dmax1 = 1, dmax2 = 1;
  bool two_pass = false;
};

// Plans one global level.  When every segment's bucket id fits one digit
// (<= max_digit_bits) the level scatters once; otherwise twice, and
// segments with a one-digit id copy themselves in the second pass.
// fixed: alpha..delta of every segment instead of the policy's (the
// bucketing-only entry point)
void plan_level(const Policy& P, const pcf_tuning& tu, ParamCache& pc,
                const std::vector<InSeg>& in, Plan& pl, const Params* fixed = nullptr) {
  const uint32_t tile_keys = 1u << tu.tile_log2;
  const uint32_t S = (uint32_t)in.size();
  const uint32_t dbits = std::min(tu.max_digit_bits, kMaxDigitBits);
  pl.segs.resize(S);
  pl.range_base.assign(S + 1, 0);
  pl.k1_base.assign(S + 1, 0);
  pl.tile1_base.assign(S + 1, 0);
  pl.group_base.assign(S + 1, 0);
  pl.bucket_base.assign(S + 1, 0);
  pl.tpool = pl.cmat1 = pl.cmat2_bound = pl.tiles2_bound = 0;
  pl.dmax1 = pl.dmax2 = 1;
  pl.two_pass = false;
  std::vector<Params> prs(S);
  for (uint32_t s = 0; s < S; ++s) {
    Params tmp;
    prs[s] = fixed ? *fixed : pc.get(P, in[s].n, tmp);
    if (std::max(1u, bits_of(prs[s].gamma)) > dbits) pl.two_pass = true;
  }
  for (uint32_t s = 0; s < S; ++s) {
    Seg g;
    memset(&g, 0, sizeof g);
    g.off = in[s].off;
    g.n = in[s].n;
    g.start = in[s].start;
    g.seed = in[s].seed;
    g.depth = in[s].depth;
    const Params& pr = prs[s];
    g.alpha = pr.alpha;
    g.beta = pr.beta;
    g.gamma = pr.gamma;
    g.delta = pr.delta;
    const uint32_t jb = std::max(1u, bits_of(pr.gamma));
    // two digits: make the low digit as wide as allowed, so that pass-2
    // groups (n / 2^b1 keys each) stay large
    uint32_t b1 = jb;
    if (jb > dbits) {
      const uint32_t b2 = std::min(dbits, jb - 1);
      b1 = std::min(jb - b2, kMaxDigitBits);
    }
    g.b1 = b1;
    g.b2 = jb - b1;
    g.T_off = pl.tpool;
    pl.tpool += (uint64_t)pr.beta + 1;
    g.tiles1 = (uint32_t)((g.n + tile_keys - 1) / tile_keys);
    g.cbase1 = pl.cmat1;
    pl.cmat1 += (uint64_t)g.tiles1 << g.b1;
    g.group_base = pl.group_base[s];
    g.bucket_base = pl.bucket_base[s];
    g.ord_lo = ~0ull;
    g.ord_hi = 0;
    g.status = SEG_BUCKET;
    pl.segs[s] = g;
    pl.range_base[s + 1] = pl.range_base[s] + (uint32_t)((g.n + kRangeTile - 1) / kRangeTile);
    pl.k1_base[s + 1] = pl.k1_base[s] + (pr.alpha + kSamplesPerCta - 1) / kSamplesPerCta;
    pl.tile1_base[s + 1] = pl.tile1_base[s] + g.tiles1;
    // one group per pass-1 digit; a one-digit id copies the segment as one group
    pl.group_base[s + 1] = pl.group_base[s] + (g.b2 ? (1ull << g.b1) : 1ull);
    pl.bucket_base[s + 1] = pl.bucket_base[s] + (uint64_t)pr.gamma + 1;
    const uint64_t t2 = g.tiles1 + (g.b2 ? (1ull << g.b1) : 1ull);
    pl.tiles2_bound += t2;
    pl.cmat2_bound += t2 << g.b2;
    pl.dmax1 = std::max(pl.dmax1, 1u << g.b1);
    pl.dmax2 = std::max(pl.dmax2, 1u << g.b2);
  }
  pl.n_groups = pl.group_base[S];
  pl.n_buckets = pl.bucket_base[S];
}

// A level's plan on the device (Seg rows and base arrays in one buffer) and
// the totals the host needs to launch the level.
struct PlanLayout {
  size_t o_rb, o_k1, o_t1, o_gb, o_bb, bytes;
};

PlanLayout plan_layout(uint64_t rows) {
  PlanLayout L;
  L.o_rb = rows * sizeof(Seg);
  L.o_k1 = L.o_rb + (rows + 1) * 4;
  L.o_t1 = L.o_k1 + (rows + 1) * 4;
  L.o_gb = (L.o_t1 + (rows + 1) * 4 + 7) & ~(size_t)7;
  L.o_bb = L.o_gb + (rows + 1) * 8;
  L.bytes = L.o_bb + (rows + 1) * 8;
  return L;
}

DevPlan dev_plan(void* base, const PlanLayout& L) {
  char* b = (char*)base;
  DevPlan d;
  d.segs = (Seg*)b;
  d.rb = (uint32_t*)(b + L.o_rb);
  d.k1 = (uint32_t*)(b + L.o_k1);
  d.t1 = (uint32_t*)(b + L.o_t1);
  d.gb = (uint64_t*)(b + L.o_gb);
  d.bb = (uint64_t*)(b + L.o_bb);
  return d;
}

struct LevelPlan {
  uint32_t S = 0;
  uint64_t n_level = 0, wb = 0, we = 0;  // keys, first offset, end
  uint32_t n_range = 0, n_k1 = 0, n_t1 = 0;
  uint64_t n_groups = 0, n_buckets = 0, tpool = 0, cmat1 = 0, cmat2_bound = 0,
           tiles2_bound = 0;
  uint32_t dmax1 = 1, dmax2 = 1;
  bool two_pass = false;
  uint32_t tile_log2 = 14;  // the level's pass-1 count tiles
  DevPlan dp{};
};

// Tiles of a level's passes: the tuning's pass-1 size (halved, down to 2^12,
// while the level would have fewer than 4 tiles per SM, so that small
// arrays still spread over the GPU) and pass-2 tiles up to 4x that, while
// they still give 4 per SM.  Level 0 only: later levels are planned on the
// device with the tuning's size.
uint32_t level0_tile_log2(const pcf_tuning& tu, uint64_t n_level, int num_sms) {
  uint32_t t = tu.tile_log2;
  while (t > 12 && (n_level >> t) < 4ull * (uint64_t)num_sms) --t;
  return t;
}
uint32_t pass2_shift(uint32_t tile_log2, uint64_t n_level, int num_sms) {
  uint32_t sh = 2;
  while (sh > 0 && (n_level >> (tile_log2 + sh)) < 4ull * (uint64_t)num_sms) --sh;
  return sh;
}

// alpha, beta, gamma, delta of every on-chip size n <= cap, so the leaf
// kernel looks them up instead of evaluating floor(n^{p/q}) per bucket.
cudaError_t ensure_ptab(pcf_ctx* ctx, cudaStream_t st) {
  const Policy& P = ctx->policy;
  const uint32_t cap = ctx->tuning.leaf_cap;
  const uint64_t key = ((uint64_t)P.a_num << 56) ^ ((uint64_t)P.b_num << 48) ^
                       ((uint64_t)P.c_num << 40) ^ ((uint64_t)P.d_num << 32) ^
                       ((uint64_t)P.den << 24) ^ ((uint64_t)cap << 8) ^ (P.tau & 0xFF) ^
                       (P.tau << 12);
  if (ctx->ptab_key == key && ctx->ptab.p) return cudaSuccess;
  std::vector<uint16_t> t((size_t)(cap + 1) * 4, 0);
  for (uint32_t n = 2; n <= cap; ++n) {
    Params pr = params_of(P, n);
    t[n * 4 + 0] = (uint16_t)pr.alpha;
    t[n * 4 + 1] = (uint16_t)pr.beta;
    t[n * 4 + 2] = (uint16_t)pr.gamma;
    t[n * 4 + 3] = (uint16_t)pr.delta;
  }
  cudaError_t e = ensure(ctx->ptab, t.size() * 2);
  if (e) return e;
  e = cudaMemcpyAsync(ctx->ptab.p, t.data(), t.size() * 2, cudaMemcpyHostToDevice, st);
  if (e) return e;
  e = cudaStreamSynchronize(st);
  if (e) return e;
  ctx->ptab_key = key;
  return cudaSuccess;
}

struct Timer {
  pcf_ctx* ctx;
  cudaStream_t st;
  cudaEvent_t ev[64];
  int n = 0;
  int stage_of[64];
  Timer(pcf_ctx* c, cudaStream_t s) : ctx(c), st(s) {
    if (ctx->timing)
      for (int i = 0; i < 64; ++i) cudaEventCreate(&ev[i]);
  }
  void mark(int stage) {
    if (!ctx->timing || n >= 64) return;
    stage_of[n] = stage;
    cudaEventRecord(ev[n++], st);
  }
  ~Timer() {
    if (!ctx->timing) return;
    if (n > 0) cudaEventSynchronize(ev[n - 1]);
    for (int i = 1; i < n; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      if (stage_of[i] >= 0 && stage_of[i] < 8) ctx->stage_ms[stage_of[i]] += ms;
    }
    for (int i = 0; i < 64; ++i) cudaEventDestroy(ev[i]);
  }
};

constexpr uint64_t kSpinLimit = 1ull << 24;

// Rounds of three-way splits before the merge sort takes every item left.
constexpr uint32_t kSplitRounds = 8;

uint32_t tiles_of(uint64_t n, uint32_t tile) { return (uint32_t)((n + tile - 1) / tile); }

// A sort's host decisions, for a CUDA graph of the same sort.  Everything
// the host launches follows from the segment sizes and from what it reads
// back: at each global level's end the next level's plan (device built) and
// the buckets sent to the standard sort; in each round of that sort the
// items' ranges, pivots and split decisions and the sizes of the split
// parts.  RUN_RECORD keeps those read-backs; RUN_CAPTURE launches the same
// work from them without reading back (for stream capture), with a guard
// kernel in place of each read-back that compares the device's value with
// the kept one and sets STATUS_REPLAN on a difference.
enum RunMode { RUN_EAGER = 0, RUN_RECORD = 1, RUN_CAPTURE = 2 };
enum { FB_LOHI = 0, FB_PIVOT = 1, FB_DOM = 2, FB_PART = 3 };
struct FbRound {
  std::vector<uint8_t> got[4];  // the round's read-backs (FB_*), as read
};
struct SortRecord {
  std::vector<LevelOut> levels;
  std::vector<std::vector<FbItem>> fb_lists;  // each standard-sort list, by offset
  std::vector<FbRound> rounds;                // every round of those sorts, in order
  size_t arena_bytes = 0;                     // the rounds' host-to-device staging
};
// A capture's view of a recording: the read-backs, their device copy (one
// blob: the level records, the lists, the rounds' buffers) and a pinned
// arena for the rounds' uploads, never reused within the capture (the
// graph's copies read it at every replay).
struct Replay {
  const SortRecord* rec = nullptr;
  const uint8_t* d_blob = nullptr;
  size_t levels_at = 0;
  std::vector<size_t> list_at;
  std::vector<std::vector<size_t>> round_at;  // [round][FB_*]
  HostBuf* arena = nullptr;
  size_t arena_off = 0, next_list = 0, next_round = 0;
};

// The standard sort of one level's fallback items (failure-guard buckets,
// |c| >= delta, and degenerate ones), keys in C, scratch D (both free at
// the items' offsets), result in out.  Per round: the range of every item
// and the most frequent value of a sample of it; an item that one value
// dominates is split stably into below / equal / above (the equal part is
// final, the others go to the next round, their keys now in D, so C and D
// swap), every other item is merge-sorted.  Equal keys keep their order
// throughout, so the pair sorts stay stable.
pcf_status run_fallback(pcf_ctx* ctx, const LaunchCfg& lc, std::vector<FbItem> work, uint64_t* C,
                        uint32_t* Cv, uint64_t* D, uint32_t* Dv, uint64_t* out_k, uint32_t* out_v,
                        uint32_t* tile_counter, uint64_t spin_limit, RunMode mode = RUN_EAGER,
                        SortRecord* rec = nullptr, Replay* rp = nullptr) {
  NvtxRange nvtx_fb("pcf fallback");
  const cudaStream_t st = lc.stream;
  const bool capture = mode == RUN_CAPTURE;
  const uint64_t kv = lc.pairs ? 12 : 8;  // bytes per key (+ value)
  for (uint32_t round = 0; !work.empty(); ++round) {
    const uint32_t nf = (uint32_t)work.size();
    const bool try_split = round < kSplitRounds;
    FbRound* rr = nullptr;  // this round's record (RUN_RECORD)
    size_t rno = 0;         // ... or its recording (RUN_CAPTURE)
    if (mode == RUN_RECORD) {
      rec->rounds.emplace_back();
      rr = &rec->rounds.back();
    } else if (capture) {
      rno = rp->next_round++;
      if (rno >= rp->rec->rounds.size()) return PCF_ERR_INTERNAL;
    }
    // device layout of the round: items | sort items | split items | done
    // items (at most three parts per split item)
    CK(ensure(ctx->fb_items, (size_t)6 * nf * sizeof(FbItem)));
    CK(ensure(ctx->fb_bases, ((size_t)6 * nf + 4) * 4));
    CK(ensure(ctx->fb_lohi, (size_t)9 * nf * 8 + (size_t)nf * 4 + 64));
    FbItem* d_items = as<FbItem>(ctx->fb_items);
    FbItem* d_items_s = d_items + nf;
    FbItem* d_items_p = d_items + 2 * nf;
    FbItem* d_items_d = d_items + 3 * nf;
    uint32_t* d_rb = as<uint32_t>(ctx->fb_bases);
    uint32_t* d_mb_s = d_rb + (nf + 1);
    uint32_t* d_mb_p = d_mb_s + (nf + 1);
    uint32_t* d_mb_d = d_mb_p + (nf + 1);
    uint64_t* d_lohi = as<uint64_t>(ctx->fb_lohi);
    uint64_t* d_pivot = d_lohi + 2 * nf;
    uint64_t* d_lohi_s = d_pivot + nf;
    uint64_t* d_piv_p = d_lohi_s + 2 * nf;
    uint64_t* d_item_cnt = d_piv_p + nf;
    uint32_t* d_dom = (uint32_t*)(d_item_cnt + 3 * nf);
    // host side of the round's transfers: one pinned arena, filled in order
    // (every use of the previous round's ended at its last synchronisation)
    CK(ensure_host(ctx->h_fb, (size_t)256 * nf + 1024));
    size_t aoff = 0;
    auto put = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
      const size_t step = (bytes + 15) & ~(size_t)15;
      if (mode == RUN_RECORD) rec->arena_bytes += step;
      if (capture) {  // the capture's own arena, one slice per upload
        if (rp->arena_off + step > rp->arena->cap) return cudaErrorInvalidValue;
        char* h = (char*)rp->arena->p + rp->arena_off;
        rp->arena_off += step;
        memcpy(h, src, bytes);
        return launch_xfer(st, dst, dview(*rp->arena, h), bytes);
      }
      char* h = (char*)ctx->h_fb.p + aoff;
      memcpy(h, src, bytes);
      aoff += step;
      return launch_xfer(st, dst, dview(ctx->h_fb, h), bytes);
    };
    std::vector<std::pair<void*, std::pair<const char*, size_t>>> gets;
    std::vector<std::pair<int, std::pair<const void*, size_t>>> kept;  // (FB_*, host copy)
    // a read-back: copied to the host (kind >= 0: kept when recording), or,
    // in a capture, the recorded value with a guard against the device's
    auto get = [&](void* dst, const void* src, size_t bytes, int kind) -> cudaError_t {
      if (capture) {
        const std::vector<uint8_t>& v = rp->rec->rounds[rno].got[kind];
        if (v.size() != bytes) return cudaErrorInvalidValue;
        memcpy(dst, v.data(), bytes);
        return launch_guard_words(lc, src, rp->d_blob + rp->round_at[rno][kind], bytes / 4);
      }
      char* h = (char*)ctx->h_fb.p + aoff;
      aoff += (bytes + 15) & ~(size_t)15;
      gets.push_back({dst, {h, bytes}});
      if (mode == RUN_RECORD && kind >= 0) kept.push_back({kind, {dst, bytes}});
      return launch_xfer(st, dview(ctx->h_fb, h), src, bytes);
    };
    auto sync = [&]() -> cudaError_t { return capture ? cudaSuccess : cudaStreamSynchronize(st); };
    // after a synchronisation: the gets land in their host vectors
    auto land = [&]() {
      for (auto& g : gets) memcpy(g.first, g.second.first, g.second.second);
      gets.clear();
      for (auto& k : kept) {
        const uint8_t* b = (const uint8_t*)k.second.first;
        rr->got[k.first].assign(b, b + k.second.second);
      }
      kept.clear();
    };

    std::vector<uint32_t> rb(nf + 1, 0);
    for (uint32_t i = 0; i < nf; ++i) rb[i + 1] = rb[i] + tiles_of(work[i].n, kRangeTile);
    std::vector<uint64_t> lohi(2 * nf);
    for (uint32_t i = 0; i < nf; ++i) {
      lohi[2 * i] = ~0ull;
      lohi[2 * i + 1] = 0;
    }
    CK(put(d_items, work.data(), nf * sizeof(FbItem)));
    CK(put(d_rb, rb.data(), (nf + 1) * 4));
    CK(put(d_lohi, lohi.data(), nf * 16));
    CK(launch_fb_range(lc, d_items, nf, d_rb, rb[nf], C, d_lohi));
    std::vector<uint64_t> pivot(nf, 0);
    std::vector<uint32_t> dom(nf, 0);
    if (try_split) CK(launch_fb_mode(lc, d_items, nf, C, d_lohi, d_pivot, d_dom));
    CK(get(lohi.data(), d_lohi, nf * 16, FB_LOHI));
    if (try_split) {
      CK(get(pivot.data(), d_pivot, nf * 8, FB_PIVOT));
      CK(get(dom.data(), d_dom, nf * 4, FB_DOM));
    }
    CK(sync());
    land();

    std::vector<FbItem> sw_items, sp_items;
    std::vector<uint64_t> lohi_s, piv_p;
    std::vector<uint32_t> mb_s(1, 0), mb_p(1, 0);
    uint64_t max_n_s = 0, keys_s = 0, keys_p = 0;
    for (uint32_t i = 0; i < nf; ++i) {
      const FbItem& it = work[i];
      if (dom[i]) {
        sp_items.push_back(it);
        piv_p.push_back(pivot[i]);
        mb_p.push_back(mb_p.back() + tiles_of(it.n, kMergeTile));
        keys_p += it.n;
      } else {
        sw_items.push_back(it);
        lohi_s.push_back(lohi[2 * i]);
        lohi_s.push_back(lohi[2 * i + 1]);
        mb_s.push_back(mb_s.back() + tiles_of(it.n, kMergeTile));
        max_n_s = std::max<uint64_t>(max_n_s, it.n);
        keys_s += it.n;
      }
    }
    ctx->stats.bytes_moved += (keys_s + keys_p) * 8;  // the range pass
    // merge sort: block sort, the merge passes up to the largest item, the copy
    if (const uint32_t ns = (uint32_t)sw_items.size()) {
      uint32_t passes = 2;
      for (uint64_t run = kMergeTile; run < max_n_s; run *= 2) ++passes;
      ctx->stats.bytes_moved += keys_s * 2 * kv * passes;
      CK(put(d_items_s, sw_items.data(), ns * sizeof(FbItem)));
      CK(put(d_mb_s, mb_s.data(), (ns + 1) * 4));
      CK(put(d_lohi_s, lohi_s.data(), ns * 16));
      CK(launch_fb_sort(lc, d_items_s, ns, d_mb_s, mb_s[ns], max_n_s, d_lohi_s, C, D, Cv, Dv,
                        out_k, out_v));
    }
    std::vector<FbItem> next;
    if (const uint32_t np = (uint32_t)sp_items.size()) {
      const uint32_t mp = mb_p[np];
      ctx->stats.bytes_moved += keys_p * (8 + 2 * kv);  // count, then move
      ctx->stats.fallback_splits += np;
      CK(ensure(ctx->fb_cnt, (size_t)3 * (mp + 1) * 4));
      CK(ensure(ctx->sw, ((size_t)tiles_of(3 * (uint64_t)(mp + 1), kScanTile) + 8) * 8));
      CK(put(d_items_p, sp_items.data(), np * sizeof(FbItem)));
      CK(put(d_mb_p, mb_p.data(), (np + 1) * 4));
      CK(put(d_piv_p, piv_p.data(), np * 8));
      CK(cudaMemsetAsync(d_item_cnt, 0, (size_t)np * 24, st));
      uint32_t* cnt = as<uint32_t>(ctx->fb_cnt);
      CK(launch_fb_part_count(lc, d_items_p, np, d_mb_p, mp, C, d_piv_p, cnt, d_item_cnt));
      CK(launch_scan(lc, cnt, 3 * (uint64_t)(mp + 1), nullptr, as<uint64_t>(ctx->sw),
                     tile_counter, 0xFFFFFFFFu, spin_limit, nullptr));
      CK(launch_fb_part_scatter(lc, d_items_p, np, d_mb_p, mp, C, Cv, d_piv_p, cnt, D, Dv));
      std::vector<uint64_t> part(3 * (size_t)np);
      uint32_t stw = 0;
      CK(get(part.data(), d_item_cnt, (size_t)np * 24, FB_PART));
      if (!capture) CK(get(&stw, lc.status, 4, -1));
      CK(sync());
      land();
      if (stw & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
      // the parts: below and above go round again (unless they are too short
      // to need sorting), the equal part is final; every final part is in D
      std::vector<FbItem> done;
      std::vector<uint32_t> mb_d(1, 0);
      for (uint32_t i = 0; i < np; ++i) {
        const uint64_t nl = part[3 * i], ne = part[3 * i + 1], ng = part[3 * i + 2];
        if (nl + ne + ng != sp_items[i].n || ne == 0) return PCF_ERR_INTERNAL;
        const FbItem parts[3] = {{sp_items[i].off, nl},
                                 {sp_items[i].off + nl, ne},
                                 {sp_items[i].off + nl + ne, ng}};
        for (int q = 0; q < 3; ++q) {
          if (!parts[q].n) continue;
          if (q != 1 && parts[q].n > 1) {
            next.push_back(parts[q]);
          } else {
            done.push_back(parts[q]);
            mb_d.push_back(mb_d.back() + tiles_of(parts[q].n, kMergeTile));
          }
        }
      }
      if (D != out_k && !done.empty()) {
        const uint32_t nd = (uint32_t)done.size();
        uint64_t done_keys = 0;
        for (const FbItem& it : done) done_keys += it.n;
        ctx->stats.bytes_moved += done_keys * 2 * kv;
        CK(put(d_items_d, done.data(), nd * sizeof(FbItem)));
        CK(put(d_mb_d, mb_d.data(), (nd + 1) * 4));
        CK(launch_fb_move(lc, d_items_d, nd, d_mb_d, mb_d[nd], D, out_k, Dv, out_v));
      }
    }
    CK(sync());
    work.swap(next);
    std::swap(C, D);
    std::swap(Cv, Dv);
  }
  return PCF_OK;
}


// The addresses of every buffer a context holds, hashed: a captured graph's
// nodes point into them, so a graph captured under another signature may
// point at freed memory and must not be replayed.
uint64_t buffers_signature(const pcf_ctx* c) {
  const void* ptrs[] = {c->tmp_k.p, c->tmp_v.p, c->tmp_aux.p, c->host_keys.p, c->segs.p,
                        c->bases.p, c->tpool.p, c->done.p, c->cmat1.p, c->cmat2.p, c->sw.p,
                        c->groups.p, c->gtiles.p, c->gcent.p, c->gtot.p, c->leaf.p, c->next.p,
                        c->fb.p, c->lout.p, c->status.p, c->misc.p, c->fb_items.p,
                        c->fb_bases.p, c->fb_lohi.p, c->small_items.p, c->segs_b.p, c->pcols.p,
                        c->pbsums.p, c->olist.p, c->mid.p, c->jbuf.p, c->small_segs.p,
                        c->fb_cnt.p,
                        c->bcounts.p, c->bmax.p, c->ptab.p, c->pipe_keys.p, c->h_stage.p,
                        c->h_lout.p, c->h_status.p, c->h_items.p, c->h_stage_small.p, c->h_fb.p,
                        c->h_offs.p};
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the addresses
  for (const void* q : ptrs) {
    uint64_t v = (uint64_t)(uintptr_t)q;
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xFFu;
      h *= 1099511628211ull;
    }
  }
  return h;
}

// Device bytes a context holds (every workspace buffer's capacity).
uint64_t workspace_held(const pcf_ctx* c) {
  const DevBuf* bufs[] = {&c->tmp_k, &c->tmp_v, &c->tmp_aux, &c->host_keys, &c->segs, &c->bases,
                          &c->tpool, &c->done, &c->cmat1, &c->cmat2, &c->sw, &c->groups,
                          &c->gtiles, &c->gcent, &c->gtot, &c->leaf, &c->next, &c->fb, &c->lout,
                          &c->status, &c->misc, &c->fb_items, &c->fb_bases, &c->fb_lohi,
                          &c->small_items, &c->segs_b, &c->pcols, &c->pbsums, &c->olist, &c->mid,
                          &c->jbuf, &c->small_segs, &c->fb_cnt, &c->bcounts, &c->bmax, &c->ptab,
                          &c->pipe_keys};
  uint64_t b = 0;
  for (const DevBuf* d : bufs) b += d->cap;
  return b;
}

// An upper bound on the workspace a sort of n keys in S arrays grows a
// context to, following the sizes run_sort asks for.  Level buffers are
// reused from level to level, so each takes the larger of two cases: level
// 0 with S arrays of equal size (floor(n_s^(c)) summed over the arrays is
// largest when they are equal), and a later level of n / (cap + 1)
// (sub)arrays of cap + 1 keys (every key one level further down, in the
// smallest (sub)arrays a level takes).  Standard-sort rounds are bounded by
// items of more than 1024 keys, each split in at most three parts.  Every
// buffer is allocated a quarter larger than asked (ensure()).
uint64_t workspace_bound(const Policy& P, const pcf_tuning& tu, uint64_t n, uint32_t S,
                         bool pairs) {
  if (n == 0) return 0;
  const uint32_t cap = onchip_cap(tu.leaf_cap, P, pairs);
  const bool leaf_sort = !pairs && tu.leaf_mode == 1;
  const uint64_t olist_per = 8ull * (leaf_sort ? leaf_sort_classes(cap) : onchip_classes(cap));
  auto grow = [](uint64_t b) { return b + b / 4; };
  // k_mid's work list and leaf records (counted with the class lists)
  const bool mid = leaf_sort && P.model == MODEL_PCF && P.range_mode == RANGE_ARRAY;
  auto mid_bytes = [&](uint64_t n_level) -> uint64_t {
    if (!mid) return 0;
    uint64_t at = ((n_level / ((uint64_t)cap + 1) + 1) * 4 + 15) / 16 * 2;
    for (uint32_t q = 0; q < kMaxLeafClasses; ++q) at += mid_class_cap(q, n_level, cap);
    return at * 8;
  };
  enum { LEAF, NEXT, FB, TPOOL, SW, CMAT1, GROUPS, GTILES, GCENT, CMAT2, OLIST, PLAN, PLAN2,
         PCOLS, PBSUMS, NNEED };
  uint64_t need[NNEED] = {0};
  ParamCache pc;
  auto level = [&](uint64_t rows, uint64_t size, uint64_t n_level) {
    if (!rows) return;
    std::vector<InSeg> in(rows);
    uint64_t off = 0;
    for (uint64_t r = 0; r < rows; ++r) {
      in[r] = InSeg{off, size, 0, 0, 0};
      off += size;
    }
    Plan pl;
    plan_level(P, tu, pc, in, pl);
    const uint64_t max_items = std::max<uint64_t>(pl.n_buckets, rows) + 16;
    const uint64_t scan_max =
        std::max(std::max(pl.cmat1, pl.cmat2_bound), std::max(pl.tpool, pl.n_buckets));
    const uint64_t s_max = std::min<uint64_t>(pl.n_buckets, n_level / (cap + 1)) + 1;
    const uint64_t v[NNEED] = {
        max_items * sizeof(BRec), max_items * 4, max_items * sizeof(FbItem), pl.tpool * 4,
        ((scan_max + kScanTile - 1) / kScanTile + (pl.n_groups + kScanTile - 1) / kScanTile + 8) * 8,
        pl.cmat1 * 4, pl.n_groups * sizeof(Group), pl.n_groups * 4, pl.n_groups * 4,
        pl.cmat2_bound * 4, pl.n_buckets * olist_per + mid_bytes(n_level), plan_layout(rows).bytes,
        plan_layout(s_max).bytes, (uint64_t)PC_NCOL * s_max * 4,
        (uint64_t)PC_NCOL * ((s_max + 2047) / 2048) * 4};
    for (int i = 0; i < NNEED; ++i) need[i] = std::max(need[i], v[i]);
  };
  const uint64_t per = (n + S - 1) / S;
  if (per > cap) level(S, per, n);
  level(n / (cap + 1), cap + 1, n);
  // the arrays of at most cap keys, straight to the on-chip kernels
  const uint64_t small = per <= cap ? S : 0;
  uint64_t b = 0;
  for (int i = 0; i < NNEED; ++i) b += grow(need[i]);
  // the plan buffers are two (this level's and the next's)
  b += grow(std::max(need[PLAN], need[PLAN2])) - grow(need[PLAN]);
  b += grow(small * sizeof(Seg) + (small + 1) * 4) + grow(small * sizeof(BRec) + 64);
  b += grow(std::max<uint64_t>(small * olist_per, need[OLIST])) - grow(need[OLIST]);
  b += grow(n * 8) + grow(n * 2) + grow(n * 4) + (pairs ? grow(n * 4) : 0);
  // standard-sort rounds
  const uint64_t nf = 3 * (n / 1025 + S) + 1;
  const uint64_t mp = n / kMergeTile + nf;
  b += grow(6 * nf * sizeof(FbItem)) + grow((6 * nf + 4) * 4) + grow(9 * nf * 8 + nf * 4 + 64);
  b += grow(3 * (mp + 1) * 4);
  b += grow(((3 * (mp + 1) + kScanTile - 1) / kScanTile + 8) * 8);
  // status, level record, misc, the on-chip parameter table
  b += grow(64) + grow(sizeof(LevelOut) + 64) + grow(256) + grow((uint64_t)(tu.leaf_cap + 1) * 8);
  return b;
}

// The status word and the decision counters after it (DecisionCounters at
// byte 16 of the status buffer), read back together.
constexpr size_t kStatusReadBytes = 16 + sizeof(DecisionCounters);

void take_counters(pcf_ctx* ctx) {
  DecisionCounters d;
  memcpy(&d, (const char*)ctx->h_status.p + 16, sizeof d);
  ctx->stats.guard_buckets = d.guard_buckets;
  ctx->stats.guard_keys = d.guard_keys;
  ctx->stats.bucketings = d.bucketings;
}

// The whole sort of a batch of arrays.  Level-0 segments are the caller's
// arrays; keys flow src -> tmp (pass 1) -> out (pass 2); leaf buckets are
// finished in place in out; fallback buckets are merge-sorted in out.
// mode / rec / rp: see SortRecord and Replay.
// Waits for every piece of a sort still in flight: the caller's stream and
// the side stream (a call that failed between the fork and the join leaves
// work on both).
void drain(pcf_ctx* ctx, cudaStream_t st) {
  cudaStreamSynchronize(st);
  if (ctx->side.ready) {
    cudaStreamSynchronize(ctx->side.st);
    cudaStreamSynchronize(ctx->side.st2);
  }
}

pcf_status run_sort(pcf_ctx* ctx, const uint64_t* in_k, const uint32_t* in_v, uint64_t* out_k,
                    uint32_t* out_v, const std::vector<InSeg>& user, uint32_t kt, bool pairs,
                    cudaStream_t st, uint32_t scan_withhold = 0xFFFFFFFFu,
                    uint64_t spin_limit = kSpinLimit, RunMode mode = RUN_EAGER,
                    SortRecord* rec = nullptr, Replay* rp = nullptr) {
  NvtxRange nvtx_sort("pcf sort");
  ctx->stats = pcf_call_stats{};
  for (int i = 0; i < 8; ++i) ctx->stage_ms[i] = 0;
  uint64_t n_total = 0;
  for (auto& s : user) n_total = std::max(n_total, s.off + s.n);
  if (n_total == 0) return PCF_OK;
  CK(cudaSetDevice(ctx->device));
  LaunchCfg lc;
  lc.stream = st;
  lc.kt = kt;
  lc.pairs = pairs;
  lc.launches = &ctx->stats.kernel_launches;
  lc.model = ctx->policy.model;
  lc.range_mode = ctx->policy.range_mode;
  lc.leaf_sort = !pairs && ctx->tuning.leaf_mode == 1;
  const bool use_mid = lc.leaf_sort && ctx->policy.model == MODEL_PCF &&
                       ctx->policy.range_mode == RANGE_ARRAY;
  CK(ensure(ctx->status, 64));
  lc.status = as<uint32_t>(ctx->status);
  CK(cudaMemsetAsync(lc.status, 0, 64, st));
  CK(ensure_host(ctx->h_status, 64));
#ifdef PCF_CHECKED
  // the key buffers' length, for the checked build's index checks
  *(uint64_t*)((char*)ctx->h_status.p + 8) = n_total;
  CK(launch_xfer(st, (char*)lc.status + 8, (char*)ctx->h_status.dp + 8, 8));
#endif
  CK(ensure_host(ctx->h_lout, sizeof(LevelOut)));
  CK(ensure(ctx->lout, sizeof(LevelOut) + 64));
  CK(ensure(ctx->misc, 256));
  const uint32_t tile_keys = 1u << ctx->tuning.tile_log2;
  // the largest bucket finished on chip (the alpha..delta table covers the
  // tuning's leaf_cap, at least this)
  const uint32_t cap = onchip_cap(ctx->tuning.leaf_cap, ctx->policy, pairs);
  const size_t olist_per_bucket =
      (size_t)8 * (lc.leaf_sort ? leaf_sort_classes(cap) : onchip_classes(cap));
  CK(ensure_ptab(ctx, st));
  const uint16_t* ptab = as<uint16_t>(ctx->ptab);
  Timer tm(ctx, st);
  tm.mark(-1);

  // NaN check of every key by the range passes (the small arrays' here,
  // the others' at level 0); every later kernel is gated on the status word
  // (pcf_aborted), so none writes once a NaN is seen.
  std::vector<InSeg> small, big;
  for (auto& s : user) {
    if (s.n == 0) continue;
    if (s.n <= cap) small.push_back(s);
    else big.push_back(s);
  }
  if (kt == KEY_F64) {
    // range + NaN of the small segments in one launch (big ones: level 0)
    std::vector<InSeg> all = small;
    if (!all.empty()) {
      Plan pl;
      plan_level(ctx->policy, ctx->tuning, ctx->pcache, all, pl);
      const uint32_t S = (uint32_t)all.size();
      size_t need = S * sizeof(Seg) + (S + 1) * 4;
      // its own staging buffer: the level-0 plan below is staged while this
      // copy may still be queued
      CK(ensure_host(ctx->h_stage_small, need));
      CK(ensure(ctx->small_segs, need));
      memcpy(ctx->h_stage_small.p, pl.segs.data(), S * sizeof(Seg));
      memcpy((char*)ctx->h_stage_small.p + S * sizeof(Seg), pl.range_base.data(), (S + 1) * 4);
      CK(launch_xfer(st, ctx->small_segs.p, ctx->h_stage_small.dp, need));
      CK(launch_range(lc, as<Seg>(ctx->small_segs), S,
                      (const uint32_t*)((char*)ctx->small_segs.p + S * sizeof(Seg)),
                      pl.range_base[S], in_k, true));
    }
  }

  // ---- level 0 of the small arrays: straight to the shared-memory kernel,
  // launched after the range passes that check every key for NaN (and gated
  // on their flag)
  auto launch_small = [&]() -> pcf_status {
    if (small.empty()) return PCF_OK;
    const uint32_t S = (uint32_t)small.size();
    std::vector<BRec> recs(S);
    for (uint32_t i = 0; i < S; ++i) {
      recs[i].off = (uint32_t)small[i].off;
      recs[i].n = (uint32_t)small[i].n;
      recs[i].kind = BK_LEAF | (small[i].n < ctx->policy.tau ? BK_STD : 0u);
      recs[i].depth = small[i].depth;
      recs[i].start = small[i].start;
      recs[i].seed = small[i].seed;
    }
    const size_t need = S * sizeof(BRec) + 64;
    CK(ensure(ctx->small_items, need));
    CK(ensure_host(ctx->h_items, need));
    memcpy(ctx->h_items.p, recs.data(), S * sizeof(BRec));
    CK(launch_xfer(st, ctx->small_items.p, ctx->h_items.dp, S * sizeof(BRec)));
    CK(ensure(ctx->olist, (size_t)S * olist_per_bucket));
    CK(launch_onchip(lc, as<BRec>(ctx->small_items), S, cap, in_k, in_v, out_k, out_v,
                     ctx->policy, ptab, as<uint32_t>(ctx->olist),
                     (uint32_t*)((char*)ctx->misc.p + 128)));
    ctx->stats.leaf_buckets += S;
    return PCF_OK;
  };
  if (big.empty()) {
    pcf_status r = launch_small();
    if (r != PCF_OK) return r;
    tm.mark(6);
  }

  // ---- global levels
  // Each level reads `src`; pass 1 writes P1 (the other buffer), pass 2 (if
  // any) writes P2; X is where the level's buckets end.  On-chip buckets go
  // X -> out, next-level (sub)arrays stay in X, fallback buckets are sorted
  // from X into out.
  CK(ensure(ctx->tmp_k, n_total * 8));
  CK(ensure(ctx->tmp_aux, n_total * 2));
  CK(ensure(ctx->jbuf, n_total * 4));
  if (pairs) CK(ensure(ctx->tmp_v, n_total * 4));
  uint64_t* const tmp_k = as<uint64_t>(ctx->tmp_k);
  uint32_t* const tmp_v = pairs ? as<uint32_t>(ctx->tmp_v) : nullptr;
  const uint64_t* src = in_k;
  const uint32_t* src_v = in_v;
  const uint32_t dbits = std::min(ctx->tuning.max_digit_bits, kMaxDigitBits);
  // Level 0 is planned on the host (the caller's arrays); every later level
  // is planned on the device by the level before it, in the other buffer.
  DevBuf* pbuf[2] = {&ctx->segs, &ctx->segs_b};
  int cur = 0;
  LevelPlan L;
  if (!big.empty()) {
    Plan pl;
    uint64_t n_big = 0;
    for (auto& sg : big) n_big += sg.n;
    pcf_tuning tu0 = ctx->tuning;
    tu0.tile_log2 = level0_tile_log2(ctx->tuning, n_big, ctx->num_sms);
    L.tile_log2 = tu0.tile_log2;
    plan_level(ctx->policy, tu0, ctx->pcache, big, pl);
    const uint32_t S = (uint32_t)big.size();
    const PlanLayout PL = plan_layout(S);
    CK(ensure_host(ctx->h_stage, PL.bytes));
    CK(ensure(*pbuf[cur], PL.bytes));
    char* hs = (char*)ctx->h_stage.p;
    memcpy(hs, pl.segs.data(), S * sizeof(Seg));
    memcpy(hs + PL.o_rb, pl.range_base.data(), (S + 1) * 4);
    memcpy(hs + PL.o_k1, pl.k1_base.data(), (S + 1) * 4);
    memcpy(hs + PL.o_t1, pl.tile1_base.data(), (S + 1) * 4);
    memcpy(hs + PL.o_gb, pl.group_base.data(), (S + 1) * 8);
    memcpy(hs + PL.o_bb, pl.bucket_base.data(), (S + 1) * 8);
    CK(launch_xfer(st, pbuf[cur]->p, ctx->h_stage.dp, PL.bytes));
    L.S = S;
    for (auto& sg : big) L.n_level += sg.n;
    L.wb = big.front().off;
    L.we = big.back().off + big.back().n;
    L.n_range = pl.range_base[S];
    L.n_k1 = pl.k1_base[S];
    L.n_t1 = pl.tile1_base[S];
    L.n_groups = pl.n_groups;
    L.n_buckets = pl.n_buckets;
    L.tpool = pl.tpool;
    L.cmat1 = pl.cmat1;
    L.cmat2_bound = pl.cmat2_bound;
    L.tiles2_bound = pl.tiles2_bound;
    L.dmax1 = pl.dmax1;
    L.dmax2 = pl.dmax2;
    L.two_pass = pl.two_pass;
    L.dp = dev_plan(pbuf[cur]->p, PL);
  }
  bool first = true;
  size_t level_no = 0;
  // the status word was read after the last launch (the final read below
  // would repeat it)
  bool status_current = false;
  while (L.S) {
    NvtxRange nvtx_level(first ? "pcf level 0" : "pcf level");
    const uint32_t S = L.S;
    const uint64_t n_level = L.n_level;
    ctx->stats.levels += 1;
    uint64_t* P1 = (src == tmp_k) ? out_k : tmp_k;
    uint32_t* P1v = (src == tmp_k) ? out_v : tmp_v;
    uint64_t* P2 = (P1 == tmp_k) ? out_k : tmp_k;
    uint32_t* P2v = (P1 == tmp_k) ? out_v : tmp_v;
    uint64_t* X = L.two_pass ? P2 : P1;
    uint32_t* Xv = L.two_pass ? P2v : P1v;
    Seg* d_segs = L.dp.segs;

    // range, model.  NaN keys (level 0, binary64) are flagged by the full
    // range pass, or with a sample range by k_hist1 and the range pass of
    // the segments that need one; either way before any kernel that writes
    // the output runs (those are gated on the flag)
    const bool srange = lc.range_mode == RANGE_SAMPLE;
    const bool check_nan = first && kt == KEY_F64;
    if (srange) {
      // the samples' range; the array's where it is equal or degenerate (R14)
      CK(launch_sample_range(lc, d_segs, S, L.dp.k1, L.n_k1, src));
      CK(launch_model(lc, d_segs, S, 1));
      CK(launch_range(lc, d_segs, S, L.dp.rb, L.n_range, src, check_nan, SEG_NEEDRANGE));
      CK(launch_model(lc, d_segs, S, 2));
    } else {
      CK(launch_range(lc, d_segs, S, L.dp.rb, L.n_range, src, check_nan));
      if (first) {
        const pcf_status r = launch_small();
        if (r != PCF_OK) return r;
      }
      CK(launch_model(lc, d_segs, S));
    }
    tm.mark(0);
    // (sub)arrays with one value are final; degenerate ones join the
    // fallback list, whose keys are taken from X (with a sample range on
    // binary64 keys at level 0: after the NaN gate below, as they write
    // the output)
    auto copy_special = [&]() -> cudaError_t {
      cudaError_t e = cudaSuccess;
      if (src != out_k)
        e = launch_copy_segs(lc, d_segs, S, L.dp.rb, L.n_range, src, out_k, src_v, out_v,
                             1u << SEG_SINGLE);
      if (!e && src != X)
        e = launch_copy_segs(lc, d_segs, S, L.dp.rb, L.n_range, src, X, src_v, Xv,
                             1u << SEG_DEGEN);
      return e;
    };
    const bool late_gate = srange && first;
    if (!late_gate) CK(copy_special());
    // lists
    const uint64_t max_items = std::max<uint64_t>(L.n_buckets, S) + 16;
    CK(ensure(ctx->leaf, max_items * sizeof(BRec)));
    CK(ensure(ctx->next, max_items * 4));
    CK(ensure(ctx->fb, max_items * sizeof(FbItem)));
    LevelOut* d_lo = as<LevelOut>(ctx->lout);
    CK(cudaMemsetAsync(d_lo, 0, sizeof(LevelOut), st));
    CK(launch_seg_status_lists(lc, d_segs, S, as<FbItem>(ctx->fb), d_lo, (uint32_t)max_items));
    // sample + PCF: counts per bin, then b by one inclusive scan of the pool
    CK(ensure(ctx->tpool, L.tpool * 4));
    CK(cudaMemsetAsync(ctx->tpool.p, 0, L.tpool * 4, st));
    const uint64_t scan_max =
        std::max(std::max(L.cmat1, L.cmat2_bound), std::max(L.tpool, L.n_buckets));
    const uint64_t sw_need = ((scan_max + kScanTile - 1) / kScanTile +
                              (L.n_groups + kScanTile - 1) / kScanTile + 8) * 8;
    CK(ensure(ctx->sw, sw_need));
    uint32_t* tile_counter = as<uint32_t>(ctx->misc);
    uint64_t* totals = (uint64_t*)((char*)ctx->misc.p + 64);
    CK(launch_sample(lc, d_segs, S, L.dp.k1, L.n_k1, src, as<uint32_t>(ctx->tpool)));
    CK(launch_table(lc, d_segs, S, as<uint32_t>(ctx->tpool), L.tpool, as<uint64_t>(ctx->sw),
                    tile_counter, spin_limit));
    tm.mark(1);
    // pass 1
    KeyBufs kb;
    kb.src = src;
    kb.src_v = src_v;
    kb.tmp = P1;
    kb.tmp_v = P1v;
    kb.tmp_aux = as<uint16_t>(ctx->tmp_aux);
    kb.jbuf = as<uint32_t>(ctx->jbuf);
    kb.out = P2;
    kb.out_v = P2v;
    CK(ensure(ctx->cmat1, L.cmat1 * 4));
    CK(cudaMemsetAsync(ctx->cmat1.p, 0, L.cmat1 * 4, st));
    const uint32_t tk = 1u << L.tile_log2;
    CK(launch_hist1(lc, d_segs, S, L.dp.t1, L.n_t1, tk, src, as<uint32_t>(ctx->tpool),
                    as<uint32_t>(ctx->cmat1), L.dmax1, as<uint32_t>(ctx->jbuf),
                    srange && check_nan));
    if (late_gate) {
      const pcf_status r = launch_small();
      if (r != PCF_OK) return r;
      CK(copy_special());
    }
    CK(launch_scan(lc, as<uint32_t>(ctx->cmat1), L.cmat1, nullptr, as<uint64_t>(ctx->sw),
                   tile_counter, scan_withhold, spin_limit, nullptr));
    tm.mark(2);
    CK(launch_scatter1(lc, d_segs, S, L.dp.t1, L.n_t1, tk, kb, as<uint32_t>(ctx->tpool),
                       as<uint32_t>(ctx->cmat1), L.dmax1));
    tm.mark(3);
    ctx->stats.global_passes += 1;
    ctx->stats.bytes_moved += n_level * (8 /*range*/ + 8 + 4 /*hist1*/ + 12 + 10 /*scatter1*/) +
                              (pairs ? n_level * 8 : 0);
    // pass 2: count tiles up to 4x larger than pass 1's.  Its digit is the
    // wider one, and larger tiles keep its count matrix (written and read
    // with a stride of one row per digit) small; the plan's bounds, taken
    // with pass 1's tile size, still hold (there are fewer tiles)
    if (L.two_pass) {
      const uint32_t tile_keys2 = tk << pass2_shift(L.tile_log2, n_level, ctx->num_sms);
      CK(ensure(ctx->groups, L.n_groups * sizeof(Group)));
      CK(ensure(ctx->gtiles, L.n_groups * 4));
      CK(ensure(ctx->gcent, L.n_groups * 4));
      CK(launch_groups(lc, d_segs, S, L.dp.gb, L.n_groups, as<uint32_t>(ctx->cmat1), tile_keys2,
                       as<Group>(ctx->groups), as<uint32_t>(ctx->gtiles),
                       as<uint32_t>(ctx->gcent)));
      CK(launch_scan(lc, as<uint32_t>(ctx->gtiles), L.n_groups, nullptr, as<uint64_t>(ctx->sw),
                     tile_counter, 0xFFFFFFFFu, spin_limit, &totals[0]));
      CK(launch_scan(lc, as<uint32_t>(ctx->gcent), L.n_groups, nullptr, as<uint64_t>(ctx->sw),
                     tile_counter, 0xFFFFFFFFu, spin_limit, &totals[1]));
      CK(launch_group_bases(lc, as<Group>(ctx->groups), L.n_groups, as<uint32_t>(ctx->gcent)));
      CK(ensure(ctx->cmat2, L.cmat2_bound * 4));
      CK(cudaMemsetAsync(ctx->cmat2.p, 0, L.cmat2_bound * 4, st));
      CK(launch_hist2(lc, as<Group>(ctx->groups), (uint32_t)L.n_groups, d_segs,
                      as<uint32_t>(ctx->gtiles), &totals[0], (uint32_t)L.tiles2_bound, tile_keys2,
                      kb.tmp_aux, as<uint32_t>(ctx->cmat2), L.dmax2));
      CK(launch_scan(lc, as<uint32_t>(ctx->cmat2), L.cmat2_bound, &totals[1],
                     as<uint64_t>(ctx->sw), tile_counter, 0xFFFFFFFFu, spin_limit, nullptr));
      tm.mark(4);
      CK(launch_scatter2(lc, as<Group>(ctx->groups), (uint32_t)L.n_groups, d_segs,
                         as<uint32_t>(ctx->gtiles), &totals[0], (uint32_t)L.tiles2_bound,
                         tile_keys2, kb, as<uint32_t>(ctx->cmat2), L.dmax2));
      // segments whose bucket id has one digit were already bucketed by pass 1
      CK(launch_copy_segs(lc, d_segs, S, L.dp.rb, L.n_range, P1, P2, P1v, P2v, kCopyOneDigit));
      tm.mark(5);
      ctx->stats.global_passes += 1;
      ctx->stats.bytes_moved += n_level * (2 /*hist2*/ + 10 + 8 /*scatter2*/) +
                                (pairs ? n_level * 8 : 0);
    }
    // buckets: Alg. 1's per-bucket decision (for the block-local leaf sort
    // it also lists the leaf buckets by size class), then the on-chip finish
    uint32_t* next_flag = as<uint32_t>(ctx->next);
    uint32_t* leaf_counts = (uint32_t*)((char*)ctx->misc.p + 128);
    CK(ensure(ctx->olist, (size_t)L.n_buckets * olist_per_bucket));
    // mid-size next-level buckets: one Learned-Sort call per CTA (k_mid),
    // keys-only block-local sorts under the default policy
    const bool mid = use_mid;
    uint32_t* mid_counts = (uint32_t*)((char*)ctx->misc.p + 160);  // per class
    uint32_t* mid_count = (uint32_t*)((char*)ctx->misc.p + 192);
    MidLists ml{};
    uint32_t* mid_list = nullptr;
    uint2* mid_lists = nullptr;
    if (mid) {
      const uint64_t n_mid_max = n_level / ((uint64_t)cap + 1) + 1;
      uint64_t at = (n_mid_max * 4 + 15) / 16 * 2;  // u64 units after the work list
      for (uint32_t q = 0; q < kMaxLeafClasses; ++q) {
        ml.cap[q] = mid_class_cap(q, n_level, cap);
        ml.base[q] = at;
        at += ml.cap[q];
      }
      CK(ensure(ctx->mid, at * 8));
      mid_list = as<uint32_t>(ctx->mid);
      mid_lists = (uint2*)ctx->mid.p;
    }
    if (lc.leaf_sort) CK(cudaMemsetAsync(leaf_counts, 0, mid ? 68 : 4 * kMaxLeafClasses, st));
    CK(launch_buckets(lc, d_segs, S, L.n_buckets, L.dp.bb, as<Group>(ctx->groups),
                      as<uint32_t>(ctx->cmat1), as<uint32_t>(ctx->cmat2), L.two_pass, cap,
                      (uint32_t)ctx->policy.tau, X, Xv, out_k, out_v, as<BRec>(ctx->leaf),
                      next_flag, as<FbItem>(ctx->fb), d_lo, (uint32_t)max_items,
                      lc.leaf_sort ? as<uint2>(ctx->olist) : nullptr,
                      lc.leaf_sort ? leaf_counts : nullptr, leaf_sort_classes(cap), mid_list,
                      mid_count));
    if (mid) {
      // the mid (sub)arrays' buckets land in Y (free at their offsets); the
      // mid calls and their leaf sort run on the side stream beside the
      // level's leaf sort (they touch other keys), joined before the
      // next level's planning reads their flags
      uint64_t* Y = (X == tmp_k) ? out_k : tmp_k;
      CK(ctx->side.init());
      LaunchCfg ls = lc;
      ls.stream = ctx->side.st;
      CK(cudaEventRecord(ctx->side.fork, st));
      CK(cudaStreamWaitEvent(ls.stream, ctx->side.fork, 0));
      CK(launch_mid(ls, mid_list, mid_count, as<BRec>(ctx->leaf), X, Y, out_k, next_flag,
                    mid_lists, ml, mid_counts, leaf_sort_classes(cap), cap, ctx->policy, d_lo));
      CK(launch_onchip(ls, nullptr, 1u, cap, Y, nullptr, out_k, nullptr, ctx->policy, ptab,
                       (uint32_t*)mid_lists, mid_counts, true, ml.base));
      // the level's classes above 512 keys on a second side stream, so that
      // the classes' launches overlap one another's tails
      CK(cudaStreamWaitEvent(ctx->side.st2, ctx->side.fork, 0));
      cudaStream_t cls_st[kMaxLeafClasses];
      for (uint32_t q = 0; q < kMaxLeafClasses; ++q) cls_st[q] = q < 4 ? st : ctx->side.st2;
      CK(launch_onchip(lc, as<BRec>(ctx->leaf), (uint32_t)L.n_buckets, cap, X, Xv, out_k,
                       out_v, ctx->policy, ptab, as<uint32_t>(ctx->olist), leaf_counts,
                       lc.leaf_sort, nullptr, cls_st));
      CK(cudaEventRecord(ctx->side.join, ls.stream));
      CK(cudaEventRecord(ctx->side.join2, ctx->side.st2));
      CK(cudaStreamWaitEvent(st, ctx->side.join, 0));
      CK(cudaStreamWaitEvent(st, ctx->side.join2, 0));
    } else {
      CK(launch_onchip(lc, as<BRec>(ctx->leaf), (uint32_t)L.n_buckets, cap, X, Xv, out_k,
                       out_v, ctx->policy, ptab, as<uint32_t>(ctx->olist), leaf_counts,
                       lc.leaf_sort));
    }
    tm.mark(6);
    // the next level's plan, built on the device into the other buffer; a
    // next-level (sub)array holds more than cap keys, which bounds its rows
    const uint64_t s_max = std::min<uint64_t>(L.n_buckets, n_level / (cap + 1)) + 1;
    const PlanLayout NL = plan_layout(s_max);
    CK(ensure(*pbuf[cur ^ 1], NL.bytes));
    const DevPlan ndp = dev_plan(pbuf[cur ^ 1]->p, NL);
    const uint32_t ncb = (uint32_t)((s_max + 2047) / 2048);
    CK(ensure(ctx->pcols, (size_t)PC_NCOL * s_max * 4));
    CK(ensure(ctx->pbsums, (size_t)PC_NCOL * ncb * 4));
    CK(launch_plan_next(lc, as<BRec>(ctx->leaf), next_flag, L.n_buckets, (uint32_t)s_max,
                        ctx->policy, dbits, tile_keys, ndp, as<uint32_t>(ctx->pcols),
                        as<uint32_t>(ctx->pbsums), d_lo, as<uint64_t>(ctx->sw), tile_counter,
                        spin_limit, &totals[2]));
    LevelOut lo;
    if (mode == RUN_CAPTURE) {
      if (level_no >= rp->rec->levels.size()) return PCF_ERR_INTERNAL;
      const LevelOut* d_levels = (const LevelOut*)(rp->d_blob + rp->levels_at);
      CK(launch_guard(lc, d_lo, d_levels + level_no));
      lo = rp->rec->levels[level_no];
    } else {
      CK(launch_xfer(st, ctx->h_lout.dp, d_lo, sizeof(LevelOut)));
      CK(launch_xfer(st, ctx->h_status.dp, lc.status, kStatusReadBytes));
      CK(cudaStreamSynchronize(st));
      lo = *(LevelOut*)ctx->h_lout.p;
      take_counters(ctx);
      const uint32_t stw = *(uint32_t*)ctx->h_status.p;
      if (stw & STATUS_NAN) return PCF_ERR_INVALID_KEY;
      if (stw & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
      if (stw & (STATUS_INTERNAL | STATUS_BOUNDS)) return PCF_ERR_INTERNAL;
      if (mode == RUN_RECORD) rec->levels.push_back(lo);
    }
    ++level_no;
    ctx->stats.leaf_buckets += lo.n_leaf;
    uint64_t level_fb_keys = 0;
    // standard sort of the large failure-guard / degenerate buckets, in
    // offset order (the device lists them in any order)
    if (lo.n_fb) {
      std::vector<FbItem> items;
      if (mode == RUN_CAPTURE) {
        const size_t li = rp->next_list++;
        if (li >= rp->rec->fb_lists.size() || rp->rec->fb_lists[li].size() != lo.n_fb)
          return PCF_ERR_INTERNAL;
        items = rp->rec->fb_lists[li];
        CK(launch_guard_list(lc, as<FbItem>(ctx->fb),
                             (const FbItem*)(rp->d_blob + rp->list_at[li]), lo.n_fb));
      } else {
        items.resize(lo.n_fb);
        CK(ensure_host(ctx->h_fb, (size_t)lo.n_fb * sizeof(FbItem)));
        CK(launch_xfer(st, ctx->h_fb.dp, ctx->fb.p, lo.n_fb * sizeof(FbItem)));
        CK(cudaStreamSynchronize(st));
        memcpy(items.data(), ctx->h_fb.p, lo.n_fb * sizeof(FbItem));
        std::sort(items.begin(), items.end(),
                  [](const FbItem& a, const FbItem& b) { return a.off < b.off; });
        if (mode == RUN_RECORD) rec->fb_lists.push_back(items);
      }
      for (const FbItem& it : items) level_fb_keys += it.n;
      ctx->stats.fallback_keys += level_fb_keys;
      ctx->stats.fallback_buckets += lo.n_fb;
      // scratch: the buffer that is not X (the items' ranges there are free)
      uint64_t* Y = (X == tmp_k) ? out_k : tmp_k;
      uint32_t* Yv = (X == tmp_k) ? out_v : tmp_v;
      const pcf_status fs = run_fallback(ctx, lc, std::move(items), X, Xv, Y, Yv, out_k, out_v,
                                         tile_counter, spin_limit, mode, rec, rp);
      if (fs != PCF_OK) return fs;
      tm.mark(7);
    }
    // keys finished on chip (or copied as one value) this level: read and
    // written once
    ctx->stats.bytes_moved += (n_level - lo.plan.n_keys - level_fb_keys) * (pairs ? 24 : 16);
    // keys bucketed by k_mid: read for the range, the bins and the append,
    // written once (their leaf sort is counted above)
    ctx->stats.bytes_moved += lo.mid_keys * 32;
    // the next level
    const PlanTotals& pt = lo.plan;
    LevelPlan N;
    N.S = pt.S;
    if (N.S) {
      N.n_level = pt.n_keys;
      N.wb = pt.lo;
      N.we = pt.hi;
      N.n_range = (uint32_t)pt.col[PC_RANGE];
      N.n_k1 = (uint32_t)pt.col[PC_K1];
      N.n_t1 = (uint32_t)pt.col[PC_TILES1];
      N.n_groups = pt.col[PC_GROUPS];
      N.n_buckets = pt.col[PC_BUCKETS];
      N.tpool = pt.col[PC_TPOOL];
      N.cmat1 = pt.col[PC_CMAT1];
      N.cmat2_bound = pt.col[PC_CMAT2];
      N.tiles2_bound = pt.col[PC_TILES2];
      N.dmax1 = std::max(1u, pt.dmax1);
      N.dmax2 = std::max(1u, pt.dmax2);
      N.two_pass = pt.two_pass != 0;
      N.tile_log2 = ctx->tuning.tile_log2;  // as the device planner used
      N.dp = ndp;
    }
    L = N;
    cur ^= 1;
    src = X;
    src_v = Xv;
    first = false;
    // read at this level's end, and nothing launched since unless the
    // standard sort ran
    status_current = mode != RUN_CAPTURE && lo.n_fb == 0;
  }
  if (mode == RUN_CAPTURE) return PCF_OK;  // the replay reads the status word
  if (status_current) return PCF_OK;
  CK(launch_xfer(st, ctx->h_status.dp, lc.status, kStatusReadBytes));
  CK(cudaStreamSynchronize(st));
  take_counters(ctx);
  const uint32_t stw = *(uint32_t*)ctx->h_status.p;
  if (stw & STATUS_NAN) return PCF_ERR_INVALID_KEY;
  if (stw & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
  if (stw & (STATUS_INTERNAL | STATUS_BOUNDS)) return PCF_ERR_INTERNAL;
  return PCF_OK;
}

}  // namespace

// A sort captured in a CUDA graph: one graph launch replays every kernel,
// copy and memset of the sort of fixed buffers and segments.  Its private
// context owns the scratch the graph's nodes point at, so no other call
// can move it.
struct pcf_graph {
  pcf_ctx* ctx = nullptr;
  const uint64_t* in_k = nullptr;
  const uint32_t* in_v = nullptr;
  uint64_t* out_k = nullptr;
  uint32_t* out_v = nullptr;
  std::vector<InSeg> segs;
  uint64_t n = 0;  // keys in all segments (0: every launch has nothing to do)
  uint32_t kt = 0;
  bool pairs = false;
  SortRecord rec;              // the plan the graph holds
  SortRecord pending;          // the plan of the last input that missed it
  bool has_pending = false;
  bool last_missed = false;    // the last launch did not replay
  DevBuf d_blob;               // the recording's read-backs on the device, for the guards
  HostBuf arena;               // the captured standard-sort rounds' uploads
  cudaStream_t cs = nullptr;   // the stream captures run on
  cudaGraphExec_t exec = nullptr;
  uint64_t sig = 0;            // the context's buffers_signature when exec was captured
  uint64_t replays = 0, eager_runs = 0;
  ~pcf_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cs) cudaStreamDestroy(cs);
  }
};

namespace {

// The decisions a capture depends on (what the guards compare): per level
// the next level's plan and the standard-sort items, and every read-back of
// the standard-sort rounds.
bool same_plan(const SortRecord& a, const SortRecord& b) {
  if (a.levels.size() != b.levels.size() || a.fb_lists.size() != b.fb_lists.size() ||
      a.rounds.size() != b.rounds.size())
    return false;
  for (size_t i = 0; i < a.levels.size(); ++i) {
    const LevelOut &x = a.levels[i], &y = b.levels[i];
    if (x.n_fb != y.n_fb || x.max_fb_n != y.max_fb_n ||
        memcmp(&x.plan, &y.plan, sizeof(PlanTotals)) != 0)
      return false;
  }
  for (size_t i = 0; i < a.fb_lists.size(); ++i) {
    if (a.fb_lists[i].size() != b.fb_lists[i].size() ||
        memcmp(a.fb_lists[i].data(), b.fb_lists[i].data(),
               a.fb_lists[i].size() * sizeof(FbItem)) != 0)
      return false;
  }
  for (size_t i = 0; i < a.rounds.size(); ++i)
    for (int k = 0; k < 4; ++k)
      if (a.rounds[i].got[k] != b.rounds[i].got[k]) return false;
  return true;
}

// Sorts the graph's input once without a graph, keeping its host decisions.
// A new graph captures the same sort from them.  A graph whose plan the
// input missed keeps its capture unless the plan just recorded is the one
// the previous miss recorded too (a plan that comes back is worth a
// capture; one input's plan alone is not: on inputs whose plans keep
// changing every launch would pay a capture).  If the capture fails the
// graph's launches sort without it.
pcf_status graph_build(pcf_graph* g, cudaStream_t st) {
  pcf_ctx* ctx = g->ctx;
  SortRecord nrec;
  pcf_status r = run_sort(ctx, g->in_k, g->in_v, g->out_k, g->out_v, g->segs, g->kt, g->pairs, st,
                          0xFFFFFFFFu, kSpinLimit, RUN_RECORD, &nrec);
  if (r != PCF_OK) {
    drain(ctx, st);
    return r;
  }
  ++g->eager_runs;
  if (g->n == 0) return PCF_OK;  // nothing to capture (no status buffers either)
  const bool first = g->eager_runs == 1;
  // a capture made before one of the context's buffers moved is stale
  if (g->exec && g->sig != buffers_signature(ctx)) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  const bool captured_plan = !first && same_plan(nrec, g->rec);
  if (g->exec && captured_plan) {  // the captured plan holds again: replay next time
    g->last_missed = false;
    g->has_pending = false;
    return PCF_OK;
  }
  const bool repeat = captured_plan || (g->has_pending && same_plan(nrec, g->pending));
  if (!first && !repeat) {
    g->pending = std::move(nrec);
    g->has_pending = true;
    g->last_missed = true;
    return PCF_OK;
  }
  g->last_missed = false;
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  g->rec = std::move(nrec);
  g->has_pending = false;
  // the read-backs the guards compare with, in one device blob
  const SortRecord& rec = g->rec;
  Replay rp;
  rp.rec = &rec;
  std::vector<uint8_t> blob;
  auto add = [&](const void* p, size_t bytes) {
    const size_t at = (blob.size() + 15) & ~(size_t)15;
    blob.resize(at + bytes);
    if (bytes) memcpy(blob.data() + at, p, bytes);
    return at;
  };
  rp.levels_at = add(rec.levels.data(), rec.levels.size() * sizeof(LevelOut));
  for (const auto& l : rec.fb_lists)
    rp.list_at.push_back(add(l.data(), l.size() * sizeof(FbItem)));
  for (const FbRound& rd : rec.rounds) {
    rp.round_at.emplace_back();
    for (int k = 0; k < 4; ++k)
      rp.round_at.back().push_back(add(rd.got[k].data(), rd.got[k].size()));
  }
  CK(ensure(g->d_blob, blob.size() + 16));
  CK(cudaMemcpy(g->d_blob.p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  CK(ensure_host(g->arena, rec.arena_bytes + 64));
  rp.d_blob = (const uint8_t*)g->d_blob.p;
  rp.arena = &g->arena;
  CK(cudaStreamBeginCapture(g->cs, cudaStreamCaptureModeThreadLocal));
  g->sig = buffers_signature(ctx);
  g_capturing = true;
  r = run_sort(ctx, g->in_k, g->in_v, g->out_k, g->out_v, g->segs, g->kt, g->pairs, g->cs,
               0xFFFFFFFFu, kSpinLimit, RUN_CAPTURE, nullptr, &rp);
  g_capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(g->cs, &graph);
  if (r == PCF_OK && e == cudaSuccess && graph &&
      cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess)
    g->exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();  // a failed capture leaves the graph eager, not the context broken
  return PCF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

uint32_t pcf_version(void) { return 100; }

const char* pcf_status_string(pcf_status s) {
  switch (s) {
    case PCF_OK: return "ok";
    case PCF_ERR_INVALID_ARG: return "invalid argument";
    case PCF_ERR_INVALID_KEY: return "invalid key (NaN)";
    case PCF_ERR_OOM: return "out of memory";
    case PCF_ERR_CUDA: return "CUDA error";
    case PCF_ERR_TIMEOUT: return "device wait timed out";
    case PCF_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

pcf_status pcf_ctx_create(pcf_ctx** out, int device) {
  if (!out) return PCF_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PCF_ERR_INVALID_ARG;
  }
  pcf_ctx* c = new (std::nothrow) pcf_ctx();
  if (!c) return PCF_ERR_OOM;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return PCF_ERR_CUDA;
  }
  *out = c;
  return PCF_OK;
}

pcf_status pcf_ctx_destroy(pcf_ctx* ctx) {
  if (!ctx) return PCF_OK;
  cudaSetDevice(ctx->device);
  delete ctx;
  return PCF_OK;
}

pcf_status pcf_ctx_set_policy(pcf_ctx* ctx, const pcf_policy* p) {
  if (!ctx || !p) return PCF_ERR_INVALID_ARG;
  Policy P{p->a_num, p->b_num, p->c_num, p->d_num, p->den, p->model, p->tau, p->range_mode, 0};
  if (!policy_ok(P)) return PCF_ERR_INVALID_ARG;
  ctx->policy = P;
  return PCF_OK;
}

pcf_status pcf_ctx_set_tuning(pcf_ctx* ctx, const pcf_tuning* t) {
  if (!ctx || !t) return PCF_ERR_INVALID_ARG;
  pcf_tuning n = ctx->tuning;
  if (t->max_digit_bits) n.max_digit_bits = t->max_digit_bits;
  if (t->tile_log2) n.tile_log2 = t->tile_log2;
  if (t->leaf_cap) n.leaf_cap = t->leaf_cap;
  if (t->leaf_mode) n.leaf_mode = t->leaf_mode;
  if (n.max_digit_bits < 4 || n.max_digit_bits > kMaxDigitBits) return PCF_ERR_INVALID_ARG;
  if (n.tile_log2 < 12 || n.tile_log2 > 18) return PCF_ERR_INVALID_ARG;
  if (n.leaf_cap < 64 || n.leaf_cap > 8192 || (n.leaf_cap & (n.leaf_cap - 1))) return PCF_ERR_INVALID_ARG;
  if (n.leaf_mode != 1 && n.leaf_mode != 2) return PCF_ERR_INVALID_ARG;
  ctx->tuning = n;
  return PCF_OK;
}

pcf_status pcf_ctx_get_tuning(const pcf_ctx* ctx, pcf_tuning* out) {
  if (!ctx || !out) return PCF_ERR_INVALID_ARG;
  *out = ctx->tuning;
  return PCF_OK;
}

pcf_status pcf_workspace_bytes(const pcf_ctx* ctx, uint64_t n_total, uint32_t S, pcf_key_type kt,
                               int pairs, uint64_t* out) {
  if (!out || (kt != PCF_KEY_F64 && kt != PCF_KEY_U64)) return PCF_ERR_INVALID_ARG;
  if (n_total > 0xFFFFFFFFull || (n_total && S == 0)) return PCF_ERR_INVALID_ARG;
  const Policy P = ctx ? ctx->policy : Policy{3, 3, 3, 3, 4, MODEL_PCF, 100, RANGE_ARRAY, 0};
  const pcf_tuning tu = ctx ? ctx->tuning : pcf_tuning{11, 14, 8192, 1};
  if (!policy_ok(P)) return PCF_ERR_INVALID_ARG;
  *out = workspace_bound(P, tu, n_total, S, pairs != 0);
  return PCF_OK;
}

pcf_status pcf_ctx_workspace_held(const pcf_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return PCF_ERR_INVALID_ARG;
  *out = workspace_held(ctx);
  return PCF_OK;
}

pcf_status pcf_ctx_sync(pcf_ctx* ctx, void* stream) {
  if (!ctx) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return ctx->last_status;
}

pcf_status pcf_ctx_reserve(pcf_ctx* ctx, uint64_t n_total, int pairs) {
  if (!ctx) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(ensure(ctx->tmp_k, n_total * 8));
  CK(ensure(ctx->tmp_aux, n_total * 2));
  CK(ensure(ctx->jbuf, n_total * 4));
  if (pairs) CK(ensure(ctx->tmp_v, n_total * 4));
  return PCF_OK;
}

pcf_status pcf_ctx_last_stats(const pcf_ctx* ctx, pcf_call_stats* out) {
  if (!ctx || !out) return PCF_ERR_INVALID_ARG;
  *out = ctx->stats;
  return PCF_OK;
}

pcf_status pcf_ctx_enable_timing(pcf_ctx* ctx, int on) {
  if (!ctx) return PCF_ERR_INVALID_ARG;
  ctx->timing = on != 0;
  return PCF_OK;
}

pcf_status pcf_ctx_stage_ms(const pcf_ctx* ctx, float out[8]) {
  if (!ctx || !out) return PCF_ERR_INVALID_ARG;
  for (int i = 0; i < 8; ++i) out[i] = ctx->stage_ms[i];
  return PCF_OK;
}

const char* pcf_last_cuda_error(const pcf_ctx* ctx) { return ctx ? ctx->last_err.c_str() : ""; }

static bool overlap(const void* a, const void* b, uint64_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x != y && x < y + bytes && y < x + bytes;
}

static pcf_status sort_common(pcf_ctx* ctx, const void* kin, const uint32_t* vin, void* kout,
                              uint32_t* vout, const std::vector<InSeg>& segs, uint64_t n,
                              pcf_key_type kt, bool pairs, void* stream) {
  if (!ctx) return PCF_ERR_INVALID_ARG;
  if (kt != PCF_KEY_F64 && kt != PCF_KEY_U64) return PCF_ERR_INVALID_ARG;
  if (n > 0xFFFFFFFFull) return PCF_ERR_INVALID_ARG;
  if (n == 0) return PCF_OK;
  if (!kin || !kout || (pairs && (!vin || !vout))) return PCF_ERR_INVALID_ARG;
  if (((uintptr_t)kin & 7) || ((uintptr_t)kout & 7)) return PCF_ERR_INVALID_ARG;
  if (pairs && (((uintptr_t)vin & 3) || ((uintptr_t)vout & 3))) return PCF_ERR_INVALID_ARG;
  if (overlap(kin, kout, n * 8)) return PCF_ERR_INVALID_ARG;
  if (pairs && overlap(vin, vout, n * 4)) return PCF_ERR_INVALID_ARG;
  if (!policy_ok(ctx->policy)) return PCF_ERR_INVALID_ARG;
  const pcf_status r = run_sort(ctx, (const uint64_t*)kin, vin, (uint64_t*)kout, vout, segs,
                               (uint32_t)kt, pairs, (cudaStream_t)stream);
  // a call that fails part-way returns with none of its work in flight
  if (r != PCF_OK) drain(ctx, (cudaStream_t)stream);
  ctx->last_status = r;
  return r;
}

pcf_status pcf_sort_keys(pcf_ctx* ctx, const void* d_in, void* d_out, uint64_t n, pcf_key_type kt,
                         uint64_t seed, void* stream) {
  std::vector<InSeg> segs{InSeg{0, n, 0, seed, 0}};
  // offsets in the kernels are relative to the buffer base
  return sort_common(ctx, d_in, nullptr, d_out, nullptr, segs, n, kt, false, stream);
}

pcf_status pcf_sort_pairs(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                          void* d_keys_out, uint32_t* d_vals_out, uint64_t n, pcf_key_type kt,
                          uint64_t seed, void* stream) {
  std::vector<InSeg> segs{InSeg{0, n, 0, seed, 0}};
  return sort_common(ctx, d_keys_in, d_vals_in, d_keys_out, d_vals_out, segs, n, kt, true,
                     stream);
}

pcf_status pcf_sort_segmented(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                              void* d_keys_out, uint32_t* d_vals_out, const uint64_t* h_offsets,
                              uint32_t S, pcf_key_type kt, uint64_t seed, void* stream) {
  if (!ctx || (!h_offsets && S)) return PCF_ERR_INVALID_ARG;
  if (S == 0) return PCF_OK;
  if (h_offsets[0] != 0) return PCF_ERR_INVALID_ARG;
  std::vector<InSeg> segs;
  segs.reserve(S);
  for (uint32_t s = 0; s < S; ++s) {
    if (h_offsets[s + 1] < h_offsets[s]) return PCF_ERR_INVALID_ARG;
    segs.push_back(InSeg{h_offsets[s], h_offsets[s + 1] - h_offsets[s], 0, seed + s, 0});
  }
  const bool pairs = d_vals_in != nullptr || d_vals_out != nullptr;
  return sort_common(ctx, d_keys_in, d_vals_in, d_keys_out, d_vals_out, segs, h_offsets[S], kt,
                     pairs, stream);
}

pcf_status pcf_sort_segmented_dev(pcf_ctx* ctx, const void* d_keys_in, const uint32_t* d_vals_in,
                                  void* d_keys_out, uint32_t* d_vals_out,
                                  const uint64_t* d_offsets, uint32_t S, uint64_t n_cap,
                                  pcf_key_type kt, uint64_t seed, void* stream) {
  if (!ctx || (!d_offsets && S) || ((uintptr_t)d_offsets & 7)) return PCF_ERR_INVALID_ARG;
  if (S == 0) return PCF_OK;
  if (S == 0xFFFFFFFFu) return PCF_ERR_INVALID_ARG;
  const cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  CK(ensure_host(ctx->h_offs, ((size_t)S + 1) * 8));
  // read on the sort's stream: after whatever produced the offsets there
  CK(launch_xfer(st, ctx->h_offs.dp, d_offsets, ((size_t)S + 1) * 8));
  CK(cudaStreamSynchronize(st));
  const uint64_t* h = (const uint64_t*)ctx->h_offs.p;
  if (h[S] > n_cap) return PCF_ERR_INVALID_ARG;  // (the rest is checked below)
  return pcf_sort_segmented(ctx, d_keys_in, d_vals_in, d_keys_out, d_vals_out, h, S, kt, seed,
                            stream);
}

pcf_status pcf_graph_create(pcf_graph** out, const pcf_ctx* like, const void* d_keys_in,
                            const uint32_t* d_vals_in, void* d_keys_out, uint32_t* d_vals_out,
                            const uint64_t* h_offsets, uint32_t S, pcf_key_type kt, uint64_t seed,
                            void* stream) {
  if (!out) return PCF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!like || (!h_offsets && S)) return PCF_ERR_INVALID_ARG;
  if (kt != PCF_KEY_F64 && kt != PCF_KEY_U64) return PCF_ERR_INVALID_ARG;
  if (S && h_offsets[0] != 0) return PCF_ERR_INVALID_ARG;
  std::vector<InSeg> segs;
  segs.reserve(S);
  for (uint32_t s = 0; s < S; ++s) {
    if (h_offsets[s + 1] < h_offsets[s]) return PCF_ERR_INVALID_ARG;
    segs.push_back(InSeg{h_offsets[s], h_offsets[s + 1] - h_offsets[s], 0, seed + s, 0});
  }
  const uint64_t n = S ? h_offsets[S] : 0;
  const bool pairs = d_vals_in != nullptr || d_vals_out != nullptr;
  if (n > 0xFFFFFFFFull) return PCF_ERR_INVALID_ARG;
  if (n) {
    if (!d_keys_in || !d_keys_out || (pairs && (!d_vals_in || !d_vals_out)))
      return PCF_ERR_INVALID_ARG;
    if (((uintptr_t)d_keys_in & 7) || ((uintptr_t)d_keys_out & 7)) return PCF_ERR_INVALID_ARG;
    if (pairs && (((uintptr_t)d_vals_in & 3) || ((uintptr_t)d_vals_out & 3)))
      return PCF_ERR_INVALID_ARG;
    // out of place only: a replay whose plan no longer holds sorts the
    // input again, so the graph must never write it
    if (d_keys_in == d_keys_out || overlap(d_keys_in, d_keys_out, n * 8))
      return PCF_ERR_INVALID_ARG;
    if (pairs && (d_vals_in == d_vals_out || overlap(d_vals_in, d_vals_out, n * 4)))
      return PCF_ERR_INVALID_ARG;
  }
  if (!policy_ok(like->policy)) return PCF_ERR_INVALID_ARG;
  pcf_graph* g = new (std::nothrow) pcf_graph();
  if (!g) return PCF_ERR_OOM;
  pcf_status r = pcf_ctx_create(&g->ctx, like->device);
  if (r != PCF_OK) {
    delete g;
    return r;
  }
  pcf_ctx* ctx = g->ctx;
  ctx->policy = like->policy;
  ctx->tuning = like->tuning;
  g->in_k = (const uint64_t*)d_keys_in;
  g->in_v = d_vals_in;
  g->out_k = (uint64_t*)d_keys_out;
  g->out_v = d_vals_out;
  g->segs = std::move(segs);
  g->n = n;
  g->kt = (uint32_t)kt;
  g->pairs = pairs;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (!e) e = cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking);
  if (e) {
    r = cuda_fail(ctx, e);
  } else {
    r = graph_build(g, (cudaStream_t)stream);
  }
  if (r != PCF_OK) {
    pcf_graph_destroy(g);
    return r;
  }
  *out = g;
  return PCF_OK;
}

pcf_status pcf_graph_launch(pcf_graph* g, void* stream, int* replayed) {
  if (replayed) *replayed = 0;
  if (!g) return PCF_ERR_INVALID_ARG;
  if (g->n == 0) return PCF_OK;
  pcf_ctx* ctx = g->ctx;
  const cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  if (g->exec && g->sig != buffers_signature(ctx)) {
    // a workspace buffer has moved since the capture: its nodes are stale
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  // after a miss the next input is sorted without the graph first (its
  // plan decides whether the graph replays again): inputs whose plans keep
  // changing pay one eager sort each, not a replay cut short and a sort
  if (g->exec && !g->last_missed) {
    CK(cudaGraphLaunch(g->exec, st));
    CK(launch_xfer(st, ctx->h_status.dp, ctx->status.p, 4));
    CK(cudaStreamSynchronize(st));
    const uint32_t stw = *(uint32_t*)ctx->h_status.p;
    if (!(stw & STATUS_ABORT)) {
      ++g->replays;
      if (replayed) *replayed = 1;
      return PCF_OK;
    }
    if (stw & STATUS_NAN) return PCF_ERR_INVALID_KEY;
    if (stw & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
    if (stw & (STATUS_INTERNAL | STATUS_BOUNDS)) return PCF_ERR_INTERNAL;
    // STATUS_REPLAN: this input takes another plan than the recorded one;
    // the graph stopped at that level's end and left the input as it was
    g->last_missed = true;
  }
  return graph_build(g, st);
}

pcf_status pcf_graph_info(const pcf_graph* g, int* captured, uint64_t* replays,
                          uint64_t* eager_runs) {
  if (!g) return PCF_ERR_INVALID_ARG;
  if (captured) *captured = g->exec != nullptr;
  if (replays) *replays = g->replays;
  if (eager_runs) *eager_runs = g->eager_runs;
  return PCF_OK;
}

pcf_status pcf_graph_destroy(pcf_graph* g) {
  if (!g) return PCF_OK;
  pcf_ctx* ctx = g->ctx;
  if (ctx) cudaSetDevice(ctx->device);
  delete g;  // the graph and its stream before the context's buffers
  pcf_ctx_destroy(ctx);
  return PCF_OK;
}

pcf_status pcf_sort_keys_host(pcf_ctx* ctx, void* h_keys, uint64_t n, pcf_key_type kt,
                              uint64_t seed, void* stream) {
  if (!ctx || (!h_keys && n)) return PCF_ERR_INVALID_ARG;
  if (n == 0) return PCF_OK;
  if (n > 0xFFFFFFFFull) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(ensure(ctx->host_keys, n * 8));
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(ctx->host_keys.p, h_keys, n * 8, cudaMemcpyHostToDevice, st));
  std::vector<InSeg> segs{InSeg{0, n, 0, seed, 0}};
  pcf_status s = sort_common(ctx, ctx->host_keys.p, nullptr, ctx->host_keys.p, nullptr, segs, n,
                             kt, false, stream);
  if (s != PCF_OK) return s;
  CK(cudaMemcpyAsync(h_keys, ctx->host_keys.p, n * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PCF_OK;
}

// Several arrays on HOST buffers, each sorted as pcf_sort_keys_host would
// sort it (seed + i for array i), with the copies of one array overlapping
// the sorts of its neighbours: three device slots rotate through upload
// (copy stream "in"), sort (the caller's stream) and download (copy stream
// "out"), ordered by events.  Host buffers should be pinned for the copies
// to overlap.
pcf_status pcf_sort_keys_host_batch(pcf_ctx* ctx, void* const* h_keys, const uint64_t* ns,
                                    uint32_t count, pcf_key_type kt, uint64_t seed,
                                    void* stream) {
  if (!ctx || (count && (!h_keys || !ns))) return PCF_ERR_INVALID_ARG;
  if (kt != PCF_KEY_F64 && kt != PCF_KEY_U64) return PCF_ERR_INVALID_ARG;
  uint64_t max_n = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (ns[i] > 0xFFFFFFFFull || (ns[i] && !h_keys[i])) return PCF_ERR_INVALID_ARG;
    max_n = std::max(max_n, ns[i]);
  }
  if (max_n == 0) return PCF_OK;
  CK(cudaSetDevice(ctx->device));
  CK(ctx->pipe.init());
  const size_t slot_bytes = (max_n * 8 + 255) & ~(size_t)255;
  CK(ensure(ctx->pipe_keys, slot_bytes * kPipeSlots));
  cudaStream_t st = (cudaStream_t)stream;
  CopyPipe& cp = ctx->pipe;
  auto slot_ptr = [&](uint32_t i) { return (char*)ctx->pipe_keys.p + (i % kPipeSlots) * slot_bytes; };
  // upload of array i into its slot, once the download of array i - 3 (the
  // slot's previous array) has left it
  auto upload = [&](uint32_t i) -> cudaError_t {
    const int k = (int)(i % kPipeSlots);
    cudaError_t e = cudaSuccess;
    if (i >= (uint32_t)kPipeSlots) e = cudaStreamWaitEvent(cp.in, cp.stored[k], 0);
    if (!e && ns[i]) e = cudaMemcpyAsync(slot_ptr(i), h_keys[i], ns[i] * 8, cudaMemcpyHostToDevice,
                                         cp.in);
    if (!e) e = cudaEventRecord(cp.loaded[k], cp.in);
    return e;
  };
  pcf_status status = PCF_OK;
  cudaError_t e = upload(0);
  for (uint32_t i = 0; i < count && !e && status == PCF_OK; ++i) {
    const int k = (int)(i % kPipeSlots);
    if (i + 1 < count && (e = upload(i + 1))) break;
    if ((e = cudaStreamWaitEvent(st, cp.loaded[k], 0))) break;
    std::vector<InSeg> segs{InSeg{0, ns[i], 0, seed + i, 0}};
    status = sort_common(ctx, slot_ptr(i), nullptr, slot_ptr(i), nullptr, segs, ns[i], kt, false,
                         stream);
    if (status != PCF_OK) break;
    if ((e = cudaEventRecord(cp.sorted[k], st))) break;
    if ((e = cudaStreamWaitEvent(cp.out, cp.sorted[k], 0))) break;
    if (ns[i] && (e = cudaMemcpyAsync(h_keys[i], slot_ptr(i), ns[i] * 8, cudaMemcpyDeviceToHost,
                                      cp.out)))
      break;
    if ((e = cudaEventRecord(cp.stored[k], cp.out))) break;
  }
  // return with no copy of this call in flight, whatever happened
  const cudaError_t e_in = cudaStreamSynchronize(cp.in);
  const cudaError_t e_out = cudaStreamSynchronize(cp.out);
  if (status != PCF_OK) return status;
  if (!e) e = e_in ? e_in : e_out;
  CK(e);
  return PCF_OK;
}

// Level-0 model-based bucketing only, with alpha, beta, gamma given: the
// bucket sizes of each array and the largest of them (the experiment of
// Sec. 4.2 behind Lemma pcf-divide-success-prob).  The same kernels as a
// sort's level 0 (range, model, sample + table, k_hist1), then a count.
pcf_status pcf_bucket_sizes(pcf_ctx* ctx, const void* d_keys, const uint64_t* h_offsets,
                            uint32_t S, pcf_key_type kt, uint64_t seed, uint64_t alpha,
                            uint64_t beta, uint64_t gamma, uint32_t* d_counts, uint64_t* h_max,
                            void* stream) {
  if (!ctx || !d_keys || !h_offsets || !h_max || S == 0) return PCF_ERR_INVALID_ARG;
  if (kt != PCF_KEY_F64 && kt != PCF_KEY_U64) return PCF_ERR_INVALID_ARG;
  if (alpha < 1 || beta < 1 || gamma < 1 || alpha > 0xFFFFFFFFull || beta >= 0xFFFFFFFFull ||
      gamma >= (1ull << (2 * kMaxDigitBits)))
    return PCF_ERR_INVALID_ARG;
  if (((uintptr_t)d_keys & 7) || h_offsets[0] != 0) return PCF_ERR_INVALID_ARG;
  std::vector<InSeg> segs(S);
  for (uint32_t s = 0; s < S; ++s) {
    const uint64_t a = h_offsets[s], b = h_offsets[s + 1];
    if (b < a + 2 || b - a > 0xFFFFFFFFull) return PCF_ERR_INVALID_ARG;
    segs[s] = InSeg{a, b - a, 0, seed + s, 0};
  }
  const uint64_t n_total = h_offsets[S];
  if (n_total > 0xFFFFFFFFull) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  LaunchCfg lc;
  lc.stream = st;
  lc.kt = (uint32_t)kt;
  lc.pairs = false;
  lc.launches = &ctx->stats.kernel_launches;
  lc.model = ctx->policy.model;
  lc.range_mode = ctx->policy.range_mode;
  ctx->stats = pcf_call_stats{};
  CK(ensure(ctx->status, 64));
  lc.status = as<uint32_t>(ctx->status);
  CK(cudaMemsetAsync(lc.status, 0, 16, st));
  CK(ensure_host(ctx->h_status, 64));
  CK(ensure(ctx->misc, 256));
  Params fixed;
  fixed.alpha = (uint32_t)alpha;
  fixed.beta = (uint32_t)beta;
  fixed.gamma = (uint32_t)gamma;
  fixed.delta = 0;
  Plan pl;
  plan_level(ctx->policy, ctx->tuning, ctx->pcache, segs, pl, &fixed);
  const PlanLayout PL = plan_layout(S);
  CK(ensure_host(ctx->h_stage, PL.bytes));
  CK(ensure(ctx->segs, PL.bytes));
  char* hs = (char*)ctx->h_stage.p;
  memcpy(hs, pl.segs.data(), S * sizeof(Seg));
  memcpy(hs + PL.o_rb, pl.range_base.data(), (S + 1) * 4);
  memcpy(hs + PL.o_k1, pl.k1_base.data(), (S + 1) * 4);
  memcpy(hs + PL.o_t1, pl.tile1_base.data(), (S + 1) * 4);
  memcpy(hs + PL.o_gb, pl.group_base.data(), (S + 1) * 8);
  memcpy(hs + PL.o_bb, pl.bucket_base.data(), (S + 1) * 8);
  CK(launch_xfer(st, ctx->segs.p, ctx->h_stage.dp, PL.bytes));
  const DevPlan dp = dev_plan(ctx->segs.p, PL);
  const uint32_t tile_keys = 1u << ctx->tuning.tile_log2;
  const uint64_t spin_limit = kSpinLimit;
  const bool srange = lc.range_mode == RANGE_SAMPLE;
  if (srange) {
    CK(launch_sample_range(lc, dp.segs, S, dp.k1, pl.k1_base[S], (const uint64_t*)d_keys));
    CK(launch_model(lc, dp.segs, S, 1));
    CK(launch_range(lc, dp.segs, S, dp.rb, pl.range_base[S], (const uint64_t*)d_keys,
                    kt == PCF_KEY_F64, SEG_NEEDRANGE));
    CK(launch_model(lc, dp.segs, S, 2));
  } else {
    CK(launch_range(lc, dp.segs, S, dp.rb, pl.range_base[S], (const uint64_t*)d_keys,
                    kt == PCF_KEY_F64));
    if (kt == PCF_KEY_F64) {
      CK(launch_xfer(st, ctx->h_status.dp, lc.status, 4));
      CK(cudaStreamSynchronize(st));
      if (*(uint32_t*)ctx->h_status.p & STATUS_NAN) return PCF_ERR_INVALID_KEY;
    }
    CK(launch_model(lc, dp.segs, S));
  }
  CK(ensure(ctx->tpool, pl.tpool * 4));
  CK(cudaMemsetAsync(ctx->tpool.p, 0, pl.tpool * 4, st));
  const uint64_t scan_max = std::max(pl.cmat1, pl.tpool);
  CK(ensure(ctx->sw, ((scan_max + kScanTile - 1) / kScanTile + 8) * 8));
  uint32_t* tile_counter = as<uint32_t>(ctx->misc);
  CK(launch_sample(lc, dp.segs, S, dp.k1, pl.k1_base[S], (const uint64_t*)d_keys,
                   as<uint32_t>(ctx->tpool)));
  CK(launch_table(lc, dp.segs, S, as<uint32_t>(ctx->tpool), pl.tpool, as<uint64_t>(ctx->sw),
                  tile_counter, spin_limit));
  CK(ensure(ctx->cmat1, pl.cmat1 * 4));
  CK(cudaMemsetAsync(ctx->cmat1.p, 0, pl.cmat1 * 4, st));
  CK(ensure(ctx->jbuf, n_total * 4));
  CK(launch_hist1(lc, dp.segs, S, dp.t1, pl.tile1_base[S], tile_keys, (const uint64_t*)d_keys,
                  as<uint32_t>(ctx->tpool), as<uint32_t>(ctx->cmat1), pl.dmax1,
                  as<uint32_t>(ctx->jbuf), srange && kt == PCF_KEY_F64));
  const size_t n_counts = (size_t)S * (gamma + 1);
  uint32_t* counts = d_counts;
  if (!counts) {
    CK(ensure(ctx->bcounts, n_counts * 4));
    counts = as<uint32_t>(ctx->bcounts);
  }
  CK(cudaMemsetAsync(counts, 0, n_counts * 4, st));
  CK(ensure(ctx->bmax, (size_t)S * 8));
  CK(launch_bucket_sizes(lc, dp.segs, S, dp.t1, pl.tile1_base[S], tile_keys,
                         as<uint32_t>(ctx->jbuf), counts, as<uint64_t>(ctx->bmax)));
  CK(ensure_host(ctx->h_items, (size_t)S * 8));
  CK(launch_xfer(st, ctx->h_items.dp, ctx->bmax.p, (size_t)S * 8));
  CK(launch_xfer(st, ctx->h_status.dp, lc.status, 4));
  CK(cudaStreamSynchronize(st));
  const uint32_t w = *(uint32_t*)ctx->h_status.p;
  if (w & STATUS_NAN) return PCF_ERR_INVALID_KEY;
  if (w & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
  memcpy(h_max, ctx->h_items.p, (size_t)S * 8);
  return PCF_OK;
}

// Device copy bandwidth with the passes' access pattern: reps copies of
// `bytes` from d_src to d_dst (16-byte aligned, bytes a multiple of 16),
// timed with CUDA events on `stream` after one untimed copy; *gb_per_s =
// 2 bytes (read + written) per copy / mean time.
pcf_status pcf_copy_bandwidth(pcf_ctx* ctx, const void* d_src, void* d_dst, uint64_t bytes,
                              uint32_t reps, void* stream, double* gb_per_s) {
  if (!ctx || !d_src || !d_dst || !gb_per_s || reps == 0 || bytes == 0 || (bytes & 15) ||
      (((uintptr_t)d_src | (uintptr_t)d_dst) & 15))
    return PCF_ERR_INVALID_ARG;
  if (overlap(d_src, d_dst, bytes)) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t grid = (uint32_t)ctx->num_sms * 8;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, e);
  }
  e = launch_copy128(st, d_src, d_dst, bytes / 16, grid);
  if (!e) e = cudaEventRecord(e0, st);
  for (uint32_t r = 0; r < reps && !e; ++r) e = launch_copy128(st, d_src, d_dst, bytes / 16, grid);
  if (!e) e = cudaEventRecord(e1, st);
  if (!e) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  *gb_per_s = ms > 0.f ? 2.0 * (double)bytes * reps / (ms * 1e-3) / 1e9 : 0.0;
  return PCF_OK;
}

// ---- self-test hooks (used by the test suite) ----

// The k-th device workspace allocation from now (0: the next) on this host
// thread fails as an out-of-memory error; k < 0 clears the injection.
void pcf_debug_fail_alloc_after(int64_t k) { g_fail_alloc_after = k < 0 ? -1 : k; }

// Host copy of the kernels' bin function, for CPU checks of the fast path.
// Returns 1 (and writes nothing) if the range [lo, hi] is degenerate.
int pcf_debug_bins_host(uint32_t kt, uint64_t lo_bits, uint64_t hi_bits, uint32_t beta,
                        const uint64_t* xs, uint64_t m, uint32_t* out, uint8_t* fast_decided) {
  BinModel M;
  if (make_bin_model(kt, lo_bits, hi_bits, beta, &M)) return 1;
  for (uint64_t i = 0; i < m; ++i) {
    out[i] = bin_of(M, xs[i]);
    if (fast_decided) fast_decided[i] = bin_fast_decides(M, xs[i]) ? 1 : 0;
  }
  return 0;
}

// Host copy of floor(n^{p/q}) and of the sample index stream.
uint64_t pcf_debug_root_floor(uint64_t n, uint32_t p, uint32_t q) { return root_floor(n, p, q); }
uint64_t pcf_debug_sample_index(uint64_t seed, uint64_t depth, uint64_t start, uint64_t n,
                                uint64_t j) {
  return sample_index(sample_state(seed, depth, start, n), j, n);
}

// Runs the decoupled-lookback scan on d_data[0..n) in place.  withhold_tile:
// a tile that never publishes (timeout test), or UINT32_MAX.
pcf_status pcf_debug_scan(pcf_ctx* ctx, uint32_t* d_data, uint64_t n, uint32_t withhold_tile,
                          uint64_t spin_limit, void* stream) {
  if (!ctx || (!d_data && n)) return PCF_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  CK(ensure(ctx->status, 64));
  CK(ensure(ctx->misc, 256));
  CK(ensure(ctx->sw, ((n + kScanTile - 1) / kScanTile + 8) * 8));
  CK(ensure_host(ctx->h_status, 64));
  LaunchCfg lc;
  lc.stream = st;
  lc.kt = 0;
  lc.pairs = false;
  lc.launches = nullptr;
  lc.status = as<uint32_t>(ctx->status);
  CK(cudaMemsetAsync(lc.status, 0, 16, st));
  CK(launch_scan(lc, d_data, n, nullptr, as<uint64_t>(ctx->sw), as<uint32_t>(ctx->misc),
                 withhold_tile, spin_limit ? spin_limit : kSpinLimit, nullptr));
  CK(launch_xfer(st, ctx->h_status.dp, lc.status, 4));
  CK(cudaStreamSynchronize(st));
  const uint32_t w = *(uint32_t*)ctx->h_status.p;
  if (w & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
  return PCF_OK;
}

// Level-0 model of one array on the device (for intermediate parity): the
// range bits, alpha..delta, status, and T (beta + 1 u32) copied to h_T.
pcf_status pcf_debug_level0(pcf_ctx* ctx, const void* d_keys, uint64_t n, pcf_key_type kt,
                            uint64_t seed, uint64_t* h_params8, uint32_t* h_T, uint64_t T_cap) {
  if (!ctx || !d_keys || n < 2 || !h_params8) return PCF_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  std::vector<InSeg> in{InSeg{0, n, 0, seed, 0}};
  Plan pl;
  plan_level(ctx->policy, ctx->tuning, ctx->pcache, in, pl);
  const uint32_t S = 1;
  CK(ensure(ctx->status, 64));
  CK(ensure(ctx->segs, sizeof(Seg) + 64));
  CK(ensure(ctx->bases, 64));
  CK(ensure(ctx->tpool, pl.tpool * 4));
  CK(ensure(ctx->done, 16));
  LaunchCfg lc;
  lc.stream = 0;
  lc.kt = kt;
  lc.pairs = false;
  lc.launches = nullptr;
  lc.status = as<uint32_t>(ctx->status);
  CK(cudaMemset(lc.status, 0, 4));
  CK(cudaMemcpy(ctx->segs.p, pl.segs.data(), sizeof(Seg), cudaMemcpyHostToDevice));
  uint32_t bases[4] = {0, pl.range_base[1], 0, pl.k1_base[1]};
  CK(cudaMemcpy(ctx->bases.p, bases, 16, cudaMemcpyHostToDevice));
  CK(cudaMemset(ctx->tpool.p, 0, pl.tpool * 4));
  CK(cudaMemset(ctx->done.p, 0, 4));
  CK(launch_range(lc, as<Seg>(ctx->segs), S, as<uint32_t>(ctx->bases), pl.range_base[1],
                  (const uint64_t*)d_keys, kt == PCF_KEY_F64));
  CK(launch_model(lc, as<Seg>(ctx->segs), S));
  CK(ensure(ctx->misc, 256));
  CK(ensure(ctx->sw, ((pl.tpool + kScanTile - 1) / kScanTile + 8) * 8));
  CK(launch_sample(lc, as<Seg>(ctx->segs), S, as<uint32_t>(ctx->bases) + 2, pl.k1_base[1],
                   (const uint64_t*)d_keys, as<uint32_t>(ctx->tpool)));
  CK(launch_table(lc, as<Seg>(ctx->segs), S, as<uint32_t>(ctx->tpool), pl.tpool,
                  as<uint64_t>(ctx->sw), as<uint32_t>(ctx->misc), kSpinLimit));
  Seg g;
  CK(cudaMemcpy(&g, ctx->segs.p, sizeof(Seg), cudaMemcpyDeviceToHost));
  h_params8[0] = g.alpha;
  h_params8[1] = g.beta;
  h_params8[2] = g.gamma;
  h_params8[3] = g.delta;
  h_params8[4] = bits_of_ord(g.ord_lo, kt);
  h_params8[5] = bits_of_ord(g.ord_hi, kt);
  h_params8[6] = g.status;
  h_params8[7] = 0;
  if (h_T && g.status == SEG_BUCKET) {
    if (T_cap < (uint64_t)g.beta + 1) return PCF_ERR_INVALID_ARG;
    CK(cudaMemcpy(h_T, ctx->tpool.p, ((size_t)g.beta + 1) * 4, cudaMemcpyDeviceToHost));
    for (uint32_t k = 0; k <= g.beta; ++k) h_T[k] = bucket_of_count(h_T[k] - g.tbase, g.alpha, g.gamma);
  }
  return PCF_OK;
}

}  // extern "C"

// pcf_leaf.cu -- buckets finished on chip, and the standard-sort fallback.
//
// k_leaf: one warp runs Learned-Sort (Algorithm 1 of Sato & Matsui, TMLR
// 2025, PCF model of Sec. 3.3) on one bucket held in shared memory: the
// range, alpha samples, the cumulative bin counts b, the bucket table, the
// stable counting scatter into gamma + 1 sub-buckets, and, per sub-bucket,
// the standard sort (|c| >= delta or |c| < tau) or another Learned-Sort
// step.  Pending steps live on a per-warp stack; their ranges are disjoint
// and longer than 16 keys, so at most cap/17 + 1 are pending at once.
//
// k_fb_*: the standard sort of buckets that are too large for one warp
// (|c| >= delta or a degenerate range): a stable merge sort -- block-local
// sorted runs, then merge passes split with merge-path partitioning.
#include "pcf_internal.h"

namespace pcf {

__device__ __forceinline__ uint32_t lmask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ uint32_t ub_dev(const T* a, uint32_t n, T v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

enum : uint32_t { JOB_LEARN = 0, JOB_SORT = 1 };
constexpr uint32_t kStdFlag = 0x80000000u;  // WorkItem.depth: standard sort only

struct Job {
  uint16_t o, c;
  uint16_t depth, kind;
};

struct WarpSmem {
  uint64_t* A;   // keys
  uint64_t* B;   // scatter target / merge scratch
  uint32_t* Av;  // values (pairs)
  uint32_t* Bv;
  uint16_t* J;   // sub-bucket id per key
  uint32_t* tab; // counts -> b -> T   (tmax)
  uint32_t* bcnt;  // sub-bucket sizes (gmax)
  uint32_t* bpos;  // sub-bucket cursors (gmax)
  Job* stack;
  BinModel* bm;
};

__host__ __device__ inline size_t warp_smem_bytes(uint32_t cap, bool pairs, uint32_t tmax,
                                                  uint32_t gmax) {
  size_t b = (size_t)cap * 16 + (pairs ? (size_t)cap * 8 : 0) + (size_t)cap * 2;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)tmax * 4 + (size_t)gmax * 8;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)(cap / 16 + 2) * sizeof(Job);
  b = (b + 15) & ~(size_t)15;
  b += sizeof(BinModel);
  return (b + 15) & ~(size_t)15;
}

__device__ inline WarpSmem carve_warp(uint8_t* p, uint32_t cap, bool pairs, uint32_t tmax,
                                      uint32_t gmax) {
  WarpSmem s;
  s.A = (uint64_t*)p;
  p += (size_t)cap * 8;
  s.B = (uint64_t*)p;
  p += (size_t)cap * 8;
  s.Av = s.Bv = nullptr;
  if (pairs) {
    s.Av = (uint32_t*)p;
    p += (size_t)cap * 4;
    s.Bv = (uint32_t*)p;
    p += (size_t)cap * 4;
  }
  s.J = (uint16_t*)p;
  p += (size_t)cap * 2;
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.tab = (uint32_t*)p;
  p += (size_t)tmax * 4;
  s.bcnt = (uint32_t*)p;
  p += (size_t)gmax * 4;
  s.bpos = (uint32_t*)p;
  p += (size_t)gmax * 4;
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.stack = (Job*)p;
  p += (size_t)(cap / 16 + 2) * sizeof(Job);
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.bm = (BinModel*)p;
  return s;
}

// ---------------------------------------------------------------------------
// standard sort (stable) of A[o, o+c) by one lane: insertion sort
// ---------------------------------------------------------------------------
template <bool PAIRS>
__device__ void lane_insertion_sort(uint64_t* A, uint32_t* Av, uint32_t o, uint32_t c,
                                    uint32_t kt) {
  for (uint32_t i = 1; i < c; ++i) {
    const uint64_t key = A[o + i];
    const uint64_t ok = ord_of(key, kt);
    uint32_t val = PAIRS ? Av[o + i] : 0u;
    uint32_t j = i;
    while (j > 0 && ord_of(A[o + j - 1], kt) > ok) {
      A[o + j] = A[o + j - 1];
      if (PAIRS) Av[o + j] = Av[o + j - 1];
      --j;
    }
    A[o + j] = key;
    if (PAIRS) Av[o + j] = val;
  }
}

// merge-path split: number of elements taken from L among the first k
// outputs of the stable merge of L (nL) and R (nR) (ties: L first)
__device__ __forceinline__ uint32_t merge_path(const uint64_t* L, uint32_t nL, const uint64_t* R,
                                               uint32_t nR, uint32_t k, uint32_t kt) {
  uint32_t lo = k > nR ? k - nR : 0u, hi = min(k, nL);
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (ord_of(L[mid], kt) <= ord_of(R[k - 1 - mid], kt)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// standard sort (stable) of A[o, o+c) by the whole warp: lane runs, then
// log2(32) rounds of merge-path merges through B.
template <bool PAIRS>
__device__ void warp_merge_sort(const WarpSmem& s, uint32_t o, uint32_t c, uint32_t kt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t r = (c + 31) / 32;
  {
    const uint32_t a = min(c, lane * r), b = min(c, a + r);
    if (b > a) lane_insertion_sort<PAIRS>(s.A, s.Av, o + a, b - a, kt);
  }
  __syncwarp();
  for (uint32_t w = r; w < c; w *= 2) {
    const uint32_t per = (c + 31) / 32;
    uint32_t a = min(c, lane * per);
    const uint32_t b = min(c, a + per);
    while (a < b) {
      const uint32_t p0 = (a / (2 * w)) * (2 * w);
      const uint32_t pe = min(c, p0 + 2 * w);
      const uint32_t nL = min(w, c - p0), nR = pe - p0 - nL;
      const uint64_t* L = s.A + o + p0;
      const uint64_t* R = L + nL;
      const uint32_t e = min(b, pe);
      uint32_t k = a - p0;
      uint32_t i = merge_path(L, nL, R, nR, k, kt), j = k - i;
      for (uint32_t q = a; q < e; ++q) {
        const bool takeL = j >= nR || (i < nL && ord_of(L[i], kt) <= ord_of(R[j], kt));
        if (takeL) {
          s.B[o + q] = L[i];
          if (PAIRS) s.Bv[o + q] = s.Av[o + p0 + i];
          ++i;
        } else {
          s.B[o + q] = R[j];
          if (PAIRS) s.Bv[o + q] = s.Av[o + p0 + nL + j];
          ++j;
        }
      }
      a = e;
    }
    __syncwarp();
    for (uint32_t q = lane; q < c; q += 32) {
      s.A[o + q] = s.B[o + q];
      if (PAIRS) s.Av[o + q] = s.Bv[o + q];
    }
    __syncwarp();
  }
}

// warp inclusive scan of v over lanes
__device__ __forceinline__ uint32_t wscan_incl(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t u = __shfl_up_sync(~0u, v, d);
    if (lane >= (uint32_t)d) v += u;
  }
  return v;
}

// ---------------------------------------------------------------------------
// One Learned-Sort step on A[o, o+c) (c >= tau).  Pushes sub-bucket jobs.
// Returns the updated stack depth (warp-uniform).
// ---------------------------------------------------------------------------
template <bool PAIRS>
__device__ uint32_t learned_step(const WarpSmem& s, uint32_t sp, uint32_t o, uint32_t c,
                                 uint32_t depth, uint64_t start, uint64_t seed, uint32_t kt,
                                 const Policy& P, const uint16_t* __restrict__ ptab,
                                 uint32_t stack_cap, uint32_t tmax, uint32_t gmax,
                                 uint32_t* status) {
  const uint32_t lane = threadIdx.x & 31;
  // range of the sub-array (Sec. 3.3: x_min, x_max)
  uint64_t mn = ~0ull, mx = 0ull;
  for (uint32_t i = lane; i < c; i += 32) {
    uint64_t v = ord_of(s.A[o + i], kt);
    mn = min(mn, v);
    mx = max(mx, v);
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d));
    mx = max(mx, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d));
  }
  if (mn == mx) return sp;  // one distinct value: already sorted
  Params pr;
  {
    const ushort4 q = __ldg(reinterpret_cast<const ushort4*>(ptab) + c);
    pr.alpha = q.x;
    pr.beta = q.y;
    pr.gamma = q.z;
    pr.delta = q.w;
  }
  if (pr.beta + 1 > tmax || pr.gamma + 1 > gmax) {
    if (lane == 0) atomicOr(status, STATUS_INTERNAL);
    warp_merge_sort<PAIRS>(s, o, c, kt);
    return sp;
  }
  int degen = 0;
  if (lane == 0) degen = make_bin_model(kt, bits_of_ord(mn, kt), bits_of_ord(mx, kt), pr.beta, s.bm);
  degen = __shfl_sync(~0u, degen, 0);
  __syncwarp();
  if (degen) {
    warp_merge_sort<PAIRS>(s, o, c, kt);
    return sp;
  }
  const BinModel& bm = *s.bm;
  // training: alpha samples counted per bin
  for (uint32_t k = lane; k <= pr.beta; k += 32) s.tab[k] = 0;
  __syncwarp();
  const uint64_t st = sample_state(seed, depth, start, c);
  for (uint32_t j = lane; j < pr.alpha; j += 32) {
    const uint32_t idx = (uint32_t)sample_index(st, j, c);
    atomicAdd(&s.tab[bin_of(bm, s.A[o + idx])], 1u);
  }
  __syncwarp();
  // b_k (inclusive scan) and the bucket table T[k] = floor(b_k gamma / alpha)
  {
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 <= pr.beta; k0 += 32) {
      const uint32_t k = k0 + lane;
      uint32_t v = k <= pr.beta ? s.tab[k] : 0u;
      uint32_t inc = wscan_incl(v) + carry;
      if (k <= pr.beta) s.tab[k] = bucket_of_count(inc, pr.alpha, pr.gamma);
      carry = __shfl_sync(~0u, inc, 31);
    }
  }
  for (uint32_t k = lane; k <= pr.gamma; k += 32) s.bcnt[k] = 0;
  __syncwarp();
  // inference: bucket of every key
  for (uint32_t i = lane; i < c; i += 32) {
    const uint32_t jj = s.tab[bin_of(bm, s.A[o + i])];
    s.J[i] = (uint16_t)jj;
    atomicAdd(&s.bcnt[jj], 1u);
  }
  __syncwarp();
  {
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 <= pr.gamma; k0 += 32) {
      const uint32_t k = k0 + lane;
      uint32_t v = k <= pr.gamma ? s.bcnt[k] : 0u;
      uint32_t inc = wscan_incl(v) + carry;
      if (k <= pr.gamma) s.bpos[k] = inc - v;
      carry = __shfl_sync(~0u, inc, 31);
    }
  }
  __syncwarp();
  // Append in input order: stable scatter A -> B
  const uint32_t lm = lmask_lt();
  for (uint32_t b0 = 0; b0 < c; b0 += 32) {
    const uint32_t i = b0 + lane;
    const bool v = i < c;
    const uint32_t jj = v ? s.J[i] : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(~0u, jj);
    const uint32_t prior = v ? s.bpos[jj] : 0u;
    __syncwarp();
    if (v && lane == (uint32_t)(__ffs(peers) - 1)) s.bpos[jj] = prior + __popc(peers);
    __syncwarp();
    if (v) {
      const uint32_t pos = o + prior + __popc(peers & lm);
      s.B[pos] = s.A[o + i];
      if (PAIRS) s.Bv[pos] = s.Av[o + i];
    }
  }
  __syncwarp();
  for (uint32_t i = lane; i < c; i += 32) {
    s.A[o + i] = s.B[o + i];
    if (PAIRS) s.Av[o + i] = s.Bv[o + i];
  }
  __syncwarp();
  // per sub-bucket decision of Alg. 1
  for (uint32_t k0 = 0; k0 <= pr.gamma; k0 += 32) {
    const uint32_t k = k0 + lane;
    const uint32_t ck = k <= pr.gamma ? s.bcnt[k] : 0u;
    const uint32_t ok = k <= pr.gamma ? s.bpos[k] - ck : 0u;
    const bool std = ck > 1 && (ck >= pr.delta || ck < P.tau);
    const bool tiny = std && ck <= 16;
    if (tiny) lane_insertion_sort<PAIRS>(s.A, s.Av, o + ok, ck, kt);
    const bool push_sort = std && !tiny;
    const bool push_learn = ck > 1 && !std;
    const uint32_t m = __ballot_sync(~0u, push_sort || push_learn);
    if (m) {
      const uint32_t slot = sp + __popc(m & lm);
      if (push_sort || push_learn) {
        if (slot < stack_cap) {
          Job jb;
          jb.o = (uint16_t)(o + ok);
          jb.c = (uint16_t)ck;
          jb.depth = (uint16_t)(depth + 1);
          jb.kind = push_sort ? JOB_SORT : JOB_LEARN;
          s.stack[slot] = jb;
        } else {
          atomicOr(status, STATUS_INTERNAL);
        }
      }
      sp = min(stack_cap, sp + __popc(m));
    }
  }
  __syncwarp();
  return sp;
}

// Learned-Sort of A[0, n) (or the standard sort when std_only)
template <bool PAIRS>
__device__ void warp_learned_sort(const WarpSmem& s, uint32_t n, uint32_t depth0, uint64_t start0,
                                  uint64_t seed, uint32_t kt, const Policy& P,
                                  const uint16_t* __restrict__ ptab, bool std_only,
                                  uint32_t stack_cap, uint32_t tmax, uint32_t gmax,
                                  uint32_t* status) {
  const uint32_t lane = threadIdx.x & 31;
  if (lane == 0) {
    Job jb;
    jb.o = 0;
    jb.c = (uint16_t)n;
    jb.depth = (uint16_t)depth0;
    jb.kind = std_only ? JOB_SORT : JOB_LEARN;
    s.stack[0] = jb;
  }
  __syncwarp();
  uint32_t sp = 1;
  while (sp > 0) {
    const Job jb = s.stack[sp - 1];
    --sp;
    __syncwarp();
    if (jb.kind == JOB_SORT || jb.c < P.tau) {
      if (jb.c > 1) warp_merge_sort<PAIRS>(s, jb.o, jb.c, kt);
    } else {
      sp = learned_step<PAIRS>(s, sp, jb.o, jb.c, jb.depth, start0 + jb.o, seed, kt, P, ptab,
                               stack_cap, tmax, gmax, status);
    }
    __syncwarp();
  }
}

template <bool PAIRS>
__global__ void __launch_bounds__(256) k_leaf(const WorkItem* __restrict__ items,
                                              const uint32_t* n_items, uint32_t* cursor,
                                              const uint64_t* __restrict__ src, uint64_t* dst,
                                              const uint32_t* __restrict__ src_v, uint32_t* dst_v,
                                              uint32_t kt, Policy P,
                                              const uint16_t* __restrict__ ptab, uint32_t cap,
                                              uint32_t tmax, uint32_t gmax, uint32_t* status) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t per = warp_smem_bytes(cap, PAIRS, tmax, gmax);
  const WarpSmem s = carve_warp(smem_raw + per * warp, cap, PAIRS, tmax, gmax);
  const uint32_t stack_cap = cap / 16 + 2;
  const uint32_t total = *n_items;
  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(cursor, 1u);
    it = __shfl_sync(~0u, it, 0);
    if (it >= total) break;
    const WorkItem w = items[it];
    if (w.n > cap) {  // never produced by the planner
      if (lane == 0) atomicOr(status, STATUS_INTERNAL);
      continue;
    }
    for (uint32_t i = lane; i < w.n; i += 32) {
      s.A[i] = __ldg(src + w.off + i);
      if (PAIRS) s.Av[i] = __ldg(src_v + w.off + i);
    }
    __syncwarp();
    const bool std_only = (w.depth & kStdFlag) != 0;
    warp_learned_sort<PAIRS>(s, w.n, w.depth & ~kStdFlag, w.start, w.seed, kt, P, ptab, std_only,
                             stack_cap, tmax, gmax, status);
    __syncwarp();
    for (uint32_t i = lane; i < w.n; i += 32) {
      dst[w.off + i] = s.A[i];
      if (PAIRS) dst_v[w.off + i] = s.Av[i];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Fallback standard sort of large buckets: stable merge sort
// ---------------------------------------------------------------------------
// per item range -> ord_lohi[2i], [2i+1]; tiles of kRangeTile
__global__ void __launch_bounds__(256) k_fb_range(const FbItem* items, uint32_t n_items,
                                                  const uint32_t* tile_base,
                                                  const uint64_t* __restrict__ keys, uint32_t kt,
                                                  uint64_t* ord_lohi) {
  const uint32_t t = blockIdx.x;
  const uint32_t i = ub_dev(tile_base, n_items + 1, t) - 1;
  const FbItem it = items[i];
  const uint64_t base = it.off + (uint64_t)(t - tile_base[i]) * kRangeTile;
  const uint64_t end = min(it.off + it.n, base + kRangeTile);
  uint64_t mn = ~0ull, mx = 0;
  for (uint64_t q = base + threadIdx.x; q < end; q += 256) {
    uint64_t o = ord_of(__ldg(keys + q), kt);
    mn = min(mn, o);
    mx = max(mx, o);
  }
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d));
    mx = max(mx, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin((unsigned long long*)&ord_lohi[2 * i], (unsigned long long)mn);
    atomicMax((unsigned long long*)&ord_lohi[2 * i + 1], (unsigned long long)mx);
  }
}

// block-local stable sort of kMergeTile-key runs (in place)
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_fb_block_sort(const FbItem* items, uint32_t n_items,
                                                       const uint32_t* tile_base,
                                                       const uint64_t* ord_lohi, uint64_t* keys,
                                                       uint32_t* vals, uint32_t kt) {
  __shared__ uint64_t sk[2][kMergeTile];
  __shared__ uint32_t sv[PAIRS ? 2 : 1][PAIRS ? kMergeTile : 1];
  const uint32_t t = blockIdx.x;
  const uint32_t i = ub_dev(tile_base, n_items + 1, t) - 1;
  if (ord_lohi[2 * i] == ord_lohi[2 * i + 1]) return;  // one value: sorted
  const FbItem it = items[i];
  const uint64_t base = it.off + (uint64_t)(t - tile_base[i]) * kMergeTile;
  const uint32_t cnt = (uint32_t)min((uint64_t)kMergeTile, it.off + it.n - base);
  for (uint32_t q = threadIdx.x; q < cnt; q += 256) {
    sk[0][q] = keys[base + q];
    if (PAIRS) sv[0][q] = vals[base + q];
  }
  __syncthreads();
  // each thread: insertion sort of 8 consecutive keys
  {
    const uint32_t a = min(cnt, threadIdx.x * 8u), b = min(cnt, a + 8u);
    for (uint32_t x = a + 1; x < b; ++x) {
      uint64_t key = sk[0][x];
      uint32_t val = PAIRS ? sv[0][x] : 0u;
      uint64_t ok = ord_of(key, kt);
      uint32_t y = x;
      while (y > a && ord_of(sk[0][y - 1], kt) > ok) {
        sk[0][y] = sk[0][y - 1];
        if (PAIRS) sv[0][y] = sv[0][y - 1];
        --y;
      }
      sk[0][y] = key;
      if (PAIRS) sv[0][y] = val;
    }
  }
  __syncthreads();
  int cur = 0;
  for (uint32_t w = 8; w < cnt; w *= 2) {
    const uint32_t a = min(cnt, threadIdx.x * 8u), b = min(cnt, a + 8u);
    if (a < b) {
      const uint32_t p0 = (a / (2 * w)) * (2 * w);
      const uint32_t pe = min(cnt, p0 + 2 * w);
      const uint32_t nL = min(w, cnt - p0), nR = pe - p0 - nL;
      const uint64_t* L = sk[cur] + p0;
      const uint64_t* R = L + nL;
      uint32_t k = a - p0;
      uint32_t ii = merge_path(L, nL, R, nR, k, kt), jj = k - ii;
      for (uint32_t q = a; q < b; ++q) {
        const bool takeL = jj >= nR || (ii < nL && ord_of(L[ii], kt) <= ord_of(R[jj], kt));
        if (takeL) {
          sk[cur ^ 1][q] = L[ii];
          if (PAIRS) sv[cur ^ 1][q] = sv[cur][p0 + ii];
          ++ii;
        } else {
          sk[cur ^ 1][q] = R[jj];
          if (PAIRS) sv[cur ^ 1][q] = sv[cur][p0 + nL + jj];
          ++jj;
        }
      }
    }
    cur ^= 1;
    __syncthreads();
  }
  for (uint32_t q = threadIdx.x; q < cnt; q += 256) {
    keys[base + q] = sk[cur][q];
    if (PAIRS) vals[base + q] = sv[cur][q];
  }
}

// global merge pass: runs of width w -> 2w, src -> dst, kMergeTile outputs
// per CTA.  Items with one value are skipped (their keys stay in `src`
// slots of both buffers' views; the host copies nothing for them).
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_fb_merge(const FbItem* items, uint32_t n_items,
                                                  const uint32_t* tile_base,
                                                  const uint64_t* ord_lohi, uint64_t w,
                                                  const uint64_t* __restrict__ src, uint64_t* dst,
                                                  const uint32_t* __restrict__ src_v,
                                                  uint32_t* dst_v, uint32_t kt) {
  __shared__ uint64_t sk[kMergeTile];
  __shared__ uint32_t sv[PAIRS ? kMergeTile : 1];
  __shared__ uint32_t s_split[2];
  const uint32_t t = blockIdx.x;
  const uint32_t i = ub_dev(tile_base, n_items + 1, t) - 1;
  if (ord_lohi[2 * i] == ord_lohi[2 * i + 1]) return;
  const FbItem it = items[i];
  const uint64_t a = (uint64_t)(t - tile_base[i]) * kMergeTile;  // output offset in the item
  const uint32_t cnt = (uint32_t)min((uint64_t)kMergeTile, it.n - a);
  const uint64_t p0 = (a / (2 * w)) * (2 * w);
  const uint64_t pe = min(it.n, p0 + 2 * w);
  const uint64_t nL = min(w, it.n - p0), nR = pe - p0 - nL;
  const uint64_t* L = src + it.off + p0;
  const uint64_t* R = L + nL;
  const uint64_t k0 = a - p0, k1 = k0 + cnt;
  if (threadIdx.x < 2) {
    const uint64_t k = threadIdx.x ? k1 : k0;
    uint64_t lo = k > nR ? k - nR : 0, hi = min(k, nL);
    while (lo < hi) {
      uint64_t mid = (lo + hi) >> 1;
      if (ord_of(L[mid], kt) <= ord_of(R[k - 1 - mid], kt)) lo = mid + 1;
      else hi = mid;
    }
    s_split[threadIdx.x] = (uint32_t)lo;
  }
  __syncthreads();
  // the tile's inputs: L[i0, i1) and R[j0, j1), i1 - i0 + j1 - j0 = cnt
  const uint64_t i0 = s_split[0], i1 = s_split[1];
  const uint64_t j0 = k0 - i0, j1 = k1 - i1;
  const uint32_t nl = (uint32_t)(i1 - i0), nr = (uint32_t)(j1 - j0);
  for (uint32_t q = threadIdx.x; q < cnt; q += 256) {
    const bool fromL = q < nl;
    sk[q] = fromL ? L[i0 + q] : R[j0 + (q - nl)];
    if (PAIRS) sv[q] = fromL ? src_v[it.off + p0 + i0 + q] : src_v[it.off + p0 + nL + j0 + (q - nl)];
  }
  __syncthreads();
  const uint32_t qa = min(cnt, threadIdx.x * 8u), qb = min(cnt, qa + 8u);
  if (qa < qb) {
    const uint64_t* SL = sk;
    const uint64_t* SR = sk + nl;
    uint32_t ii = merge_path(SL, nl, SR, nr, qa, kt), jj = qa - ii;
    for (uint32_t q = qa; q < qb; ++q) {
      const bool takeL = jj >= nr || (ii < nl && ord_of(SL[ii], kt) <= ord_of(SR[jj], kt));
      const uint32_t from = takeL ? ii : nl + jj;
      dst[it.off + a + q] = sk[from];
      if (PAIRS) dst_v[it.off + a + q] = sv[from];
      if (takeL) ++ii;
      else ++jj;
    }
  }
}

// copy tmp -> out for items that were merged an odd number of times
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_fb_copy(const FbItem* items, uint32_t n_items,
                                                 const uint32_t* tile_base,
                                                 const uint64_t* ord_lohi, const uint64_t* src,
                                                 uint64_t* dst, const uint32_t* src_v,
                                                 uint32_t* dst_v, const uint64_t* orig,
                                                 const uint32_t* orig_v) {
  const uint32_t t = blockIdx.x;
  const uint32_t i = ub_dev(tile_base, n_items + 1, t) - 1;
  if (ord_lohi[2 * i] == ord_lohi[2 * i + 1]) {  // never moved: copy from where it is
    src = orig;
    src_v = orig_v;
  }
  if (src == dst) return;
  const FbItem it = items[i];
  const uint64_t base = it.off + (uint64_t)(t - tile_base[i]) * kMergeTile;
  const uint64_t end = min(it.off + it.n, base + kMergeTile);
  for (uint64_t q = base + threadIdx.x; q < end; q += 256) {
    dst[q] = src[q];
    if (PAIRS) dst_v[q] = src_v[q];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline uint32_t cdiv32(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

cudaError_t launch_leaf(const LaunchCfg& c, const WorkItem* items, const uint32_t* n_items,
                        uint32_t* cursor, const uint64_t* src, uint64_t* dst,
                        const uint32_t* src_v, uint32_t* dst_v, Policy P, const uint16_t* ptab,
                        uint32_t cap, uint32_t tmax, uint32_t gmax, uint32_t warps_per_cta,
                        uint32_t grid) {
  const size_t sm = warp_smem_bytes(cap, c.pairs, tmax, gmax) * warps_per_cta;
  cudaError_t e;
  if (c.pairs) {
    if ((e = cudaFuncSetAttribute(k_leaf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    k_leaf<true><<<grid, 32 * warps_per_cta, sm, c.stream>>>(items, n_items, cursor, src, dst,
                                                             src_v, dst_v, c.kt, P, ptab, cap,
                                                             tmax, gmax, c.status);
    count_launch(c);
  } else {
    if ((e = cudaFuncSetAttribute(k_leaf<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    k_leaf<false><<<grid, 32 * warps_per_cta, sm, c.stream>>>(items, n_items, cursor, src, dst,
                                                              src_v, dst_v, c.kt, P, ptab, cap,
                                                              tmax, gmax, c.status);
    count_launch(c);
  }
  return cudaGetLastError();
}

size_t leaf_smem_per_warp(uint32_t cap, bool pairs, uint32_t tmax, uint32_t gmax) {
  return warp_smem_bytes(cap, pairs, tmax, gmax);
}

cudaError_t launch_fb_range(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                            const uint32_t* tile_base, uint32_t n_tiles, const uint64_t* keys,
                            uint64_t* ord_lohi) {
  if (!n_tiles) return cudaSuccess;
  k_fb_range<<<n_tiles, 256, 0, c.stream>>>(items, n_items, tile_base, keys, c.kt, ord_lohi);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_fb_sort(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint32_t* mtile_base, uint32_t n_mtiles, uint64_t max_n,
                           const uint64_t* ord_lohi, uint64_t* keys, uint64_t* tmp,
                           uint32_t* vals, uint32_t* tmp_v, uint64_t* final_k,
                           uint32_t* final_v) {
  if (!n_mtiles) return cudaSuccess;
  if (c.pairs) {
    k_fb_block_sort<true><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi,
                                                          keys, vals, c.kt);
  } else {
    k_fb_block_sort<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi,
                                                           keys, vals, c.kt);
  }
  count_launch(c);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  uint64_t* A = keys;
  uint64_t* B = tmp;
  uint32_t* Av = vals;
  uint32_t* Bv = tmp_v;
  for (uint64_t w = kMergeTile; w < max_n; w *= 2) {
    if (c.pairs) {
      k_fb_merge<true><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, w, A,
                                                       B, Av, Bv, c.kt);
    } else {
      k_fb_merge<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, w, A,
                                                        B, Av, Bv, c.kt);
    }
    count_launch(c);
    if ((e = cudaGetLastError())) return e;
    uint64_t* tk = A;
    A = B;
    B = tk;
    uint32_t* tv = Av;
    Av = Bv;
    Bv = tv;
  }
  // items with one distinct value were never moved: they are in `keys`
  if (A != final_k || keys != final_k) {
    if (c.pairs) {
      k_fb_copy<true><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, A,
                                                      final_k, Av, final_v, keys, vals);
    } else {
      k_fb_copy<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, A,
                                                       final_k, nullptr, nullptr, keys, nullptr);
    }
    count_launch(c);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

}  // namespace pcf

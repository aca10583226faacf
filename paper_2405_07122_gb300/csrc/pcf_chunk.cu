// pcf_chunk.cu -- buckets finished on chip, a window of them per CTA.
//
// Every bucket of a global level that fits on chip is a Learned-Sort call
// (Algorithm 1 of Sato & Matsui, TMLR 2025, PCF model of Sec. 3.3).  k_chunk
// gives one CTA the buckets that start in a window of H keys; it loads them
// into shared memory and runs their recursion in rounds, with the work of
// all of the window's sub-arrays done together:
//   - a warp per sub-array: x_min/x_max, then (lane 0) alpha..delta and the
//     bin constants;
//   - a thread per sample: alpha draws, counted per bin (Sec. 3.3);
//   - a warp per sub-array: b_k (scan) and its bucket table floor(b_k gamma/alpha);
//   - a thread per key: its bucket (Alg. 1);
//   - a warp per sub-array: the stable scatter into buckets ("Append");
//   - a thread per new bucket: Alg. 1's decision -- Standard-Sort when
//     |c| >= delta or |c| < tau (tiny ones insertion-sorted on the spot),
//     else another round.
// Standard-Sorts of more than 16 keys run last, a warp each (merge sort).
#include "pcf_internal.h"

namespace pcf {

namespace chunk {

__device__ __forceinline__ uint32_t lanemask_lt_() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t wscan(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(~0u, v, d);
    if (lane >= (uint32_t)d) v += u;
  }
  return v;
}

constexpr uint32_t kMaxActive = 64;   // sub-arrays learned per round
constexpr uint32_t kThreads = 256;
constexpr uint32_t kTinySort = 16;    // sorted by one thread

struct LearnItem {  // a pending Learned-Sort call
  uint16_t o, n;
  uint16_t depth, pad;
  uint64_t start, seed;
};

struct SortItem {  // a pending Standard-Sort of more than kTinySort keys
  uint16_t o, n;
};

struct Active {  // a Learned-Sort call of this round
  BinModel bm;
  uint64_t state;  // sample stream
  uint64_t start, seed;
  uint32_t o, n, depth, ok;  // ok: 1 bucketed, 0 done or sent to Standard-Sort
  uint32_t alpha, beta, gamma, delta;
  uint32_t tbase, cbase, sbase;
};

struct Smem {
  uint64_t *A, *B;
  uint32_t *Av, *Bv;
  uint8_t* own;    // [cap] position belongs to one of this window's buckets
  uint16_t* sid;   // [cap] active sub-array of the position (0xFFFF none)
  uint16_t* J;     // [cap] bucket of the position within its sub-array
  LearnItem* learn;
  SortItem* sorts;
  Active* act;
  uint32_t* tab;    // [tmax] counts -> bucket table
  uint32_t* ccnt;   // [kmax] bucket sizes
  uint32_t* cstart; // [kmax] bucket starts
  uint32_t* cpos;   // [kmax] scatter cursors
};

struct Geometry {
  uint32_t cap, tmax, kmax, max_learn, max_sorts;
};

__host__ __device__ inline size_t smem_bytes(const Geometry& g, bool pairs) {
  size_t b = (size_t)g.cap * 16 + (pairs ? (size_t)g.cap * 8 : 0);
  b += (size_t)g.cap * (1 + 2 + 2);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)g.max_learn * sizeof(LearnItem) + (size_t)g.max_sorts * sizeof(SortItem);
  b = (b + 15) & ~(size_t)15;
  b += (size_t)kMaxActive * sizeof(Active);
  b += (size_t)g.tmax * 4 + (size_t)g.kmax * 12;
  return b + 64;
}

__device__ inline Smem carve(uint8_t* p, const Geometry& g, bool pairs) {
  Smem s;
  s.A = (uint64_t*)p;
  p += (size_t)g.cap * 8;
  s.B = (uint64_t*)p;
  p += (size_t)g.cap * 8;
  s.Av = s.Bv = nullptr;
  if (pairs) {
    s.Av = (uint32_t*)p;
    p += (size_t)g.cap * 4;
    s.Bv = (uint32_t*)p;
    p += (size_t)g.cap * 4;
  }
  s.own = p;
  p += g.cap;
  s.sid = (uint16_t*)p;
  p += (size_t)g.cap * 2;
  s.J = (uint16_t*)p;
  p += (size_t)g.cap * 2;
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.learn = (LearnItem*)p;
  p += (size_t)g.max_learn * sizeof(LearnItem);
  s.sorts = (SortItem*)p;
  p += (size_t)g.max_sorts * sizeof(SortItem);
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.act = (Active*)p;
  p += (size_t)kMaxActive * sizeof(Active);
  s.tab = (uint32_t*)p;
  p += (size_t)g.tmax * 4;
  s.ccnt = (uint32_t*)p;
  p += (size_t)g.kmax * 4;
  s.cstart = (uint32_t*)p;
  p += (size_t)g.kmax * 4;
  s.cpos = (uint32_t*)p;
  return s;
}

// stable insertion sort of A[o, o+n) by one thread
template <bool PAIRS>
__device__ void thread_sort(uint64_t* A, uint32_t* Av, uint32_t o, uint32_t n, uint32_t kt) {
  for (uint32_t i = 1; i < n; ++i) {
    const uint64_t key = A[o + i];
    const uint64_t ok = ord_of(key, kt);
    const uint32_t val = PAIRS ? Av[o + i] : 0u;
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

// merge-path split (ties: left first)
__device__ __forceinline__ uint32_t mpath(const uint64_t* L, uint32_t nL, const uint64_t* R,
                                          uint32_t nR, uint32_t k, uint32_t kt) {
  uint32_t lo = k > nR ? k - nR : 0u, hi = min(k, nL);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (ord_of(L[mid], kt) <= ord_of(R[k - 1 - mid], kt)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// stable merge sort of A[o, o+c) by one warp (B[o, o+c) as scratch)
template <bool PAIRS>
__device__ void warp_sort(uint64_t* A, uint64_t* B, uint32_t* Av, uint32_t* Bv, uint32_t o,
                          uint32_t c, uint32_t kt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t r = (c + 31) / 32;
  {
    const uint32_t a = min(c, lane * r), b = min(c, a + r);
    if (b > a) thread_sort<PAIRS>(A, Av, o + a, b - a, kt);
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
      const uint64_t* L = A + o + p0;
      const uint64_t* R = L + nL;
      const uint32_t e = min(b, pe);
      const uint32_t k = a - p0;
      uint32_t i = mpath(L, nL, R, nR, k, kt), j = k - i;
      for (uint32_t q = a; q < e; ++q) {
        const bool takeL = j >= nR || (i < nL && ord_of(L[i], kt) <= ord_of(R[j], kt));
        if (takeL) {
          B[o + q] = L[i];
          if (PAIRS) Bv[o + q] = Av[o + p0 + i];
          ++i;
        } else {
          B[o + q] = R[j];
          if (PAIRS) Bv[o + q] = Av[o + p0 + nL + j];
          ++j;
        }
      }
      a = e;
    }
    __syncwarp();
    for (uint32_t q = lane; q < c; q += 32) {
      A[o + q] = B[o + q];
      if (PAIRS) Av[o + q] = Bv[o + q];
    }
    __syncwarp();
  }
}

}  // namespace chunk

using namespace chunk;

// first record of every window (a thread per window; all searches overlap)
__global__ void k_chunk_first(const BRec* __restrict__ br, uint32_t nb, uint64_t wbase, uint32_t H,
                              uint32_t n_windows, uint32_t* first) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n_windows) return;
  const uint64_t v = wbase + (uint64_t)k * H;
  uint32_t a = 0, b = nb;
  while (a < b) {
    const uint32_t m = (a + b) >> 1;
    if ((uint64_t)br[m].off < v) a = m + 1;
    else b = m;
  }
  first[k] = a;
}

template <bool PAIRS>
__global__ void __launch_bounds__(256) k_chunk(const BRec* __restrict__ br,
                                               const uint32_t* __restrict__ first,
                                               uint64_t wbase, uint32_t H, Geometry geo,
                                               const uint64_t* __restrict__ X,
                                               const uint32_t* __restrict__ Xv, uint64_t* out,
                                               uint32_t* out_v, uint32_t kt, Policy P,
                                               const uint16_t* __restrict__ ptab,
                                               uint32_t* status) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint32_t s_b[2], s_nlearn, s_nsort, s_nact, s_T, s_K, s_S, s_overflow;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lm = lanemask_lt_();
  Smem sm = carve(smem_raw, geo, PAIRS);
  const uint32_t cap = geo.cap;
  const uint64_t lo = wbase + (uint64_t)blockIdx.x * H;
  // buckets starting in [lo, lo + H)
  if (tid < 2) s_b[tid] = first[blockIdx.x + tid];
  if (tid == 0) {
    s_nlearn = 0;
    s_nsort = 0;
    s_overflow = 0;
  }
  __syncthreads();
  const uint32_t b0 = s_b[0], b1 = s_b[1];
  if (b0 >= b1) return;
  for (uint32_t i = tid; i < (cap + 15) / 16; i += kThreads)
    reinterpret_cast<uint4*>(sm.own)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < cap; i += kThreads) sm.sid[i] = 0xFFFFu;
  __syncthreads();
  // the window's on-chip buckets become the first work items
  for (uint32_t B = b0 + tid; B < b1; B += kThreads) {
    const BRec r = br[B];
    if (!(r.kind & BK_LEAF)) continue;
    const uint32_t rel = (uint32_t)(r.off - lo);
    if (r.kind & BK_STD) {
      const uint32_t i = atomicAdd(&s_nsort, 1u);
      if (i < geo.max_sorts) sm.sorts[i] = SortItem{(uint16_t)rel, (uint16_t)r.n};
      else s_overflow = 1;
    } else {
      const uint32_t i = atomicAdd(&s_nlearn, 1u);
      if (i < geo.max_learn) {
        LearnItem it;
        it.o = (uint16_t)rel;
        it.n = (uint16_t)r.n;
        it.depth = (uint16_t)r.depth;
        it.pad = 0;
        it.start = r.start;
        it.seed = r.seed;
        sm.learn[i] = it;
      } else {
        s_overflow = 1;
      }
    }
  }
  __syncthreads();
  if (s_overflow) {
    if (tid == 0) atomicOr(status, STATUS_INTERNAL);
    return;
  }
  // positions owned by the window's buckets; load them
  {
    const uint32_t nl = s_nlearn, ns = s_nsort;
    for (uint32_t i = warp; i < nl + ns; i += kThreads / 32) {
      const uint32_t o = i < nl ? sm.learn[i].o : sm.sorts[i - nl].o;
      const uint32_t n = i < nl ? sm.learn[i].n : sm.sorts[i - nl].n;
      for (uint32_t q = lane; q < n; q += 32) sm.own[o + q] = 1;
    }
  }
  __syncthreads();
  for (uint32_t p = tid; p < cap; p += kThreads) {
    if (sm.own[p]) {
      sm.A[p] = __ldg(X + lo + p);
      if (PAIRS) sm.Av[p] = __ldg(Xv + lo + p);
    }
  }
  __syncthreads();

  // ---- rounds of Learned-Sort steps
  while (s_nlearn > 0) {
    // select this round's sub-arrays (budgets: tables, buckets, count)
    if (tid == 0) {
      uint32_t na = 0, T = 0, K = 0, S = 0;
      const uint32_t nl = s_nlearn;
      while (na < nl && na < kMaxActive) {
        const LearnItem it = sm.learn[na];
        const ushort4 q = __ldg(reinterpret_cast<const ushort4*>(ptab) + it.n);
        if (T + q.y + 1u > geo.tmax || K + q.z + 1u > geo.kmax) break;
        Active& a = sm.act[na];
        a.o = it.o;
        a.n = it.n;
        a.depth = it.depth;
        a.start = it.start;
        a.seed = it.seed;
        a.alpha = q.x;
        a.beta = q.y;
        a.gamma = q.z;
        a.delta = q.w;
        a.tbase = T;
        a.cbase = K;
        a.sbase = S;
        T += q.y + 1u;
        K += q.z + 1u;
        S += q.x;
        ++na;
      }
      if (na == 0) s_overflow = 1;  // a single call larger than the budgets
      s_nact = na;
      s_T = T;
      s_K = K;
      s_S = S;
      // the rest stays pending
      for (uint32_t i = na; i < nl; ++i) sm.learn[i - na] = sm.learn[i];
      s_nlearn = nl - na;
    }
    __syncthreads();
    if (s_overflow) {
      if (tid == 0) atomicOr(status, STATUS_INTERNAL);
      return;
    }
    const uint32_t na = s_nact;
    for (uint32_t i = tid; i < s_T; i += kThreads) sm.tab[i] = 0;
    for (uint32_t i = tid; i < s_K; i += kThreads) sm.ccnt[i] = 0;
    // range + model per sub-array (a warp each)
    for (uint32_t a = warp; a < na; a += kThreads / 32) {
      Active& ac = sm.act[a];
      uint64_t mn = ~0ull, mx = 0ull;
      for (uint32_t q = lane; q < ac.n; q += 32) {
        const uint64_t v = ord_of(sm.A[ac.o + q], kt);
        mn = min(mn, v);
        mx = max(mx, v);
        sm.sid[ac.o + q] = (uint16_t)a;
      }
#pragma unroll
      for (int d = 16; d; d >>= 1) {
        mn = min(mn, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d));
        mx = max(mx, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d));
      }
      if (lane == 0) {
        ac.state = sample_state(ac.seed, ac.depth, ac.start, ac.n);
        if (mn == mx) {
          ac.ok = 0;  // one distinct value: sorted
        } else if (make_bin_model(kt, bits_of_ord(mn, kt), bits_of_ord(mx, kt), ac.beta, &ac.bm)) {
          ac.ok = 0;  // degenerate range: Standard-Sort
          const uint32_t i = atomicAdd(&s_nsort, 1u);
          if (i < geo.max_sorts) sm.sorts[i] = SortItem{(uint16_t)ac.o, (uint16_t)ac.n};
          else s_overflow = 1;
        } else {
          ac.ok = 1;
        }
      }
    }
    __syncthreads();
    // training: a thread per sample
    for (uint32_t q = tid; q < s_S; q += kThreads) {
      uint32_t a = 0, b = na;
      while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (sm.act[m].sbase <= q) a = m;
        else b = m;
      }
      const Active& ac = sm.act[a];
      if (!ac.ok) continue;
      const uint32_t idx = (uint32_t)sample_index(ac.state, q - ac.sbase, ac.n);
      const uint64_t x = sm.A[ac.o + idx];
      bool amb;
      uint32_t bn = bin_fast(ac.bm, x, amb);
      if (amb) bn = bin_exact_of(ac.bm, x);
      atomicAdd(&sm.tab[ac.tbase + bn], 1u);
    }
    __syncthreads();
    // b_k and the bucket table (a warp per sub-array)
    for (uint32_t a = warp; a < na; a += kThreads / 32) {
      const Active& ac = sm.act[a];
      if (!ac.ok) continue;
      uint32_t carry = 0;
      for (uint32_t k0 = 0; k0 <= ac.beta; k0 += 32) {
        const uint32_t k = k0 + lane;
        const uint32_t v = k <= ac.beta ? sm.tab[ac.tbase + k] : 0u;
        const uint32_t inc = wscan(v) + carry;
        if (k <= ac.beta) sm.tab[ac.tbase + k] = bucket_of_count(inc, ac.alpha, ac.gamma);
        carry = __shfl_sync(~0u, inc, 31);
      }
    }
    __syncthreads();
    // inference: the bucket of every key (a thread per key)
    for (uint32_t p0 = tid; p0 < cap; p0 += kThreads * 4) {
      uint32_t a[4], bn[4], amb = 0;
      uint64_t x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t p = p0 + u * kThreads;
        a[u] = p < cap ? sm.sid[p] : 0xFFFFu;
        if (a[u] != 0xFFFFu && !sm.act[a[u]].ok) a[u] = 0xFFFFu;
        x[u] = a[u] != 0xFFFFu ? sm.A[p] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bool am = false;
        bn[u] = a[u] != 0xFFFFu ? bin_fast(sm.act[a[u]].bm, x[u], am) : 0u;
        amb |= (uint32_t)am << u;
      }
      if (amb) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if ((amb >> u) & 1u) bn[u] = bin_exact_of(sm.act[a[u]].bm, x[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (a[u] == 0xFFFFu) continue;
        const Active& ac = sm.act[a[u]];
        const uint32_t j = sm.tab[ac.tbase + bn[u]];
        sm.J[p0 + u * kThreads] = (uint16_t)j;
        atomicAdd(&sm.ccnt[ac.cbase + j], 1u);
      }
    }
    __syncthreads();
    // bucket starts (a warp per sub-array)
    for (uint32_t a = warp; a < na; a += kThreads / 32) {
      const Active& ac = sm.act[a];
      if (!ac.ok) continue;
      uint32_t carry = 0;
      for (uint32_t k0 = 0; k0 <= ac.gamma; k0 += 32) {
        const uint32_t k = k0 + lane;
        const uint32_t v = k <= ac.gamma ? sm.ccnt[ac.cbase + k] : 0u;
        const uint32_t inc = wscan(v) + carry;
        if (k <= ac.gamma) {
          sm.cstart[ac.cbase + k] = inc - v;
          sm.cpos[ac.cbase + k] = inc - v;
        }
        carry = __shfl_sync(~0u, inc, 31);
      }
    }
    __syncthreads();
    // Append in input order: stable scatter A -> B (a warp per sub-array);
    // every other owned position is copied as it is
    for (uint32_t a = warp; a < na; a += kThreads / 32) {
      const Active& ac = sm.act[a];
      if (!ac.ok) continue;
      for (uint32_t b0 = 0; b0 < ac.n; b0 += 32) {
        const uint32_t i = b0 + lane;
        const bool v = i < ac.n;
        const uint32_t jj = v ? sm.J[ac.o + i] : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(~0u, jj);
        const int leader = __ffs(peers) - 1;
        uint32_t prior = 0;
        if (v && (int)lane == leader) {
          prior = sm.cpos[ac.cbase + jj];
          sm.cpos[ac.cbase + jj] = prior + __popc(peers);
        }
        prior = __shfl_sync(~0u, prior, leader);
        if (v) {
          const uint32_t pos = ac.o + prior + __popc(peers & lm);
          sm.B[pos] = sm.A[ac.o + i];
          if (PAIRS) sm.Bv[pos] = sm.Av[ac.o + i];
        }
      }
    }
    for (uint32_t p = tid; p < cap; p += kThreads) {
      const uint32_t a = sm.sid[p];
      if (sm.own[p] && (a == 0xFFFFu || !sm.act[a].ok)) {
        sm.B[p] = sm.A[p];
        if (PAIRS) sm.Bv[p] = sm.Av[p];
      }
    }
    __syncthreads();
    {
      uint64_t* t = sm.A;
      sm.A = sm.B;
      sm.B = t;
      uint32_t* tv = sm.Av;
      sm.Av = sm.Bv;
      sm.Bv = tv;
    }
    // Alg. 1's decision for every new bucket (a thread per bucket)
    for (uint32_t c = tid; c < s_K; c += kThreads) {
      uint32_t a = 0, b = na;
      while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (sm.act[m].cbase <= c) a = m;
        else b = m;
      }
      const Active& ac = sm.act[a];
      if (!ac.ok) continue;
      const uint32_t ck = sm.ccnt[c];
      if (ck <= 1) continue;
      const uint32_t ok = ac.o + sm.cstart[c];
      const bool std = ck >= ac.delta || ck < P.tau;
      if (std && ck <= kTinySort) {
        thread_sort<PAIRS>(sm.A, sm.Av, ok, ck, kt);
      } else if (std) {
        const uint32_t i = atomicAdd(&s_nsort, 1u);
        if (i < geo.max_sorts) sm.sorts[i] = SortItem{(uint16_t)ok, (uint16_t)ck};
        else s_overflow = 1;
      } else {
        const uint32_t i = atomicAdd(&s_nlearn, 1u);
        if (i < geo.max_learn) {
          LearnItem it;
          it.o = (uint16_t)ok;
          it.n = (uint16_t)ck;
          it.depth = (uint16_t)(ac.depth + 1);
          it.pad = 0;
          it.start = ac.start + (ok - ac.o);
          it.seed = ac.seed;
          sm.learn[i] = it;
        } else {
          s_overflow = 1;
        }
      }
    }
    for (uint32_t a = warp; a < na; a += kThreads / 32) {
      const Active& ac = sm.act[a];
      for (uint32_t q = lane; q < ac.n; q += 32) sm.sid[ac.o + q] = 0xFFFFu;
    }
    __syncthreads();
    if (s_overflow) {
      if (tid == 0) atomicOr(status, STATUS_INTERNAL);
      return;
    }
  }
  // ---- Standard-Sorts of more than kTinySort keys (a warp each)
  {
    const uint32_t ns = min(s_nsort, geo.max_sorts);
    for (uint32_t i = warp; i < ns; i += kThreads / 32) {
      const SortItem it = sm.sorts[i];
      if (it.n <= kTinySort) {
        if (lane == 0) thread_sort<PAIRS>(sm.A, sm.Av, it.o, it.n, kt);
      } else {
        warp_sort<PAIRS>(sm.A, sm.B, sm.Av, sm.Bv, it.o, it.n, kt);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (uint32_t p = tid; p < cap; p += kThreads) {
    if (sm.own[p]) {
      out[lo + p] = sm.A[p];
      if (PAIRS) out_v[lo + p] = sm.Av[p];
    }
  }
}

// ---------------------------------------------------------------------------
Geometry chunk_geometry(uint32_t window, uint32_t leaf_cap, const Policy& P) {
  Geometry g;
  g.cap = window + leaf_cap;
  // tables / buckets of one round: bounded by the budgets, rounds repeat
  g.tmax = min(g.cap / 2 + 256, 2048u);
  g.kmax = min(g.cap / 2 + 256, 2048u);
  const uint32_t tau = (uint32_t)(P.tau < 16 ? 16 : P.tau);
  g.max_learn = g.cap / tau + 8;
  g.max_sorts = g.cap / (kTinySort + 1) + 8;
  return g;
}

size_t chunk_smem_bytes(uint32_t window, uint32_t leaf_cap, const Policy& P, bool pairs) {
  return smem_bytes(chunk_geometry(window, leaf_cap, P), pairs);
}

cudaError_t launch_chunk(const LaunchCfg& c, const BRec* br, uint32_t nb, uint64_t wbase,
                         uint64_t span, uint32_t window, uint32_t leaf_cap, const uint64_t* X,
                         const uint32_t* Xv, uint64_t* out, uint32_t* out_v, Policy P,
                         const uint16_t* ptab, uint32_t* first_scratch) {
  if (!nb || !span) return cudaSuccess;
  const Geometry g = chunk_geometry(window, leaf_cap, P);
  const uint32_t H = window;
  const uint32_t grid = (uint32_t)((span + H - 1) / H);
  const size_t sm = smem_bytes(g, c.pairs);
  k_chunk_first<<<(grid + 1 + 255) / 256, 256, 0, c.stream>>>(br, nb, wbase, H, grid,
                                                               first_scratch);
  count_launch(c);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  if (c.pairs) {
    if ((e = cudaFuncSetAttribute(k_chunk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    k_chunk<true><<<grid, kThreads, sm, c.stream>>>(br, first_scratch, wbase, H, g, X, Xv, out,
                                                    out_v, c.kt, P, ptab, c.status);
  } else {
    if ((e = cudaFuncSetAttribute(k_chunk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    k_chunk<false><<<grid, kThreads, sm, c.stream>>>(br, first_scratch, wbase, H, g, X, Xv, out,
                                                     out_v, c.kt, P, ptab, c.status);
  }
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace pcf

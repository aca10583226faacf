// pcf_onchip.cu -- buckets finished on chip: a warp, or a CTA, per bucket.
//
// Every bucket of a global level that fits on chip is one call of
// Learned-Sort (Algorithm 1 of Sato & Matsui, TMLR 2025, with the PCF model
// of Sec. 3.3, or the spline model of App. A.5).  Buckets of at most 256
// keys (and every bucket of a key-value sort) go to a warp, which stages its
// keys in the warp's slice of shared memory (as order-preserving integers)
// and runs the recursion there with warp-synchronous code -- no block
// barriers, so the 30-40 warps of an SM overlap each other's latencies.
// Larger buckets of keys-only sorts go to a CTA of 64-512 threads (one slice
// per CTA, up to 8192 keys; k_onchip_cta).  The steps:
//   - Learned-Sort step: range (warp reduction), the model (lane 0; the
//     binary64 division runs in one lane), alpha samples with replacement
//     counted per bin (Sec. 3.3), b_k by a warp scan and the bucket table
//     floor(b_k gamma / alpha), the bucket of every key, the bucket sizes and
//     starts, and the Append into buckets (stable for key-value sorts);
//   - Alg. 1's decision for every new bucket: Standard-Sort when |c| >= delta
//     or |c| < tau, else a further Learned-Sort step (pushed on a per-warp
//     stack of pending calls);
//   - Standard-Sort: a new bucket of at most 32 keys by ranking each of its
//     keys among the bucket's; a whole call by ranking (at most 32 keys), a
//     bitonic network across the warp's registers (keys only, at most 64) or
//     a merge sort (larger, or key-value: stable).
// The leaf records are first listed by size class; the warps (or CTAs) of a
// launch take the buckets of one class in turn (the class's slice size
// bounds the keys of a bucket; classes (0, 256], (256, 512], ... up to
// leaf_cap).  The CDF model and the range policy are template parameters.
#include "pcf_internal.h"

namespace pcf {

namespace onchip {

constexpr uint32_t kWarps = 4;   // independent warps per CTA
constexpr uint32_t kRank = 32;     // key-value Standard-Sorts up to this size rank each key
constexpr uint32_t kRankKeys = 32; // ... keys-only ones (a bitonic network up to 64 above)

struct Item {  // a pending call on [o, o + n) of the warp's buffers
  uint16_t o, n;
  uint16_t depth, std;  // std: 1 = Standard-Sort, 0 = Learned-Sort
  uint64_t start;       // offset inside the caller's array (keys the samples)
};

// Layout of one warp's slice.
struct Slice {
  uint64_t* A;   // [capw] keys (total-order integers); calls finish here
  uint64_t* B;   // [capw] scatter target / merge scratch
  uint32_t* Av;  // [capw] values (key-value sorts)
  uint32_t* Bv;
  BinModel* bm;  // the current call's model (written by lane 0)
  Item* stk;     // [smax] pending calls
  uint32_t* tab; // [tmax] bin counts -> bucket table
  uint32_t* cnt; // [kmax] bucket sizes
  uint32_t* cur; // [kmax] bucket starts, then ends
  uint16_t* J;   // [capw] bucket of each source position
  uint16_t* Bj;  // [capw] bucket of each target position
};

__host__ __device__ inline size_t slice_bytes(const OnchipGeo& g, bool pairs) {
  size_t b = (size_t)g.capw * 16 + (pairs ? (size_t)g.capw * 8 : 0);
  b += (sizeof(BinModel) + 15) & ~(size_t)15;
  b += (size_t)g.smax * sizeof(Item);
  b += (size_t)g.tmax * 4 + (size_t)g.kmax * 8 + (size_t)g.capw * 4;
  return (b + 15) & ~(size_t)15;
}

__device__ inline Slice carve(uint8_t* p, const OnchipGeo& g, bool pairs) {
  Slice s;
  s.A = (uint64_t*)p;
  p += (size_t)g.capw * 8;
  s.B = (uint64_t*)p;
  p += (size_t)g.capw * 8;
  s.Av = s.Bv = nullptr;
  if (pairs) {
    s.Av = (uint32_t*)p;
    p += (size_t)g.capw * 4;
    s.Bv = (uint32_t*)p;
    p += (size_t)g.capw * 4;
  }
  s.bm = (BinModel*)p;
  p += (sizeof(BinModel) + 15) & ~(size_t)15;
  s.stk = (Item*)p;
  p += (size_t)g.smax * sizeof(Item);
  s.tab = (uint32_t*)p;
  p += (size_t)g.tmax * 4;
  s.cnt = (uint32_t*)p;
  p += (size_t)g.kmax * 4;
  s.cur = (uint32_t*)p;
  p += (size_t)g.kmax * 4;
  s.J = (uint16_t*)p;
  p += (size_t)g.capw * 2;
  s.Bj = (uint16_t*)p;
  return s;
}

__device__ __forceinline__ uint32_t lanemask_lt_() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t wscan(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(~0u, v, d);
    if (lane >= (uint32_t)d) v += u;
  }
  return v;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
  return (uint64_t)__shfl_sync(~0u, (unsigned long long)v, src);
}

// ---------------------------------------------------------------------------
// Standard-Sorts (R7: any sort; the output is the unique sorted order)
// ---------------------------------------------------------------------------

// Rank of key v at position p among positions [s, e) of K: the keys that
// are smaller, or equal and earlier (equal keys keep their order).
__device__ __forceinline__ uint32_t rank_in(const uint64_t* K, uint32_t s, uint32_t e, uint32_t p,
                                            uint64_t v) {
  uint32_t r = 0;
  for (uint32_t t = s; t < e; ++t) {
    const uint64_t u = K[t];
    r += (u < v || (u == v && t < p)) ? 1u : 0u;
  }
  return r;
}

// The same rank for keys whose offsets from a common base m differ only in
// their low 32 bits (keys of one part of a split whose shift is at most
// 32): the low words of the offsets decide.  vl = low word of v - m.
__device__ __forceinline__ uint32_t rank_in_lo32(const uint64_t* K, uint32_t s, uint32_t e,
                                                 uint32_t p, uint32_t vl, uint32_t ml) {
  const uint32_t* K32 = reinterpret_cast<const uint32_t*>(K);
  uint32_t r = 0;
  for (uint32_t t = s; t < e; ++t) {
    const uint32_t ul = K32[2 * t] - ml;
    r += (ul < vl || (ul == vl && t < p)) ? 1u : 0u;
  }
  return r;
}

// [o, o + c) of A ranked into B, then copied back; c <= kRank * 32.  Ties are
// broken by position, so equal keys keep their order (stable).
template <bool PAIRS>
__device__ void rank_sort(const Slice& w, uint32_t o, uint32_t c, uint32_t lane) {
  for (uint32_t p0 = 0; p0 < c; p0 += 32) {
    const uint32_t p = p0 + lane;
    if (p < c) {
      const uint64_t v = w.A[o + p];
      const uint32_t r = rank_in(w.A + o, 0, c, p, v);
      w.B[o + r] = v;
      if (PAIRS) w.Bv[o + r] = w.Av[o + p];
    }
  }
  __syncwarp();
  for (uint32_t p = lane; p < c; p += 32) {
    w.A[o + p] = w.B[o + p];
    if (PAIRS) w.Av[o + p] = w.Bv[o + p];
  }
  __syncwarp();
}

// Bitonic network over 32 E slots (keys only): element i = lane * E + e;
// the padding (all ones) sorts last and is not written back.  The stage
// loops run at run time (a fully unrolled network overflows the
// instruction cache once several kernels' warps interleave).
template <int E>
__device__ __forceinline__ void bitonic_intra(uint64_t (&v)[E], uint32_t lane, uint32_t k,
                                              uint32_t j) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int f = e ^ (int)j;
    if (f > e) {
      const bool up = ((lane * E + e) & k) == 0;
      const uint64_t a = v[e], b = v[f];
      const bool sw = up ? (a > b) : (a < b);
      v[e] = sw ? b : a;
      v[f] = sw ? a : b;
    }
  }
}

template <int E>
__device__ void bitonic_sort(uint64_t* A, uint32_t o, uint32_t c, uint32_t lane) {
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    v[e] = i < c ? A[o + i] : ~0ull;
  }
  constexpr uint32_t P = 32u * E;
#pragma unroll 1
  for (uint32_t k = 2; k <= P; k <<= 1) {
#pragma unroll 1
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= (uint32_t)E) {
        const uint32_t lj = j / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t i = lane * E + e;
          const uint64_t other = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)v[e], lj);
          const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
          v[e] = keep_min ? (other < v[e] ? other : v[e]) : (other > v[e] ? other : v[e]);
        }
      } else if (j == 1) {
        bitonic_intra<E>(v, lane, k, 1);
      } else if (j == 2) {
        if (E > 2) bitonic_intra<E>(v, lane, k, 2);
      } else {
        if (E > 4) bitonic_intra<E>(v, lane, k, 4);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = lane * E + e;
    if (i < c) A[o + i] = v[e];
  }
  __syncwarp();
}

// merge-path split of the first k outputs of merge(L, R) (ties: left first)
__device__ __forceinline__ uint32_t mpath(const uint64_t* L, uint32_t nL, const uint64_t* R,
                                          uint32_t nR, uint32_t k) {
  uint32_t lo = k > nR ? k - nR : 0u, hi = min(k, nL);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (L[mid] <= R[k - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// stable merge sort of A[o, o + c) by the warp (B as scratch): runs of
// ceil(c/32) keys by insertion in one lane each, then merge rounds
template <bool PAIRS>
__device__ void merge_sort(const Slice& w, uint32_t o, uint32_t c, uint32_t lane) {
  uint64_t* A = w.A;
  uint64_t* B = w.B;
  uint32_t* Av = w.Av;
  uint32_t* Bv = w.Bv;
  const uint32_t r = (c + 31) / 32;
  {
    const uint32_t a = min(c, lane * r), b = min(c, a + r);
    for (uint32_t i = a + 1; i < b; ++i) {
      const uint64_t key = A[o + i];
      const uint32_t val = PAIRS ? Av[o + i] : 0u;
      uint32_t j = i;
      while (j > a && A[o + j - 1] > key) {
        A[o + j] = A[o + j - 1];
        if (PAIRS) Av[o + j] = Av[o + j - 1];
        --j;
      }
      A[o + j] = key;
      if (PAIRS) Av[o + j] = val;
    }
  }
  __syncwarp();
  for (uint32_t wd = r; wd < c; wd *= 2) {
    const uint32_t a0 = min(c, lane * r), b0 = min(c, a0 + r);
    uint32_t a = a0;
    while (a < b0) {
      const uint32_t p0 = (a / (2 * wd)) * (2 * wd);
      const uint32_t pe = min(c, p0 + 2 * wd);
      const uint32_t nL = min(wd, c - p0), nR = pe - p0 - nL;
      const uint64_t* L = A + o + p0;
      const uint64_t* R = L + nL;
      const uint32_t e = min(b0, pe);
      const uint32_t k = a - p0;
      uint32_t i = mpath(L, nL, R, nR, k), j = k - i;
      for (uint32_t q = a; q < e; ++q) {
        const bool takeL = j >= nR || (i < nL && L[i] <= R[j]);
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

template <bool PAIRS>
__device__ void std_sort(const Slice& w, uint32_t o, uint32_t c, uint32_t lane) {
  if (c <= 1) return;
  if (c <= (PAIRS ? kRank : kRankKeys)) {
    rank_sort<PAIRS>(w, o, c, lane);
  } else if (PAIRS || c > 64) {
    merge_sort<PAIRS>(w, o, c, lane);
  } else {
    bitonic_sort<2>(w.A, o, c, lane);
  }
}

// ---------------------------------------------------------------------------
// One Learned-Sort step on [o, o + n) (Algorithm 1, Sec. 3.3).  New buckets
// are finished here (ranked) when small, else pushed.  Returns false when
// the per-warp stack would overflow.
// ---------------------------------------------------------------------------
template <bool PAIRS, bool SPLINE, bool SRANGE>
__device__ bool learn_step(const Slice& w, const OnchipGeo& geo, const Item it, uint64_t seed,
                           uint32_t kt, const Policy& P, const uint16_t* __restrict__ ptab,
                           uint32_t& top, uint32_t lane, bool root, uint64_t rmn, uint64_t rmx,
                           DecisionCounters* dc) {
  const uint32_t o = it.o, n = it.n;
  constexpr bool spline = SPLINE;
  // alpha..delta and the sample stream: with the array's range taken after
  // the range pass (fewer registers live across it)
  ushort4 q = make_ushort4(0, 0, 0, 0);
  uint64_t state = 0;
  if constexpr (SRANGE) {
    q = __ldg(reinterpret_cast<const ushort4*>(ptab) + n);
    state = sample_state(seed, it.depth, it.start, n);
  }
  // the samples' range (R14) when the policy asks for it and it is usable
  bool have_model = false;
  if constexpr (SRANGE) {
    const uint32_t alpha = q.x, beta = q.y, gamma = q.z;
    uint64_t smn = ~0ull, smx = 0ull;
    for (uint32_t s = lane; s < alpha; s += 32) {
      const uint64_t v = w.A[o + (uint32_t)sample_index(state, s, n)];
      smn = v < smn ? v : smn;
      smx = v > smx ? v : smx;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)smn, d);
      const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)smx, d);
      smn = a < smn ? a : smn;
      smx = b > smx ? b : smx;
    }
    int ok = 0;
    if (lane == 0 && smn != smx &&
        !make_bin_model(kt, bits_of_ord(smn, kt), bits_of_ord(smx, kt), beta, w.bm)) {
      w.bm->clamp = 1;
      if (spline) spline_set(w.bm, alpha, gamma);
      ok = 1;
    }
    have_model = __shfl_sync(~0u, ok, 0) != 0;
  }
  if (!have_model) {
    // range (a root call's per-lane range was taken while its keys loaded)
    uint64_t mn = rmn, mx = rmx;
    if (!root) {
      mn = ~0ull;
      mx = 0ull;
      for (uint32_t i = lane; i < n; i += 32) {
        const uint64_t v = w.A[o + i];
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
      }
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d);
      const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d);
      mn = a < mn ? a : mn;
      mx = b > mx ? b : mx;
    }
    if (mn == mx) return true;  // one value: sorted
    if constexpr (!SRANGE) {
      q = __ldg(reinterpret_cast<const ushort4*>(ptab) + n);
      state = sample_state(seed, it.depth, it.start, n);
    }
    int degen = 0;
    if (lane == 0) {
      degen = make_bin_model(kt, bits_of_ord(mn, kt), bits_of_ord(mx, kt), q.y, w.bm);
      if (!degen && spline) spline_set(w.bm, q.x, q.z);
    }
    degen = __shfl_sync(~0u, degen, 0);
    if (degen) {  // R5: a degenerate range goes to Standard-Sort
      std_sort<PAIRS>(w, o, n, lane);
      return true;
    }
  }
  const uint32_t alpha = q.x, beta = q.y, gamma = q.z, delta = q.w;
  if (lane == 0) atomicAdd(&dc->bucketings, 1ull);
  for (uint32_t k = lane; k <= beta; k += 32) w.tab[k] = 0;
  for (uint32_t k = lane; k <= gamma; k += 32) w.cnt[k] = 0;
  __syncwarp();
  const BinModel bm = *w.bm;
  // training: alpha samples with replacement, counted per bin
  for (uint32_t s = lane; s < alpha; s += 32) {
    const uint32_t idx = (uint32_t)sample_index(state, s, n);
    const uint64_t x = bits_of_ord(w.A[o + idx], kt);
    bool amb;
    uint32_t bn = bin_fast(bm, x, amb);
    if (amb) bn = bin_exact_of(bm, x);
    atomicAdd(&w.tab[bn], 1u);
  }
  __syncwarp();
  // b_k and the bucket table
  {
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 <= beta; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t v = k <= beta ? w.tab[k] : 0u;
      const uint32_t inc = wscan(v, lane) + carry;
      if (k <= beta) w.tab[k] = spline ? inc : bucket_of_count(inc, alpha, gamma);
      carry = __shfl_sync(~0u, inc, 31);
    }
  }
  __syncwarp();
  // the bucket of every key, and the bucket sizes
  if (spline) {
    for (uint32_t i = lane; i < n; i += 32) {
      double f;
      const uint32_t k = spline_bin(bm, bits_of_ord(w.A[o + i], kt), &f);
      const uint32_t j = spline_bucket(bm, f, k ? w.tab[k - 1] : 0u, w.tab[k]);
      w.J[i] = (uint16_t)j;
      atomicAdd(&w.cnt[j], 1u);
    }
  }
  for (uint32_t i0 = 0; i0 < (spline ? 0u : n); i0 += 64) {
    uint64_t x[2];
    uint32_t bn[2], amb = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t i = i0 + u * 32 + lane;
      x[u] = i < n ? bits_of_ord(w.A[o + i], kt) : bm.lo_bits;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      bool a;
      bn[u] = SRANGE ? bin_fast_clamped(bm, x[u], a) : bin_fast(bm, x[u], a);
      amb |= (uint32_t)a << u;
    }
    if (amb) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if ((amb >> u) & 1u) bn[u] = bin_exact_of(bm, x[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t i = i0 + u * 32 + lane;
      if (i < n) {
        const uint32_t j = w.tab[bn[u]];
        w.J[i] = (uint16_t)j;
        atomicAdd(&w.cnt[j], 1u);
      }
    }
  }
  __syncwarp();
  // bucket starts
  {
    uint32_t carry = 0;
    for (uint32_t k0 = 0; k0 <= gamma; k0 += 32) {
      const uint32_t k = k0 + lane;
      const uint32_t v = k <= gamma ? w.cnt[k] : 0u;
      const uint32_t inc = wscan(v, lane) + carry;
      if (k <= gamma) w.cur[k] = inc - v;
      carry = __shfl_sync(~0u, inc, 31);
    }
  }
  __syncwarp();
  // Append: A -> B by bucket (in input order for key-value sorts)
  if (!PAIRS) {
    for (uint32_t i = lane; i < n; i += 32) {
      const uint32_t j = w.J[i];
      const uint32_t pos = atomicAdd(&w.cur[j], 1u);
      w.B[o + pos] = w.A[o + i];
      w.Bj[pos] = (uint16_t)j;
    }
  } else {
    const uint32_t lm = lanemask_lt_();
    for (uint32_t i0 = 0; i0 < n; i0 += 32) {
      const uint32_t i = i0 + lane;
      const bool v = i < n;
      const uint32_t j = v ? w.J[i] : 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(~0u, j);
      const int leader = __ffs(peers) - 1;
      uint32_t prior = 0;
      if (v && (int)lane == leader) prior = atomicAdd(&w.cur[j], (uint32_t)__popc(peers));
      prior = __shfl_sync(~0u, prior, leader);
      if (v) {
        const uint32_t pos = prior + __popc(peers & lm);
        w.B[o + pos] = w.A[o + i];
        w.Bv[o + pos] = w.Av[o + i];
        w.Bj[pos] = (uint16_t)j;
      }
    }
  }
  __syncwarp();
  // Alg. 1 for every new bucket c (cur[j] now holds its end): ranked here
  // when a Standard-Sort of at most kRank keys, else copied back and pushed
  const uint32_t lm = lanemask_lt_();
  bool ok = true;
  for (uint32_t p0 = 0; p0 < n; p0 += 32) {
    const uint32_t p = p0 + lane;
    bool push = false;
    Item ch;
    if (p < n) {
      const uint32_t j = w.Bj[p];
      const uint32_t c = w.cnt[j], e = w.cur[j], s = e - c;
      const uint64_t v = w.B[o + p];
      const bool stdc = c >= delta || c < P.tau;
      if (p == s && c >= delta) {
        atomicAdd(&dc->guard_buckets, 1ull);
        atomicAdd(&dc->guard_keys, (unsigned long long)c);
      }
      if (c == 1) {
        w.A[o + p] = v;
        if (PAIRS) w.Av[o + p] = w.Bv[o + p];
      } else if (stdc && c <= kRank) {
        const uint32_t r = rank_in(w.B + o, s, e, p, v);
        w.A[o + s + r] = v;
        if (PAIRS) w.Av[o + s + r] = w.Bv[o + p];
      } else {
        w.A[o + p] = v;
        if (PAIRS) w.Av[o + p] = w.Bv[o + p];
        if (p == s) {
          push = true;
          ch.o = (uint16_t)(o + s);
          ch.n = (uint16_t)c;
          ch.depth = (uint16_t)(it.depth + 1);
          ch.std = stdc ? 1 : 0;
          ch.start = it.start + s;
        }
      }
    }
    const uint32_t bal = __ballot_sync(~0u, push);
    if (push) {
      const uint32_t slot = top + __popc(bal & lm);
      if (slot < geo.smax) w.stk[slot] = ch;
    }
    top += __popc(bal);
    if (top > geo.smax) ok = false;
  }
  __syncwarp();
  return ok;
}

// The leaf records of each size class, compacted (a thread per record):
// class 0 holds the buckets of at most 256 keys, class c > 0 those of
// (128 << c, 256 << c] keys.
__device__ __forceinline__ uint32_t size_class(uint32_t n) {
  return n <= 256 ? 0u : (uint32_t)(32 - __clz((int)(n - 1))) - 8u;
}

// recs: entries are (offset, size) pairs (uint2) in the block-local sort's
// classes instead of record indices in the Learned-Sort kernels' classes
__global__ void k_leaf_lists(const BRec* __restrict__ br, uint32_t nb, uint32_t ncls,
                             uint32_t* lists, uint32_t* counts, const uint32_t* gate, int recs) {
  if (pcf_aborted(gate)) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t cls = kMaxLeafClasses;
  BRec r;
  r.off = r.n = 0;
  if (i < nb) {
    r = br[i];
    if ((r.kind & BK_LEAF) && r.n > 0)
      cls = min(recs ? leaf_size_class(r.n) : size_class(r.n), ncls - 1);
  }
#pragma unroll
  for (uint32_t k = 0; k < kMaxLeafClasses; ++k) {
    const uint32_t bal = __ballot_sync(~0u, cls == k);
    if (!bal) continue;
    const int leader = __ffs(bal) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(&counts[k], (uint32_t)__popc(bal));
    base = __shfl_sync(~0u, base, leader);
    if (cls == k) {
      const size_t at = (size_t)k * nb + base + __popc(bal & lanemask_lt_());
      if (recs) reinterpret_cast<uint2*>(lists)[at] = make_uint2(r.off, r.n);
      else lists[at] = i;
    }
  }
}

template <bool PAIRS, bool SPLINE, bool SRANGE>
__global__ void __launch_bounds__(kWarps * 32, 8) k_onchip(const BRec* __restrict__ br,
                                                           const uint32_t* __restrict__ list,
                                                           const uint32_t* __restrict__ count,
                                                           OnchipGeo geo,
                                                           const uint64_t* __restrict__ X,
                                                           const uint32_t* __restrict__ Xv,
                                                           uint64_t* out, uint32_t* out_v,
                                                           uint32_t kt, Policy P,
                                                           const uint16_t* __restrict__ ptab,
                                                           uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const Slice w = carve(smem_raw + (size_t)wib * slice_bytes(geo, PAIRS), geo, PAIRS);
  const uint32_t gw = blockIdx.x * kWarps + wib, nw = gridDim.x * kWarps;
  const uint32_t nitems = *count;
  for (uint32_t li = gw; li < nitems; li += nw) {
    const BRec r = br[list[li]];
    const uint32_t off = r.off, n = r.n;
    uint64_t rmn = ~0ull, rmx = 0ull;
    for (uint32_t i = lane; i < n; i += 32) {
      const uint64_t v = ord_of(__ldg(X + off + i), kt);
      w.A[i] = v;
      rmn = v < rmn ? v : rmn;
      rmx = v > rmx ? v : rmx;
      if (PAIRS) w.Av[i] = __ldg(Xv + off + i);
    }
    __syncwarp();
    bool ok = true;
    if (r.kind & BK_STD) {
      std_sort<PAIRS>(w, 0, n, lane);
    } else {
      uint32_t top = 1;
      if (lane == 0) {
        Item it;
        it.o = 0;
        it.n = (uint16_t)n;
        it.depth = (uint16_t)r.depth;
        it.std = 0;
        it.start = r.start;
        w.stk[0] = it;
      }
      __syncwarp();
      bool root = true;
      while (top > 0 && ok) {
        --top;
        const Item it = w.stk[top];
        __syncwarp();
        if (it.std) std_sort<PAIRS>(w, it.o, it.n, lane);
        else
          ok = learn_step<PAIRS, SPLINE, SRANGE>(w, geo, it, r.seed, kt, P, ptab, top, lane, root,
                                                 rmn, rmx, pcf_counters(status));
        root = false;
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(status, STATUS_INTERNAL);
      return;
    }
    for (uint32_t i = lane; i < n; i += 32) {
      if (!PCF_IN_KEYS(off + i, status)) break;
      out[off + i] = bits_of_ord(w.A[i], kt);
      if (PAIRS) out_v[off + i] = w.Av[i];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Buckets of more than 256 keys (keys only): the NT threads of a CTA share
// one bucket.  Up to 1024 keys two warps (so that a bucket's critical path
// is about half as long, and twice as many buckets as four-warp CTAs would
// allow stay in flight per SM); above, NT grows with the bucket (128 threads
// up to 2048 keys, 256 up to 4096, 512 up to 8192), so that a bucket up to
// 8192 keys -- 128 KB of keys plus the scatter target, one CTA per SM -- is
// still finished in shared memory instead of by another global level.  The
// same steps as learn_step; Standard-Sorts of whole calls run in warp 0.
// ---------------------------------------------------------------------------
template <uint32_t NT>
struct CtaShared {
  uint64_t mn[NT / 32], mx[NT / 32];
  uint64_t smn[NT / 32], smx[NT / 32];  // the samples' range (R14)
  uint32_t wsum[NT / 32];
  uint32_t top, flag, ovf, sok;
};

// Scan of src[0..m) into dst by the CTA (each thread a contiguous run, one
// barrier; src may be dst).  EXCL: exclusive sums.  Otherwise the inclusive
// sums b_k, turned into the bucket table floor(b_k gamma / alpha) unless raw
// (the spline model reads b_k itself).
template <uint32_t NT, bool EXCL>
__device__ __forceinline__ void cta_scan(const uint32_t* src, uint32_t* dst, uint32_t m,
                                         uint32_t alpha, uint32_t gamma, CtaShared<NT>& sh,
                                         bool raw = false) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t r = (m + NT - 1) / NT;
  const uint32_t a = min(m, tid * r), b = min(m, a + r);
  uint32_t sum = 0;
  for (uint32_t k = a; k < b; ++k) sum += src[k];
  const uint32_t inc = wscan(sum, lane);
  if (lane == 31) sh.wsum[wid] = inc;
  __syncthreads();
  uint32_t run = inc - sum;
#pragma unroll
  for (uint32_t k = 0; k < NT / 32; ++k) run += k < wid ? sh.wsum[k] : 0u;
  for (uint32_t k = a; k < b; ++k) {
    const uint32_t v = src[k];
    if (EXCL) {
      dst[k] = run;
      run += v;
    } else {
      run += v;
      dst[k] = raw ? run : bucket_of_count(run, alpha, gamma);
    }
  }
}

// Samples per thread drawn before the model is ready (alpha <= this many
// times the CTA size for every call of its size class under the default
// policy; any further samples are drawn after it).
constexpr uint32_t kSampRegs = 3;

// root: the range was reduced into sh.mn / sh.mx while the keys were loaded
template <uint32_t NT, bool SPLINE, bool SRANGE>
__device__ void learn_step_cta(const Slice& w, const OnchipGeo& geo, const Item it, uint64_t seed,
                               uint32_t kt, const Policy& P, const uint16_t* __restrict__ ptab,
                               CtaShared<NT>& sh, bool root, DecisionCounters* dc) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t o = it.o, n = it.n;
  const ushort4 q = __ldg(reinterpret_cast<const ushort4*>(ptab) + n);
  const uint32_t alpha = q.x, beta = q.y, gamma = q.z, delta = q.w;
  constexpr bool spline = SPLINE;
  // the sample positions and keys do not depend on the model: with the
  // array's range they are drawn while thread 0 builds it, with the
  // samples' range first
  const uint64_t state = sample_state(seed, it.depth, it.start, n);
  uint64_t sx[kSampRegs];
  bool drawn = false;
  auto draw = [&]() {
#pragma unroll
    for (uint32_t u = 0; u < kSampRegs; ++u) {
      const uint32_t s = tid + u * NT;
      sx[u] = s < alpha ? bits_of_ord(w.A[o + (uint32_t)sample_index(state, s, n)], kt) : 0ull;
    }
    drawn = true;
  };
  // the samples' range (R14) when the policy asks for it and it is usable
  bool have_model = false;
  if constexpr (SRANGE) {
    draw();
    uint64_t smn = ~0ull, smx = 0ull;
#pragma unroll
    for (uint32_t u = 0; u < kSampRegs; ++u) {
      if (tid + u * NT < alpha) {
        const uint64_t v = ord_of(sx[u], kt);
        smn = v < smn ? v : smn;
        smx = v > smx ? v : smx;
      }
    }
    for (uint32_t s = tid + kSampRegs * NT; s < alpha; s += NT) {
      const uint64_t v = w.A[o + (uint32_t)sample_index(state, s, n)];
      smn = v < smn ? v : smn;
      smx = v > smx ? v : smx;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)smn, d);
      const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)smx, d);
      smn = a < smn ? a : smn;
      smx = b > smx ? b : smx;
    }
    if (lane == 0) {
      sh.smn[wid] = smn;
      sh.smx[wid] = smx;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (uint32_t k = 0; k < NT / 32; ++k) {
        smn = sh.smn[k] < smn ? sh.smn[k] : smn;
        smx = sh.smx[k] > smx ? sh.smx[k] : smx;
      }
      sh.sok = smn != smx &&
               !make_bin_model(kt, bits_of_ord(smn, kt), bits_of_ord(smx, kt), beta, w.bm);
      if (sh.sok) {
        w.bm->clamp = 1;
        if (spline) spline_set(w.bm, alpha, gamma);
      }
    }
    __syncthreads();
    have_model = sh.sok != 0;
  }
  if (!have_model) {
    uint64_t mn = ~0ull, mx = 0ull;
    if (!root) {
      for (uint32_t i = tid; i < n; i += NT) {
        const uint64_t v = w.A[o + i];
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
      }
#pragma unroll
      for (int d = 16; d; d >>= 1) {
        const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d);
        const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
      }
      if (lane == 0) {
        sh.mn[wid] = mn;
        sh.mx[wid] = mx;
      }
      __syncthreads();
    }
#pragma unroll
    for (uint32_t k = 0; k < NT / 32; ++k) {
      mn = sh.mn[k] < mn ? sh.mn[k] : mn;
      mx = sh.mx[k] > mx ? sh.mx[k] : mx;
    }
    if (mn == mx) return;  // one value: sorted
    if (tid == 0) {
      sh.flag = (uint32_t)make_bin_model(kt, bits_of_ord(mn, kt), bits_of_ord(mx, kt), beta, w.bm);
      if (!sh.flag && spline) spline_set(w.bm, alpha, gamma);
    }
  } else if (tid == 0) {
    sh.flag = 0;
  }
  for (uint32_t k = tid; k <= beta; k += NT) w.tab[k] = 0;
  for (uint32_t k = tid; k <= gamma; k += NT) w.cnt[k] = 0;
  if (!drawn) draw();
  __syncthreads();
  if (sh.flag) {  // R5: a degenerate range goes to Standard-Sort
    if (wid == 0) std_sort<false>(w, o, n, lane);
    return;
  }
  if (tid == 0) atomicAdd(&dc->bucketings, 1ull);
  const BinModel bm = *w.bm;
#pragma unroll
  for (uint32_t u = 0; u < kSampRegs; ++u) {
    if (tid + u * NT < alpha) {
      bool amb;
      uint32_t bn = bin_fast(bm, sx[u], amb);
      if (amb) bn = bin_exact_of(bm, sx[u]);
      atomicAdd(&w.tab[bn], 1u);
    }
  }
  for (uint32_t s = tid + kSampRegs * NT; s < alpha; s += NT) {
    const uint64_t x = bits_of_ord(w.A[o + (uint32_t)sample_index(state, s, n)], kt);
    bool amb;
    uint32_t bn = bin_fast(bm, x, amb);
    if (amb) bn = bin_exact_of(bm, x);
    atomicAdd(&w.tab[bn], 1u);
  }
  __syncthreads();
  cta_scan<NT, false>(w.tab, w.tab, beta + 1, alpha, gamma, sh, spline);
  __syncthreads();
  if (spline) {
    for (uint32_t i = tid; i < n; i += NT) {
      double f;
      const uint32_t k = spline_bin(bm, bits_of_ord(w.A[o + i], kt), &f);
      const uint32_t j = spline_bucket(bm, f, k ? w.tab[k - 1] : 0u, w.tab[k]);
      w.J[i] = (uint16_t)j;
      atomicAdd(&w.cnt[j], 1u);
    }
  }
  for (uint32_t i0 = 0; i0 < (spline ? 0u : n); i0 += 2 * NT) {
    uint64_t x[2];
    uint32_t bn[2], amb = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t i = i0 + u * NT + tid;
      x[u] = i < n ? bits_of_ord(w.A[o + i], kt) : bm.lo_bits;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      bool a;
      bn[u] = SRANGE ? bin_fast_clamped(bm, x[u], a) : bin_fast(bm, x[u], a);
      amb |= (uint32_t)a << u;
    }
    if (amb) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if ((amb >> u) & 1u) bn[u] = bin_exact_of(bm, x[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t i = i0 + u * NT + tid;
      if (i < n) {
        const uint32_t j = w.tab[bn[u]];
        w.J[i] = (uint16_t)j;
        atomicAdd(&w.cnt[j], 1u);
      }
    }
  }
  __syncthreads();
  // bucket starts into cur (cnt keeps the sizes)
  cta_scan<NT, true>(w.cnt, w.cur, gamma + 1, 0, 0, sh);
  __syncthreads();
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t j = w.J[i];
    const uint32_t pos = atomicAdd(&w.cur[j], 1u);
    w.B[o + pos] = w.A[o + i];
    w.Bj[pos] = (uint16_t)j;
  }
  __syncthreads();
  for (uint32_t p = tid; p < n; p += NT) {
    const uint32_t j = w.Bj[p];
    const uint32_t c = w.cnt[j], e = w.cur[j], s = e - c;
    const uint64_t v = w.B[o + p];
    const bool stdc = c >= delta || c < P.tau;
    if (p == s && c >= delta) {
      atomicAdd(&dc->guard_buckets, 1ull);
      atomicAdd(&dc->guard_keys, (unsigned long long)c);
    }
    if (c == 1) {
      w.A[o + p] = v;
    } else if (stdc && c <= kRank) {
      w.A[o + s + rank_in(w.B + o, s, e, p, v)] = v;
    } else {
      w.A[o + p] = v;
      if (p == s) {
        Item ch;
        ch.o = (uint16_t)(o + s);
        ch.n = (uint16_t)c;
        ch.depth = (uint16_t)(it.depth + 1);
        ch.std = stdc ? 1 : 0;
        ch.start = it.start + s;
        const uint32_t slot = atomicAdd(&sh.top, 1u);
        if (slot < geo.smax) w.stk[slot] = ch;
        else sh.ovf = 1;
      }
    }
  }
}

template <uint32_t NT, bool SPLINE, bool SRANGE>
__global__ void __launch_bounds__(NT, NT <= 64 ? 16 : 512 / NT) k_onchip_cta(const BRec* __restrict__ br,
                                                        const uint32_t* __restrict__ list,
                                                        const uint32_t* __restrict__ count,
                                                        OnchipGeo geo,
                                                        const uint64_t* __restrict__ X,
                                                        uint64_t* out, uint32_t kt, Policy P,
                                                        const uint16_t* __restrict__ ptab,
                                                        uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ CtaShared<NT> sh;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const Slice w = carve(smem_raw, geo, false);
  const uint32_t nitems = *count;
  for (uint32_t li = blockIdx.x; li < nitems; li += gridDim.x) {
    const BRec r = br[list[li]];
    const uint32_t off = r.off, n = r.n;
    {
      uint64_t mn = ~0ull, mx = 0ull;
      for (uint32_t i = tid; i < n; i += NT) {
        const uint64_t v = ord_of(__ldg(X + off + i), kt);
        w.A[i] = v;
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
      }
#pragma unroll
      for (int d = 16; d; d >>= 1) {
        const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d);
        const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
      }
      if (lane == 0) {
        sh.mn[wid] = mn;
        sh.mx[wid] = mx;
      }
    }
    if (tid == 0) {
      Item it;
      it.o = 0;
      it.n = (uint16_t)n;
      it.depth = (uint16_t)r.depth;
      it.std = (r.kind & BK_STD) ? 1 : 0;
      it.start = r.start;
      w.stk[0] = it;
      sh.top = 1;
      sh.ovf = 0;
    }
    __syncthreads();
    while (true) {
      const uint32_t top = sh.top;
      if (top == 0 || sh.ovf) break;
      const Item it = w.stk[top - 1];
      __syncthreads();
      if (tid == 0) sh.top = top - 1;  // seen by the pushes after the next barrier
      if (it.std) {
        __syncthreads();
        if (wid == 0) std_sort<false>(w, it.o, it.n, lane);
      } else {
        learn_step_cta<NT, SPLINE, SRANGE>(w, geo, it, r.seed, kt, P, ptab, sh,
                                           top == 1 && it.o == 0 && it.n == n,
                                           pcf_counters(status));
      }
      __syncthreads();
    }
    if (sh.ovf) {
      if (tid == 0) atomicOr(status, STATUS_INTERNAL);
      return;
    }
    for (uint32_t i = tid; i < n; i += NT) {
      if (!PCF_IN_KEYS(off + i, status)) break;
      out[off + i] = bits_of_ord(w.A[i], kt);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Block-local Standard-Sort of a whole leaf bucket (keys only).  Alg. 1
// leaves the choice of Standard-Sort open (Sec. 3.1: any sort), and a bucket
// that fits in shared memory is small: it is sorted here in one piece
// instead of by further Learned-Sort steps.  The output is the unique
// ascending order either way.
//
// One CTA of NT threads per bucket of at most NT * KPT keys:
//   1. the bucket's keys were staged in shared memory (P) by one bulk copy
//      (the tensor memory accelerator's 1-D form, completing on an mbarrier)
//      while the CTA sorted the previous bucket; each thread takes KPT of
//      them into registers as order-preserving integers, and the CTA reduces
//      min and max (32-bit warp reductions of the high, then the low words),
//      then stages the next bucket;
//   2. one equal-width split of [min, max] into M = 2^ceil(log2 n) parts:
//      part(v) = (v - min) >> shift, shift chosen so that parts < M (an MSD
//      radix digit of the key's offset from the minimum; no model, no
//      samples, no division); counts by shared atomics, an exclusive scan
//      (each thread a contiguous chunk of parts) that leaves every part's
//      (start, count) packed in one word, and every key written to its
//      part's range of B with that word beside it (W);
//   3. every key's final position: its part's start plus its rank among the
//      part's keys (smaller, or equal and earlier in B), written straight to
//      the output (consecutive threads write nearly consecutive positions).
//      Parts of more than kLeafRank keys (skewed or duplicate-heavy buckets)
//      are listed and sorted afterwards by one warp each (leaf_big_part).
// The key type is a template parameter, so the order conversions of u64
// keys vanish.
// ---------------------------------------------------------------------------
constexpr uint32_t kLeafRank = 16;
template <uint32_t NT>
struct LeafShared {
  uint64_t mn[NT / 32], mx[NT / 32];
  uint32_t wsum[NT / 32];
  uint32_t n_big;
};

// B [cap] u64 | P [cap + 2] u64 (the next bucket, staged; key i at slot
// i + (offset & 1), so that the bulk copy lands on a 16-byte boundary) |
// W [cap] u32 (each slot's part word) | H [cap << ovs] u32 (part counts, then
// (start, count) words) | big list | mbarrier.  W and H together are the
// merge scratch of the large parts.
__host__ __device__ inline size_t leaf_sort_smem(uint32_t cap, uint32_t ovs) {
  const size_t big = (((size_t)cap / kLeafRank + 1) * 4 + 15) & ~(size_t)15;
  return (size_t)cap * 20 + 16 + ((size_t)cap << ovs) * 4 + big + 16;
}

// 64-bit warp min / max from two 32-bit reductions (high words, then the
// low words of the lanes holding the extreme high word)
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
  const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
  const uint32_t h = __reduce_min_sync(~0u, hi);
  const uint32_t l = __reduce_min_sync(~0u, hi == h ? lo : 0xFFFFFFFFu);
  return ((uint64_t)h << 32) | l;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
  const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
  const uint32_t h = __reduce_max_sync(~0u, hi);
  const uint32_t l = __reduce_max_sync(~0u, hi == h ? lo : 0u);
  return ((uint64_t)h << 32) | l;
}

// Stages bucket (off, n) into P: one thread issues the bulk copy of the
// 16-byte-aligned middle and arrives on the barrier; the keys at either
// ragged end (at most one each) are loaded by threads 32 and 33 (or 0 and 1
// in a one-warp CTA), which runs beside the thread issuing the copy.
// q: 1 when X itself sits 8 bytes past a 16-byte boundary (keys at index
// i with i + q even start a 16-byte word)
template <uint32_t NT>
__device__ __forceinline__ void leaf_stage(uint64_t* P, uint64_t* bar, const uint64_t* X,
                                           uint32_t q, uint32_t off, uint32_t n, uint32_t tid) {
  const uint32_t sh = (off + q) & 1u;
  const uint32_t a0 = min(off + n, ((off + q + 1u) & ~1u) - q);
  const uint32_t a1 = max(a0, ((off + n + q) & ~1u) - q);
  if (tid == 0) {
    const uint32_t bytes = (a1 - a0) * 8u;
    mbar_arrive_tx(bar, bytes);
    if (bytes) bulk_g2s(P + (a0 - off + sh), X + a0, bytes, bar);
  }
  constexpr uint32_t kHead = NT > 32 ? 32u : 0u;
  if (tid == kHead && a0 > off) P[sh] = __ldg(X + off);
  if (tid == kHead + 1 && a1 < off + n && a1 >= a0) P[a1 - off + sh] = __ldg(X + a1);
}

// one part of more than kLeafRank keys, B[s, s + c): sorted by one warp
// (scratch at the same offsets of S) and written to out[off + s, ...)
__device__ __noinline__ void leaf_big_part(uint64_t* B, uint64_t* S, uint32_t s, uint32_t c,
                                           uint64_t* out, uint32_t off, uint32_t kt,
                                           uint32_t lane, uint32_t* status) {
  (void)status;
  uint64_t mn = ~0ull, mx = 0ull;
  for (uint32_t i = lane; i < c; i += 32) {
    const uint64_t v = B[s + i];
    mn = v < mn ? v : mn;
    mx = v > mx ? v : mx;
  }
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    const uint64_t a = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d);
    const uint64_t b = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (mn != mx) {  // (one value: already in order)
    Slice w;
    w.A = B;
    w.B = S;
    w.Av = w.Bv = nullptr;
    std_sort<false>(w, s, c, lane);
  }
  for (uint32_t i = lane; i < c; i += 32)
    if (PCF_IN_KEYS(off + s + i, status)) out[off + s + i] = bits_of_ord(B[s + i], kt);
  __syncwarp();
}

template <uint32_t NT, uint32_t KPT, uint32_t OVS, uint32_t KT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : 1024 / NT)
    k_leaf_sort(const uint2* __restrict__ list, const uint32_t* __restrict__ count,
                const uint64_t* __restrict__ X, uint64_t* out, uint32_t* status) {
  constexpr uint32_t CAP = NT * KPT, NW = NT / 32;
  static_assert(NT >= 32 && NT <= 1024 && (NT & (NT - 1)) == 0, "NT a power of two, 32..1024");
  static_assert(KPT >= 1 && (KPT & (KPT - 1)) == 0 && CAP <= 8192, "KPT a power of two");
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ LeafShared<NT> sh;
  uint64_t* B = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* Pf = B + CAP;
  uint32_t* Wp = reinterpret_cast<uint32_t*>(Pf + CAP + 2);
  uint32_t* H = Wp + CAP;
  uint32_t* big = H + (CAP << OVS);
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      smem_raw + (((size_t)CAP * 20 + 16 + ((size_t)CAP << OVS) * 4 +
                   (((size_t)CAP / kLeafRank + 1) * 4 + 15)) & ~(size_t)15));
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t nitems = *count;
  const uint32_t G = gridDim.x;
  uint32_t li = blockIdx.x;
  if (li >= nitems) return;
  if (tid == 0) mbar_init(bar);
  __syncthreads();
  uint2 rec = list[li];
  uint2 rec1 = li + G < nitems ? list[li + G] : make_uint2(0u, 0u);
  const uint32_t q = (uint32_t)(reinterpret_cast<uintptr_t>(X) >> 3) & 1u;
  leaf_stage<NT>(Pf, bar, X, q, rec.x, rec.y <= CAP ? rec.y : 0u, tid);
  uint32_t phase = 0;
  for (; li < nitems; li += G) {
    // a record larger than this class holds is an internal error (flagged,
    // nothing written for it)
    if (rec.y > CAP && tid == 0) atomicOr(status, STATUS_INTERNAL);
    const uint32_t off = rec.x, n = rec.y <= CAP ? rec.y : 0u, shf = (off + q) & 1u;
    const uint2 rec2 = li + 2 * G < nitems ? list[li + 2 * G] : make_uint2(0u, 0u);
    const uint32_t m = (n > 1 ? 32u - __clz(n - 1) : 0u) + OVS;  // M = 2^m >= n parts
    const uint32_t M = 1u << m;
    // the staged bucket: every thread waits on the barrier (bounded); a wait
    // that gives up flags the sort and leaves (nothing further is staged)
    const bool ok = mbar_wait(bar, phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(status, STATUS_TIMEOUT);
      // give the copy one more bounded wait before the shared memory is left
      mbar_wait(bar, phase);
      return;
    }
    phase ^= 1u;
    uint64_t k[KPT];
    uint64_t mn = ~0ull, mx = 0ull;
#pragma unroll
    for (uint32_t j = 0; j < KPT; ++j) {
      const uint32_t i = tid + j * NT;
      k[j] = ord_of(Pf[(i < n ? i : 0u) + shf], KT);
      if (i < n) {
        mn = k[j] < mn ? k[j] : mn;
        mx = k[j] > mx ? k[j] : mx;
      }
    }
    if (M >= 4) {
      for (uint32_t d = tid * 4; d < M; d += NT * 4)
        *reinterpret_cast<uint4*>(H + d) = make_uint4(0u, 0u, 0u, 0u);
    } else if (tid < M) {
      H[tid] = 0u;
    }
    if (tid == 0) sh.n_big = 0;
    mn = warp_min_u64(mn);
    mx = warp_max_u64(mx);
    if (lane == 0) {
      sh.mn[wid] = mn;
      sh.mx[wid] = mx;
    }
    __syncthreads();  // P is free again; H zeroed
    // stage the next bucket while this one is sorted
    if (li + G < nitems) leaf_stage<NT>(Pf, bar, X, q, rec1.x, rec1.y <= CAP ? rec1.y : 0u, tid);
#pragma unroll
    for (uint32_t w = 0; w < NW; ++w) {
      mn = sh.mn[w] < mn ? sh.mn[w] : mn;
      mx = sh.mx[w] > mx ? sh.mx[w] : mx;
    }
    if (mn >= mx) {  // one value (or one key, or none): already sorted
#pragma unroll
      for (uint32_t j = 0; j < KPT; ++j) {
        const uint32_t i = tid + j * NT;
        if (i < n && PCF_IN_KEYS(off + i, status)) out[off + i] = bits_of_ord(k[j], KT);
      }
    } else {
      const uint32_t nb = 64u - (uint32_t)__clzll((long long)(mx - mn));
      const uint32_t sft = nb > m ? nb - m : 0u;
      uint32_t hx[KPT], rk[KPT];
#pragma unroll
      for (uint32_t j = 0; j < KPT; ++j) {
        const uint32_t i = tid + j * NT;
        hx[j] = (uint32_t)((k[j] - mn) >> sft);
        rk[j] = i < n ? atomicAdd(&H[hx[j]], 1u) : 0u;
      }
      __syncthreads();
      // exclusive scan: thread t owns parts [t r, t r + r), r = M / NT (or
      // one part for t < M when M < NT); each entry becomes
      // start | count << 16 (both at most 8192)
      {
        const uint32_t r = M >= NT ? M / NT : 1u;
        const bool own = tid * r < M;
        uint32_t v[(KPT > 4 ? KPT : 4) << OVS];
        uint32_t sum = 0;
        if (r >= 4) {
#pragma unroll
          for (uint32_t c = 0; c < (KPT << OVS); c += 4) {
            if (c < r) {
              const uint4 h = *reinterpret_cast<const uint4*>(H + tid * r + c);
              v[c] = h.x;
              v[c + 1] = h.y;
              v[c + 2] = h.z;
              v[c + 3] = h.w;
              sum += h.x + h.y + h.z + h.w;
            }
          }
        } else {
#pragma unroll
          for (uint32_t c = 0; c < 4; ++c) {
            v[c] = (own && c < r) ? H[tid * r + c] : 0u;
            sum += v[c];
          }
        }
        uint32_t inc = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(~0u, inc, d);
          if (lane >= (uint32_t)d) inc += u;
        }
        if (lane == 31) sh.wsum[wid] = inc;
        __syncthreads();
        uint32_t run = inc - sum;
#pragma unroll
        for (uint32_t w = 0; w < NW; ++w) run += w < wid ? sh.wsum[w] : 0u;
        if (r >= 4) {
#pragma unroll
          for (uint32_t c = 0; c < (KPT << OVS); c += 4) {
            if (c < r) {
              uint4 h;
              h.x = run | (v[c] << 16);
              run += v[c];
              h.y = run | (v[c + 1] << 16);
              run += v[c + 1];
              h.z = run | (v[c + 2] << 16);
              run += v[c + 2];
              h.w = run | (v[c + 3] << 16);
              run += v[c + 3];
              *reinterpret_cast<uint4*>(H + tid * r + c) = h;
            }
          }
        } else if (own) {
#pragma unroll
          for (uint32_t c = 0; c < 4; ++c) {
            if (c < r) {
              H[tid * r + c] = run | (v[c] << 16);
              run += v[c];
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (uint32_t j = 0; j < KPT; ++j) {
        const uint32_t i = tid + j * NT;
        if (i < n) {
          const uint32_t sc = H[hx[j]];
          const uint32_t p = (sc & 0xFFFFu) + rk[j];
          if (PCF_IN(p, n, status)) {
            B[p] = k[j];
            Wp[p] = sc;
          }
        }
      }
      __syncthreads();
      const uint32_t ml = (uint32_t)mn;
#pragma unroll 2
      for (uint32_t j = 0; j < KPT; ++j) {
        const uint32_t p = tid + j * NT;
        if (p >= n) break;
        const uint64_t v = B[p];
        const uint32_t sc = Wp[p];
        const uint32_t s = sc & 0xFFFFu, c = sc >> 16;
        uint32_t pos = p;
        if (c > kLeafRank) {
          if (p == s) big[atomicAdd(&sh.n_big, 1u)] = sc;
          continue;
        }
        if (c > 1) {
          // rank among the part's keys (smaller, or equal and earlier)
          uint32_t r = 0;
          if (sft <= 32) {
            const uint32_t* K32 = reinterpret_cast<const uint32_t*>(B);
            const uint32_t vl = (uint32_t)v - ml;
#pragma unroll 1
            for (uint32_t t = s; t < s + c; ++t) {
              const uint32_t ul = K32[2 * t] - ml;
              r += (ul < vl || (ul == vl && t < p)) ? 1u : 0u;
            }
          } else {
#pragma unroll 1
            for (uint32_t t = s; t < s + c; ++t) {
              const uint64_t u = B[t];
              r += (u < v || (u == v && t < p)) ? 1u : 0u;
            }
          }
          pos = s + r;
        }
        if (PCF_IN_KEYS(off + pos, status)) out[off + pos] = bits_of_ord(v, KT);
      }
      __syncthreads();
      const uint32_t nbig = sh.n_big;
      for (uint32_t b = wid; b < nbig; b += NW)
        leaf_big_part(B, reinterpret_cast<uint64_t*>(Wp), big[b] & 0xFFFFu, big[b] >> 16, out,
                      off, KT, lane, status);
    }
    __syncthreads();  // B, H, W and the list are reused by the next bucket
    rec = rec1;
    rec1 = rec2;
  }
}

// ---------------------------------------------------------------------------
// Mid-size (sub)arrays: one Learned-Sort call (Alg. 1, PCF model of Sec.
// 3.3) on a bucket of leaf_cap < n <= kMidCap keys, by one CTA, in place of
// a further global level.  The CTA takes the bucket's range (x_min, x_max),
// builds the model, draws its alpha samples (R2, keyed like every other
// call) and the table T[k] = floor(b_k gamma / alpha), computes every key's
// bucket, counts the buckets and decides them as Alg. 1 does.  When every
// new bucket finishes on chip (at most leaf_cap keys: the block-local leaf
// sort, which also serves as the Standard-Sort of a failure-guard bucket)
// it appends each key to its bucket in Y (the level's other key buffer,
// free at these offsets) and
// lists the new buckets for the block-local leaf sort, runs of 32 small
// ones as one record as k_buckets does.  Otherwise it leaves the bucket to
// the next global level (its next-level flag set, nothing written), so
// every decision stays Alg. 1's.
// ---------------------------------------------------------------------------
constexpr uint32_t kMidThreads = 512;

struct MidShared {
  BinModel bm;
  uint64_t mn[kMidThreads / 32], mx[kMidThreads / 32];
  uint32_t wsum[kMidThreads / 32];
  uint32_t flag;
};

// T [kMidTab] u32 (bin counts, then the bucket table) | C [kMidTab] u32
// (bucket sizes, then starts, then cursors) | J [kMidCap] u16 (the bucket of
// every key)
__host__ __device__ constexpr size_t mid_smem_bytes() {
  return (size_t)kMidTab * 4 * 2 + (size_t)kMidCap * 2;
}

// exclusive (EXCL) or inclusive scan of a[0..m) in place by the CTA; each
// thread a contiguous run; returns the total
template <bool EXCL>
__device__ __forceinline__ uint32_t mid_scan(uint32_t* a, uint32_t m, MidShared& sh) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t per = (m + kMidThreads - 1) / kMidThreads;
  const uint32_t i0 = min(m, tid * per), i1 = min(m, i0 + per);
  uint32_t sum = 0;
  for (uint32_t i = i0; i < i1; ++i) sum += a[i];
  uint32_t inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(~0u, inc, d);
    if (lane >= (uint32_t)d) inc += u;
  }
  if (lane == 31) sh.wsum[wid] = inc;
  __syncthreads();
  uint32_t run = inc - sum, tot = 0;
#pragma unroll
  for (uint32_t w = 0; w < kMidThreads / 32; ++w) {
    const uint32_t x = sh.wsum[w];
    run += w < wid ? x : 0u;
    tot += x;
  }
  for (uint32_t i = i0; i < i1; ++i) {
    const uint32_t v = a[i];
    run += v;
    a[i] = EXCL ? run - v : run;
  }
  __syncthreads();
  return tot;
}

template <uint32_t KT>
__global__ void __launch_bounds__(kMidThreads, 2)
    k_mid(const uint32_t* __restrict__ mid_list, const uint32_t* __restrict__ mid_count,
          const BRec* __restrict__ brec, const uint64_t* __restrict__ X, uint64_t* Y,
          uint64_t* out, uint32_t* next_flag, uint2* lists, MidLists ml,
          uint32_t* list_counts, uint32_t leaf_classes, uint32_t leaf_cap, Policy P,
          LevelOut* lo, uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ MidShared sh;
  uint32_t* T = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* C = T + kMidTab;
  uint16_t* J = reinterpret_cast<uint16_t*>(C + kMidTab);
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr uint32_t NW = kMidThreads / 32;
  const uint32_t nitems = *mid_count;
  for (uint32_t li = blockIdx.x; li < nitems; li += gridDim.x) {
    const uint32_t B = mid_list[li];
    const BRec r = brec[B];
    const uint32_t n = r.n, off = r.off;
    const Params pr = params_of(P, n);
    // range
    uint64_t mn = ~0ull, mx = 0ull;
#pragma unroll 4
    for (uint32_t i = tid; i < n; i += kMidThreads) {
      const uint64_t v = ord_of(__ldg(X + off + i), KT);
      mn = v < mn ? v : mn;
      mx = v > mx ? v : mx;
    }
    mn = warp_min_u64(mn);
    mx = warp_max_u64(mx);
    if (lane == 0) {
      sh.mn[wid] = mn;
      sh.mx[wid] = mx;
    }
    __syncthreads();
    if (tid == 0) {
      for (uint32_t w = 1; w < NW; ++w) {
        mn = sh.mn[w] < mn ? sh.mn[w] : mn;
        mx = sh.mx[w] > mx ? sh.mx[w] : mx;
      }
      // one value: already sorted (1); a degenerate range or tables larger
      // than this kernel holds: the next global level decides (2)
      uint32_t f = 0;
      if (n > kMidCap || pr.beta + 1 > kMidTab || pr.gamma + 1 > kMidTab) f = 2;
      else if (mn == mx) f = 1;
      else if (make_bin_model(KT, bits_of_ord(mn, KT), bits_of_ord(mx, KT), pr.beta, &sh.bm))
        f = 2;
      sh.flag = f;
    }
    for (uint32_t k = tid; k <= pr.beta && k < kMidTab; k += kMidThreads) T[k] = 0u;
    for (uint32_t k = tid; k <= pr.gamma && k < kMidTab; k += kMidThreads) C[k] = 0u;
    __syncthreads();
    const uint32_t f = sh.flag;
    if (f == 1) {
      for (uint32_t i = tid; i < n; i += kMidThreads)
        if (PCF_IN_KEYS(off + i, status)) out[off + i] = __ldg(X + off + i);
      __syncthreads();
      continue;
    }
    if (f == 2) {
      if (tid == 0) {
        next_flag[B] = 1u;
        atomicAdd(&lo->n_flag, 1u);
      }
      __syncthreads();
      continue;
    }
    // samples (R2) counted per bin, then b_k and the bucket table
    const BinModel& bm = sh.bm;
    {
      const uint64_t st = sample_state(r.seed, r.depth, r.start, n);
      for (uint32_t j = tid; j < pr.alpha; j += kMidThreads) {
        const uint64_t idx = sample_index(st, j, n);
        atomicAdd(&T[bin_of(bm, __ldg(X + off + idx))], 1u);
      }
    }
    __syncthreads();
    mid_scan<false>(T, pr.beta + 1, sh);
    for (uint32_t k = tid; k <= pr.beta; k += kMidThreads)
      T[k] = bucket_of_count(T[k], pr.alpha, pr.gamma);
    __syncthreads();
    // every key's bucket, and the bucket sizes: four keys per thread and
    // step, the fast bins first and the exact sequence only for the keys
    // they leave undecided (as k_hist1 does)
    for (uint32_t i0 = tid; i0 < n; i0 += 4 * kMidThreads) {
      uint64_t x[4];
      uint32_t bn[4], amb = 0;
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t i = i0 + u * kMidThreads;
        x[u] = i < n ? __ldg(X + off + i) : bm.lo_bits;
      }
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        bool a;
        bn[u] = bin_fast(bm, x[u], a);
        amb |= (uint32_t)a << u;
      }
      if (amb) {
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u)
          if ((amb >> u) & 1u) bn[u] = bin_exact_of(bm, x[u]);
      }
#pragma unroll
      for (uint32_t u = 0; u < 4; ++u) {
        const uint32_t i = i0 + u * kMidThreads;
        if (i < n) {
          const uint32_t j = T[bn[u]];
          J[i] = (uint16_t)j;
          atomicAdd(&C[j], 1u);
        }
      }
    }
    __syncthreads();
    // Alg. 1's decision for every bucket: all must finish on chip
    bool bad = false;
    for (uint32_t k = tid; k <= pr.gamma; k += kMidThreads) {
      const uint32_t c = C[k];
      bad |= c > leaf_cap || (c >= pr.delta && c > guard_leaf_max(leaf_cap, true));
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        next_flag[B] = 1u;
        atomicAdd(&lo->n_flag, 1u);
      }
      continue;
    }
    // decided here: the call's record (a bucketing, its failure-guard
    // buckets), the buckets' leaf records (runs of 32 small ones as one)
    {
      uint32_t gb = 0, gk = 0;
      for (uint32_t k = tid; k <= pr.gamma; k += kMidThreads) {
        const uint32_t c = C[k];
        if (c >= pr.delta && c > 0) {
          ++gb;
          gk += c;
        }
      }
      gb = __reduce_add_sync(~0u, gb);
      gk = __reduce_add_sync(~0u, gk);
      if (lane == 0 && gb) {
        atomicAdd(&pcf_counters(status)->guard_buckets, (unsigned long long)gb);
        atomicAdd(&pcf_counters(status)->guard_keys, (unsigned long long)gk);
      }
      if (tid == 0) {
        atomicAdd(&pcf_counters(status)->bucketings, 1ull);
        atomicAdd((unsigned long long*)&lo->mid_keys, (unsigned long long)n);
      }
    }
    // sizes -> starts (kept in T's place: the table is no longer needed)
    for (uint32_t k = tid; k <= pr.gamma; k += kMidThreads) T[k] = C[k];
    __syncthreads();
    mid_scan<true>(T, pr.gamma + 1, sh);
    // leaf records: warp w takes buckets [32 q, 32 q + 32) for q = w, w + NW, ...
    for (uint32_t b0 = wid * 32; b0 <= pr.gamma; b0 += NW * 32) {
      const uint32_t k = b0 + lane;
      const bool in = k <= pr.gamma;
      const uint32_t c = in ? C[k] : 0u, s = in ? T[k] : 0u;
      const uint32_t run_n = __reduce_add_sync(~0u, c);
      const bool run = __all_sync(~0u, !in || c <= kRunBucket) && run_n <= leaf_cap;
      const bool lane0 = lane == 0;
      const uint32_t ln = run ? run_n : c;
      const uint32_t ls = run ? __shfl_sync(~0u, s, 0) : s;
      const uint32_t cls = (run ? lane0 && run_n > 0 : c > 0)
                               ? min(leaf_size_class(ln), leaf_classes - 1)
                               : kMaxLeafClasses;
#pragma unroll
      for (uint32_t q = 0; q < kMaxLeafClasses; ++q) {
        const uint32_t bal = __ballot_sync(~0u, cls == q);
        if (!bal) continue;
        const int leader = __ffs(bal) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(&list_counts[q], (uint32_t)__popc(bal));
        base = __shfl_sync(~0u, base, leader);
        const uint32_t at = base + __popc(bal & ((1u << lane) - 1u));
        if (cls == q) {
          if (at < ml.cap[q]) lists[ml.base[q] + at] = make_uint2(off + ls, ln);
          else atomicOr(status, STATUS_INTERNAL);
        }
      }
    }
    // the keys appended to their buckets in Y (C as cursors from the starts)
    for (uint32_t k = tid; k <= pr.gamma; k += kMidThreads) C[k] = T[k];
    __syncthreads();
#pragma unroll 4
    for (uint32_t i = tid; i < n; i += kMidThreads) {
      const uint32_t p = atomicAdd(&C[J[i]], 1u);
      if (PCF_IN(p, n, status) && PCF_IN_KEYS(off + p, status)) Y[off + p] = __ldg(X + off + i);
    }
    __syncthreads();
  }
}

}  // namespace onchip

using namespace onchip;

OnchipGeo onchip_geometry(uint32_t capw, const Policy& P, bool pairs) {
  OnchipGeo g;
  g.capw = capw;
  // floor(n^(p/q)) does not decrease with n: the largest call bounds all
  const Params pr = params_of(P, capw);
  g.tmax = (max(2u, pr.beta + 1) + 3) & ~3u;
  g.kmax = (max(2u, pr.gamma + 1) + 3) & ~3u;
  g.smax = capw / 16 + 4;
  g.bytes = (uint32_t)slice_bytes(g, pairs);
  return g;
}

static int num_sms_of_current_device() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 148;
  }
  return cached[dev];
}

uint32_t leaf_sort_classes(uint32_t leaf_cap) {
  uint32_t k = 1;
  for (uint32_t capw = 64; capw < leaf_cap && k < kMaxLeafClasses; capw *= 2) ++k;
  return k;
}

uint32_t onchip_classes(uint32_t leaf_cap) {
  uint32_t k = 1;
  for (uint32_t capw = 256; capw < leaf_cap && k < kMaxClasses; capw *= 2) ++k;
  return k;
}

// one CTA of NT threads per bucket of the class whose slices are g.bytes
template <uint32_t NT, bool SPLINE, bool SRANGE>
static cudaError_t launch_cta_model(const LaunchCfg& c, const BRec* br, const uint32_t* list,
                                    const uint32_t* count, const OnchipGeo& g, const uint64_t* X,
                                    uint64_t* out, const Policy& P, const uint16_t* ptab) {
  constexpr uint32_t kMaxPerSm = NT <= 64 ? 16u : 512u / NT;
  const uint32_t per = max(1u, min(kMaxPerSm, (uint32_t)((227u * 1024u) / (g.bytes + 1024u))));
  cudaError_t e = allow_max_smem((const void*)k_onchip_cta<NT, SPLINE, SRANGE>);
  if (e) return e;
  k_onchip_cta<NT, SPLINE, SRANGE><<<(uint32_t)num_sms_of_current_device() * per, NT, g.bytes,
                                     c.stream>>>(br, list, count, g, X, out, c.kt, P, ptab,
                                                 c.status);
  return cudaGetLastError();
}

template <uint32_t NT>
static cudaError_t launch_cta_class(const LaunchCfg& c, const BRec* br, const uint32_t* list,
                                    const uint32_t* count, const OnchipGeo& g, const uint64_t* X,
                                    uint64_t* out, const Policy& P, const uint16_t* ptab) {
  const bool sr = P.range_mode == RANGE_SAMPLE;
  if (P.model == MODEL_SPLINE)
    return sr ? launch_cta_model<NT, true, true>(c, br, list, count, g, X, out, P, ptab)
              : launch_cta_model<NT, true, false>(c, br, list, count, g, X, out, P, ptab);
  return sr ? launch_cta_model<NT, false, true>(c, br, list, count, g, X, out, P, ptab)
            : launch_cta_model<NT, false, false>(c, br, list, count, g, X, out, P, ptab);
}

template <bool PAIRS, bool SPLINE, bool SRANGE>
static cudaError_t launch_warp_model(const LaunchCfg& c, const BRec* br, const uint32_t* list,
                                     const uint32_t* count, const OnchipGeo& g, const uint64_t* X,
                                     const uint32_t* Xv, uint64_t* out, uint32_t* out_v,
                                     const Policy& P, const uint16_t* ptab) {
  const size_t sm = (size_t)kWarps * g.bytes;
  const uint32_t per_sm = max(1u, min(8u, (uint32_t)((227u * 1024u) / (sm + 1024u))));
  const uint32_t grid = (uint32_t)num_sms_of_current_device() * per_sm;
  cudaError_t e = allow_max_smem((const void*)k_onchip<PAIRS, SPLINE, SRANGE>);
  if (e) return e;
  k_onchip<PAIRS, SPLINE, SRANGE><<<grid, kWarps * 32, sm, c.stream>>>(
      br, list, count, g, X, Xv, out, out_v, c.kt, P, ptab, c.status);
  return cudaGetLastError();
}

// the block-local sort of one size class: NT threads, KPT keys each, parts
// 2^(ceil(log2 n) + OVS)
template <uint32_t NT, uint32_t KPT, uint32_t OVS, uint32_t KT>
static cudaError_t launch_leaf_sort_kt(const LaunchCfg& c, const uint2* list,
                                       const uint32_t* count, const uint64_t* X, uint64_t* out) {
  const size_t smem = leaf_sort_smem(NT * KPT, OVS);
  cudaError_t e = allow_max_smem((const void*)k_leaf_sort<NT, KPT, OVS, KT>);
  if (e) return e;
  static int per_sm_cache[64] = {0};
  int dev = 0;
  if ((e = cudaGetDevice(&dev))) return e;
  int per_sm = dev >= 0 && dev < 64 ? per_sm_cache[dev] : 0;
  if (per_sm <= 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf_sort<NT, KPT, OVS, KT>,
                                                      (int)NT, smem);
    if (e) return e;
    per_sm = per_sm > 0 ? per_sm : 1;
    if (dev >= 0 && dev < 64) per_sm_cache[dev] = per_sm;
  }
  k_leaf_sort<NT, KPT, OVS, KT><<<(uint32_t)num_sms_of_current_device() * (uint32_t)per_sm, NT,
                                  smem, c.stream>>>(list, count, X, out, c.status);
  return cudaGetLastError();
}

template <uint32_t NT, uint32_t KPT, uint32_t OVS = 0u>
static cudaError_t launch_leaf_sort(const LaunchCfg& c, const uint2* list, const uint32_t* count,
                                    const uint64_t* X, uint64_t* out) {
  return c.kt == KEY_U64 ? launch_leaf_sort_kt<NT, KPT, OVS, KEY_U64>(c, list, count, X, out)
                         : launch_leaf_sort_kt<NT, KPT, OVS, KEY_F64>(c, list, count, X, out);
}

uint32_t onchip_cap(uint32_t leaf_cap, const Policy& P, bool pairs) {
  // key-value sorts: the warp kernel (four slices per block), up to 1024
  // keys; keys only: one slice per block above 256 keys
  uint32_t cap = pairs ? min(leaf_cap, 1024u) : leaf_cap;
  while (cap > 64) {
    const OnchipGeo g = onchip_geometry(cap, P, pairs);
    const size_t need = (pairs || cap <= 256) ? (size_t)kWarps * g.bytes : (size_t)g.bytes;
    if (need + 1024 <= 227u * 1024u) break;
    cap /= 2;
  }
  return cap;
}

template <uint32_t KT>
static cudaError_t launch_mid_kt(const LaunchCfg& c, const uint32_t* mid_list,
                                 const uint32_t* mid_count, const BRec* brec, const uint64_t* X,
                                 uint64_t* Y, uint64_t* out, uint32_t* next_flag, uint2* lists,
                                 const MidLists& ml, uint32_t* list_counts, uint32_t leaf_classes,
                                 uint32_t leaf_cap, const Policy& P, LevelOut* lo) {
  constexpr size_t smem = mid_smem_bytes();
  cudaError_t e = allow_max_smem((const void*)k_mid<KT>);
  if (e) return e;
  k_mid<KT><<<(uint32_t)num_sms_of_current_device() * 2u, kMidThreads, smem, c.stream>>>(
      mid_list, mid_count, brec, X, Y, out, next_flag, lists, ml, list_counts, leaf_classes,
      leaf_cap, P, lo, c.status);
  return cudaGetLastError();
}

cudaError_t launch_mid(const LaunchCfg& c, const uint32_t* mid_list, const uint32_t* mid_count,
                       const BRec* brec, const uint64_t* X, uint64_t* Y, uint64_t* out,
                       uint32_t* next_flag, uint2* lists, const MidLists& ml,
                       uint32_t* list_counts, uint32_t leaf_classes, uint32_t leaf_cap,
                       const Policy& P, LevelOut* lo) {
  cudaError_t e =
      c.kt == KEY_U64
          ? launch_mid_kt<KEY_U64>(c, mid_list, mid_count, brec, X, Y, out, next_flag, lists, ml,
                                   list_counts, leaf_classes, leaf_cap, P, lo)
          : launch_mid_kt<KEY_F64>(c, mid_list, mid_count, brec, X, Y, out, next_flag, lists, ml,
                                   list_counts, leaf_classes, leaf_cap, P, lo);
  count_launch(c);
  return e;
}

cudaError_t launch_onchip(const LaunchCfg& c, const BRec* br, uint32_t nb, uint32_t leaf_cap,
                          const uint64_t* X, const uint32_t* Xv, uint64_t* out, uint32_t* out_v,
                          Policy P, const uint16_t* ptab, uint32_t* lists, uint32_t* counts,
                          bool prelisted, const uint64_t* class_base,
                          const cudaStream_t* class_stream) {
  if (!nb) return cudaSuccess;
  // size classes (0, 256], (256, 512], (512, 1024], ... clipped to leaf_cap
  const bool recs = c.leaf_sort && !c.pairs;
  const uint32_t ncls = recs ? leaf_sort_classes(leaf_cap) : onchip_classes(leaf_cap);
  cudaError_t e = cudaSuccess;
  if (!(prelisted && recs)) {
    e = cudaMemsetAsync(counts, 0, 4 * kMaxLeafClasses, c.stream);
    if (e) return e;
    k_leaf_lists<<<(nb + 255) / 256, 256, 0, c.stream>>>(br, nb, ncls, lists, counts, c.status,
                                                          recs ? 1 : 0);
    count_launch(c);
    if ((e = cudaGetLastError())) return e;
  }
  if (recs) {
    // the whole bucket by the block-local Standard-Sort: a warp for up to
    // 256 keys (2, 4 or 8 per lane), then NT = capw / 8 threads
    for (uint32_t cls = 0, capw = 64; cls < ncls; ++cls, capw *= 2) {
      const uint2* rl = reinterpret_cast<const uint2*>(lists) +
                        (class_base ? class_base[cls] : (size_t)cls * nb);
      const uint32_t* cnt = counts + cls;
      LaunchCfg cc = c;
      if (class_stream) cc.stream = class_stream[cls];
      switch (capw) {
        case 64: e = launch_leaf_sort<32, 2>(cc, rl, cnt, X, out); break;
        case 128: e = launch_leaf_sort<32, 4>(cc, rl, cnt, X, out); break;
        case 256: e = launch_leaf_sort<32, 8>(cc, rl, cnt, X, out); break;
        case 512: e = launch_leaf_sort<64, 8>(cc, rl, cnt, X, out); break;
        case 1024: e = launch_leaf_sort<128, 8>(cc, rl, cnt, X, out); break;
        case 2048: e = launch_leaf_sort<256, 8>(cc, rl, cnt, X, out); break;
        case 4096: e = launch_leaf_sort<512, 8>(cc, rl, cnt, X, out); break;
        default: e = launch_leaf_sort<1024, 8>(cc, rl, cnt, X, out); break;
      }
      if (e) return e;
      count_launch(c);
    }
    return cudaSuccess;
  }
  uint32_t cls = 0;
  for (uint32_t capw = 256, lo = 0; lo < leaf_cap; capw *= 2, ++cls) {
    const uint32_t hi = min(capw, leaf_cap);
    const OnchipGeo g = onchip_geometry(hi, P, c.pairs);
    const uint32_t* list = lists + (size_t)cls * nb;
    if (cls > 0 && !c.pairs) {
      // a CTA per bucket (one slice per CTA), more threads for larger buckets
      if (hi <= 1024) e = launch_cta_class<64>(c, br, list, counts + cls, g, X, out, P, ptab);
      else if (hi <= 2048) e = launch_cta_class<128>(c, br, list, counts + cls, g, X, out, P, ptab);
      else if (hi <= 4096) e = launch_cta_class<256>(c, br, list, counts + cls, g, X, out, P, ptab);
      else e = launch_cta_class<512>(c, br, list, counts + cls, g, X, out, P, ptab);
      if (e) return e;
    } else {
      const uint32_t v = (c.pairs ? 4u : 0u) | (P.model == MODEL_SPLINE ? 2u : 0u) |
                         (P.range_mode == RANGE_SAMPLE ? 1u : 0u);
      const uint32_t* cnt = counts + cls;
      switch (v) {
        case 0: e = launch_warp_model<false, false, false>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 1: e = launch_warp_model<false, false, true>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 2: e = launch_warp_model<false, true, false>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 3: e = launch_warp_model<false, true, true>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 4: e = launch_warp_model<true, false, false>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 5: e = launch_warp_model<true, false, true>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        case 6: e = launch_warp_model<true, true, false>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
        default: e = launch_warp_model<true, true, true>(c, br, list, cnt, g, X, Xv, out, out_v, P, ptab); break;
      }
      if (e) return e;
    }
    count_launch(c);
    lo = hi;
  }
  return cudaSuccess;
}

}  // namespace pcf

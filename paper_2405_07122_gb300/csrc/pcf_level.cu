// pcf_level.cu -- the kernels of one global bucketing level of PCF Learned
// Sort (Sato & Matsui, TMLR 2025, Algorithm 1 with the PCF model of
// Sec. 3.3), for a batch of (sub)arrays ("segments"):
//
//   k_range     x_min, x_max of every segment (+ NaN check)          Sec. 3.3
//   k_sample_range  the same over the alpha samples (sample-range policy)
//   k_model     degenerate-range test and the bin function's constants
//   k_sample    draw alpha keys, count them per bin, and (last CTA of the
//               segment) accumulate b_k and the bucket table
//               T[k] = floor(b_k gamma / alpha)                        Sec. 3.3, Alg. 1
//   k_hist1     per-tile histogram of the high digit of the bucket id
//   k_scan      decoupled-lookback exclusive prefix sum (Merrill & Garland)
//   k_scatter1  stable scatter by the high digit ("Append" in input order)
//   k_groups / k_hist2 / k_scatter2   the same for the low digit, per group
//   k_buckets   the per-bucket decision of Alg. 1 (|c| >= delta -> standard
//               sort; small -> shared-memory kernel; else next level)
//   k_next_segs / k_cols_*   the next level's plan, built on the device
//   k_bucket_sizes / k_bucket_max   level-0 bucket sizes only (Sec. 4.2)
//   k_xfer      small host <-> device copies through pinned host memory
//
// The gamma + 1 buckets are produced by two stable scatters on the high and
// the low bits of the bucket id; two stable passes compose to the single
// (gamma+1)-way stable partition of Alg. 1.
#include "pcf_internal.h"

namespace pcf {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// first i in [0, n) with a[i] > v, for non-decreasing a
template <typename T>
__device__ __forceinline__ uint32_t upper_bound_dev(const T* a, uint32_t n, T v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t ld_nc(const uint64_t* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// k_range: min / max under the total order (x_min, x_max of Sec. 3.3)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_range(Seg* segs, uint32_t S, const uint32_t* range_base,
                                               const uint64_t* __restrict__ keys, uint32_t kt,
                                               int check_nan, uint32_t* status,
                                               uint32_t only_status) {
  if (pcf_aborted(status)) return;
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(range_base, S + 1, t) - 1;
  if (only_status != ~0u && segs[s].status != only_status) return;
  const uint64_t off = segs[s].off, n = segs[s].n;
  const uint64_t base = off + (uint64_t)(t - range_base[s]) * kRangeTile;
  const uint64_t end = min(off + n, base + kRangeTile);
  uint64_t mn = ~0ull, mx = 0ull;
  bool nan = false;
  auto take = [&](uint64_t b) {
    if (check_nan) nan |= is_nan_bits(b);
    const uint64_t o = ord_of(b, kt);
    mn = min(mn, o);
    mx = max(mx, o);
  };
  // 16-byte loads of two keys over the 16-byte aligned middle [a0, a1); the
  // key buffers are 8-byte aligned, so at most one key at each end is loaded
  // on its own
  const uint64_t a0 = min(end, base + (((uintptr_t)(keys + base) & 15u) ? 1u : 0u));
  const uint64_t a1 = a0 + ((end - a0) & ~(uint64_t)1);
  if (threadIdx.x == 0 && base < a0) take(ld_nc(keys + base));
  if (threadIdx.x == 32 && a1 < end) take(ld_nc(keys + a1));
  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(keys + a0);
  const uint32_t n2 = (uint32_t)((a1 - a0) >> 1);
  uint32_t q = threadIdx.x;
  for (; q + 3 * 256 < n2; q += 4 * 256) {
    const ulonglong2 w0 = __ldg(v2 + q), w1 = __ldg(v2 + q + 256), w2 = __ldg(v2 + q + 512),
                     w3 = __ldg(v2 + q + 768);
    take(w0.x);
    take(w0.y);
    take(w1.x);
    take(w1.y);
    take(w2.x);
    take(w2.y);
    take(w3.x);
    take(w3.y);
  }
  for (; q < n2; q += 256) {
    const ulonglong2 w = __ldg(v2 + q);
    take(w.x);
    take(w.y);
  }
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d));
    mx = max(mx, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d));
  }
  nan = __any_sync(~0u, nan);
  __shared__ uint64_t smn[8], smx[8];
  __shared__ int snan;
  if (threadIdx.x == 0) snan = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smn[w] = mn;
    smx[w] = mx;
    if (nan) snan = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < 8; ++k) {
      mn = min(mn, smn[k]);
      mx = max(mx, smx[k]);
    }
    atomicMin((unsigned long long*)&segs[s].ord_lo, (unsigned long long)mn);
    atomicMax((unsigned long long*)&segs[s].ord_hi, (unsigned long long)mx);
    if (snan) atomicOr(status, STATUS_NAN);
  }
}

// ---------------------------------------------------------------------------
// k_model: Alg. 1's early exits and the bin constants
// ---------------------------------------------------------------------------
__global__ void k_model(Seg* segs, uint32_t S, uint32_t kt, uint32_t model, uint32_t pass,
                        const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  Seg& g = segs[s];
  if (pass == 2 && g.status != SEG_NEEDRANGE) return;
  const uint64_t lo = bits_of_ord(g.ord_lo, kt), hi = bits_of_ord(g.ord_hi, kt);
  if (pass == 1) {
    // the samples' range (R14); equal or degenerate: the array's decides
    if (g.ord_lo == g.ord_hi || make_bin_model(kt, lo, hi, g.beta, &g.bm)) {
      g.status = SEG_NEEDRANGE;
      g.ord_lo = ~0ull;
      g.ord_hi = 0ull;
      return;
    }
    g.bm.clamp = 1;
    g.status = SEG_BUCKET;
  } else {
    if (g.ord_lo == g.ord_hi) {  // one distinct value: already sorted
      g.status = SEG_SINGLE;
      return;
    }
    g.status = make_bin_model(kt, lo, hi, g.beta, &g.bm) ? SEG_DEGEN : SEG_BUCKET;
  }
  if (g.status == SEG_BUCKET && model == MODEL_SPLINE) spline_set(&g.bm, g.alpha, g.gamma);
  if (g.status == SEG_BUCKET && gate) atomicAdd(&pcf_counters(gate)->bucketings, 1ull);
}

// min / max of each segment's alpha samples (R2's positions), per CTA of
// kSamplesPerCta samples, into the segment's range (the samples' range, R14)
__global__ void __launch_bounds__(256) k_sample_range(Seg* segs, uint32_t S,
                                                      const uint32_t* k1_base,
                                                      const uint64_t* __restrict__ keys,
                                                      uint32_t kt, const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t c = blockIdx.x;
  const uint32_t s = upper_bound_dev(k1_base, S + 1, c) - 1;
  Seg& g = segs[s];
  const uint32_t cta = c - k1_base[s];
  const uint64_t st = sample_state(g.seed, g.depth, g.start, g.n);
  const uint32_t j0 = cta * kSamplesPerCta, j1 = min(g.alpha, j0 + kSamplesPerCta);
  uint64_t mn = ~0ull, mx = 0ull;
  for (uint32_t j = j0 + threadIdx.x; j < j1; j += 256) {
    const uint64_t o = ord_of(ld_nc(keys + g.off + sample_index(st, j, g.n)), kt);
    mn = min(mn, o);
    mx = max(mx, o);
  }
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mn, d));
    mx = max(mx, (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)mx, d));
  }
  if ((threadIdx.x & 31) == 0 && mn <= mx) {
    atomicMin((unsigned long long*)&g.ord_lo, (unsigned long long)mn);
    atomicMax((unsigned long long*)&g.ord_hi, (unsigned long long)mx);
  }
}

// ---------------------------------------------------------------------------
// block-wide helpers (256 threads)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T u = __shfl_up_sync(~0u, v, d);
    if (l >= d) v += u;
  }
  return v;
}

// exclusive scan across the 256 threads; returns the block total in *total
template <typename T>
__device__ __forceinline__ T block_excl_scan256(T v, T* sh8, T* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  T inc = warp_incl_scan(v);
  if (l == 31) sh8[w] = inc;
  __syncthreads();
  T wsum = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    T x = sh8[k];
    if (k < w) wsum += x;
    tot += x;
  }
  __syncthreads();
  *total = tot;
  return wsum + inc - v;
}

// ---------------------------------------------------------------------------
// k_sample: training (Sec. 3.3): alpha samples drawn with replacement and
// counted per bin.  The cumulative counts b_k = |{j : bin(a_j) <= k}| come
// from one inclusive scan of the whole table pool (k_scan) and a per-segment
// base (k_seg_base), so that b_k = pool[T_off + k] - tbase.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sample(const Seg* segs, uint32_t S,
                                                const uint32_t* k1_base,
                                                const uint64_t* __restrict__ keys, uint32_t kt,
                                                uint32_t* tpool, const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t c = blockIdx.x;
  const uint32_t s = upper_bound_dev(k1_base, S + 1, c) - 1;
  const Seg& g = segs[s];
  if (g.status != SEG_BUCKET) return;
  __shared__ BinModel bm;
  if (threadIdx.x == 0) bm = g.bm;
  __syncthreads();
  const uint32_t cta = c - k1_base[s];
  const uint64_t st = sample_state(g.seed, g.depth, g.start, g.n);
  const uint32_t j0 = cta * kSamplesPerCta, j1 = min(g.alpha, j0 + kSamplesPerCta);
  uint32_t* cnt = tpool + g.T_off;
  for (uint32_t j = j0 + threadIdx.x; j < j1; j += 256) {
    uint64_t idx = sample_index(st, j, g.n);
    uint64_t x = ld_nc(keys + g.off + idx);
    atomicAdd(&cnt[bin_of(bm, x)], 1u);
  }
}

// tbase of each segment: the inclusive pool scan just before its table
__global__ void k_seg_base(Seg* segs, uint32_t S, const uint32_t* tpool, const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const uint64_t o = segs[s].T_off;
  segs[s].tbase = o ? tpool[o - 1] : 0u;
}

// ---------------------------------------------------------------------------
// bucket id of a key under segment g: T[bin(x)]
// ---------------------------------------------------------------------------
// bucket of a key under segment g (Alg. 1: floor(F(x) gamma), F = b_bin / alpha)
__device__ __forceinline__ uint32_t bucket_id(const BinModel& bm, const uint32_t* __restrict__ T,
                                              uint32_t tbase, uint32_t alpha, uint32_t gamma,
                                              uint64_t x) {
  return bucket_of_count(__ldg(T + bin_of(bm, x)) - tbase, alpha, gamma);
}

// warp-aggregated shared-memory histogram increment (match.any)
__device__ __forceinline__ void hist_add(uint32_t* hist, uint32_t d, bool valid) {
  const uint32_t key = valid ? d : 0xFFFFFFFFu;
  const uint32_t peers = __match_any_sync(~0u, key);
  const int leader = __ffs(peers) - 1;
  if (valid && (int)(threadIdx.x & 31) == leader) atomicAdd(&hist[d], (uint32_t)__popc(peers));
}

// ---------------------------------------------------------------------------
// k_hist1: per count-tile histogram of the high digit j >> b2
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hist_inc(uint32_t* hist, uint32_t d, bool valid, bool aggregate) {
  if (aggregate) hist_add(hist, d, valid);
  else if (valid) atomicAdd(&hist[d], 1u);
}

// k_hist1's PCF loop: the bucket id of every key of [base, end) into jout
// and the histogram of its high digit; CLAMP: the model spans the samples'
// range (R14).  Returns whether a NaN key was seen (check_nan).
template <bool CLAMP>
__device__ __forceinline__ bool hist1_pcf(const BinModel& bm, const Seg& g, uint64_t base,
                                          uint64_t end, const uint64_t* __restrict__ keys,
                                          const uint32_t* __restrict__ tpool, uint32_t* hist,
                                          uint32_t* __restrict__ jout, uint32_t b2, bool agg,
                                          int check_nan) {
  bool nan = false;
  {
    const uint32_t* T = tpool + g.T_off;
    const uint32_t tb = g.tbase, al = g.alpha, ga = g.gamma;
    constexpr int U = 8;
    for (uint64_t i0 = base; i0 < end; i0 += 256 * U) {
      uint64_t x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t i = i0 + (uint64_t)u * 256 + threadIdx.x;
        x[u] = i < end ? ld_nc(keys + i) : 0ull;
      }
      if (check_nan) {
#pragma unroll
        for (int u = 0; u < U; ++u) nan |= is_nan_bits(x[u]);
      }
      uint32_t bn[U], amb = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        bool a;
        bn[u] = CLAMP ? bin_fast_clamped(bm, x[u], a) : bin_fast(bm, x[u], a);
        amb |= (uint32_t)a << u;
      }
      if (amb) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if ((amb >> u) & 1u) bn[u] = bin_exact_of(bm, x[u]);
      }
      uint32_t tv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) tv[u] = __ldg(T + bn[u]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint64_t i = i0 + (uint64_t)u * 256 + threadIdx.x;
        const bool v = i < end;
        const uint32_t j = v ? bucket_of_count(tv[u] - tb, al, ga) : 0u;
        if (v) jout[i] = j;
        hist_inc(hist, j >> b2, v, agg);
      }
    }
  }
  return nan;
}

__global__ void __launch_bounds__(256, 4) k_hist1(const Seg* segs, uint32_t S,
                                               const uint32_t* tile_base, uint32_t tile_keys,
                                               const uint64_t* __restrict__ keys, uint32_t kt,
                                               const uint32_t* __restrict__ tpool,
                                               uint32_t* cmat, uint32_t* __restrict__ jout,
                                               int check_nan, uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ uint32_t hist[];
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(tile_base, S + 1, t) - 1;
  __shared__ BinModel bm;
  bool nan = false;
  const Seg& g = segs[s];
  const uint32_t tt = t - tile_base[s];
  const uint32_t D = 1u << g.b1, b2 = g.b2;
  // few digits: collisions are common, aggregate them per warp (match.any)
  const bool agg = D <= 64;
  for (uint32_t d = threadIdx.x; d < D; d += 256) hist[d] = 0;
  if (threadIdx.x == 0) bm = g.bm;
  __syncthreads();
  const uint64_t base = g.off + (uint64_t)tt * tile_keys;
  const uint64_t end = min(g.off + g.n, base + tile_keys);
  if (g.status != SEG_BUCKET) {
    // not bucketed: keep the count matrix consistent (all keys in digit 0)
    if (threadIdx.x == 0) hist[0] = (uint32_t)(end - base);
  } else if (bm.spline) {
    // spline model: the bin and the position in it in binary64, then
    // b_{k-1} and b_k from the table pool (inclusive scan values)
    const uint32_t* T = tpool + g.T_off;
    const uint32_t tb = g.tbase;
    for (uint64_t i0 = base; i0 < end; i0 += 256) {
      const uint64_t i = i0 + threadIdx.x;
      const bool v = i < end;
      uint32_t j = 0;
      if (v) {
        double f;
        const uint64_t x = ld_nc(keys + i);
        if (check_nan) nan |= is_nan_bits(x);
        const uint32_t k = spline_bin(bm, x, &f);
        const uint32_t bk = __ldg(T + k) - tb, bkm1 = k ? __ldg(T + k - 1) - tb : 0u;
        j = spline_bucket(bm, f, bkm1, bk);
        jout[i] = j;
      }
      hist_inc(hist, j >> b2, v, agg);
    }
  } else if (bm.clamp) {
    nan |= hist1_pcf<true>(bm, g, base, end, keys, tpool, hist, jout, b2, agg, check_nan);
  } else {
    nan |= hist1_pcf<false>(bm, g, base, end, keys, tpool, hist, jout, b2, agg, check_nan);
  }
  if (check_nan && __any_sync(~0u, nan) && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_NAN);
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < D; d += 256) cmat[g.cbase1 + (uint64_t)d * g.tiles1 + tt] = hist[d];
}


// ---------------------------------------------------------------------------
// k_scan: exclusive prefix sum of u32 data[0..n) in place, single pass with
// decoupled look-back (Merrill & Garland 2016).  Tiles take their index from
// an atomic counter, so every predecessor of a tile has started; each wait
// on a predecessor's flag is bounded and gives up with STATUS_TIMEOUT.
// Status word: [63:62] flag (0 none, 1 aggregate, 2 inclusive), [31:0] value.
// `withhold` (test hook): that tile never publishes its aggregate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void publish(uint64_t* w, uint64_t flag, uint32_t v) {
  __threadfence();
  atomicExch((unsigned long long*)w, (unsigned long long)((flag << 62) | v));
}

__global__ void __launch_bounds__(256) k_scan(uint32_t* data, uint64_t n, const uint64_t* n_dev,
                                              uint64_t* sw, uint32_t* tile_counter,
                                              uint32_t withhold, uint64_t spin_limit,
                                              uint64_t* total_out, uint32_t* status,
                                              int inclusive) {
  __shared__ uint32_t s_tile, s_prefix;
  __shared__ uint32_t sh8[8];
  __shared__ uint32_t buf[kScanTile];
  // gated before taking a tile: the tiles no CTA takes are the last ones,
  // which no taken tile waits on
  if (pcf_aborted(status)) return;
  if (n_dev) n = *n_dev;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * kScanTile;
  if (base >= n) return;
  const uint32_t cnt = (uint32_t)min((uint64_t)kScanTile, n - base);
  for (uint32_t i = threadIdx.x; i < kScanTile; i += 256) buf[i] = i < cnt ? data[base + i] : 0u;
  __syncthreads();
  uint32_t v[16], sum = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = buf[threadIdx.x * 16 + k];
    sum += v[k];
  }
  uint32_t tot;
  uint32_t ex = block_excl_scan256(sum, sh8, &tot);
  if (threadIdx.x == 0) {
    uint32_t prefix = 0;
    if (tile == 0) {
      publish(&sw[0], 2, tot);
    } else {
      if (tile != withhold) publish(&sw[tile], 1, tot);
      uint64_t spins = 0;
      int64_t p = (int64_t)tile - 1;
      while (p >= 0) {
        uint64_t w = atomicAdd((unsigned long long*)&sw[p], 0ull);
        uint32_t f = (uint32_t)(w >> 62);
        if (f == 0) {
          if (++spins > spin_limit) {
            atomicOr(status, STATUS_TIMEOUT);
            break;
          }
          __nanosleep(64);
          continue;
        }
        prefix += (uint32_t)w;
        if (f == 2) break;
        --p;
      }
      if (tile != withhold) publish(&sw[tile], 2, prefix + tot);
    }
    s_prefix = prefix;
    if (total_out && base + cnt == n) *total_out = (uint64_t)prefix + tot;
  }
  __syncthreads();
  ex += s_prefix;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    buf[threadIdx.x * 16 + k] = inclusive ? ex + v[k] : ex;
    ex += v[k];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += 256) data[base + i] = buf[i];
}

// ---------------------------------------------------------------------------
// Stable scatter of one count tile (tile_n keys), by digit.  The tile is
// staged in sub-tiles of kScatterSub keys: each warp ranks its contiguous
// 512 keys in order (match.any + per-warp counters), the ranks are turned
// into a digit-sorted order in shared memory, and the sub-tile is written
// out with consecutive threads storing consecutive keys of each digit run.
// s_gofs[d] holds the next global position of digit d for this tile.
// ---------------------------------------------------------------------------
constexpr int kItems = 16;  // keys per thread per sub-tile (256 threads)

struct ScatterSmem {
  uint16_t* wcnt;   // [8][D]
  uint16_t* dbase;  // [D] sub-tile digit base
  uint16_t* dtot;   // [D]
  uint32_t* gofs;   // [D]
  uint64_t* skey;   // [kScatterSub]
  uint16_t* sdig;   // [kScatterSub]
  uint16_t* saux;   // [kScatterSub] (pass 1)
  uint32_t* sval;   // [kScatterSub] (pairs)
};

__host__ __device__ inline size_t scatter_smem_bytes(uint32_t D, bool pairs, bool aux) {
  size_t b = (size_t)8 * D * 2 + (size_t)D * 2 * 2 + (size_t)D * 4;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)kScatterSub * 8 + (size_t)kScatterSub * 2;
  if (aux) b += (size_t)kScatterSub * 2;
  if (pairs) b += (size_t)kScatterSub * 4;
  return b + 64;
}

__device__ __forceinline__ ScatterSmem carve_scatter(uint8_t* p, uint32_t D, bool pairs, bool aux) {
  ScatterSmem m;
  m.wcnt = (uint16_t*)p;
  p += (size_t)8 * D * 2;
  m.dbase = (uint16_t*)p;
  p += (size_t)D * 2;
  m.dtot = (uint16_t*)p;
  p += (size_t)D * 2;
  m.gofs = (uint32_t*)p;
  p += (size_t)D * 4;
  p = (uint8_t*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  m.skey = (uint64_t*)p;
  p += (size_t)kScatterSub * 8;
  m.sdig = (uint16_t*)p;
  p += (size_t)kScatterSub * 2;
  m.saux = nullptr;
  m.sval = nullptr;
  if (aux) {
    m.saux = (uint16_t*)p;
    p += (size_t)kScatterSub * 2;
  }
  if (pairs) m.sval = (uint32_t*)p;
  return m;
}

// PASS 1: digit = T[bin(x)] >> b2, carry = low b2 bits.  PASS 2: digit = carry.
template <int PASS, bool PAIRS>
__device__ void scatter_tile(const ScatterSmem& sm, uint32_t D, uint64_t tile_off, uint32_t tile_n,
                             const uint32_t* __restrict__ src_j, uint32_t b2,
                             const uint64_t* __restrict__ src, const uint32_t* __restrict__ src_v,
                             const uint16_t* __restrict__ src_aux, uint64_t* __restrict__ dst,
                             uint32_t* __restrict__ dst_v, uint16_t* __restrict__ dst_aux,
                             uint32_t* status = nullptr) {
  (void)status;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const uint32_t lmask = lanemask_lt();
  const uint32_t low_mask = (1u << b2) - 1u;
  for (uint32_t sub = 0; sub < tile_n; sub += kScatterSub) {
    const uint32_t nsub = min(kScatterSub, tile_n - sub);
    {
      uint4* z = reinterpret_cast<uint4*>(sm.wcnt);  // 8*D u16, D a power of two >= 1
      const uint32_t nz = (8 * D * 2 + 15) / 16;
      for (uint32_t i = tid; i < nz; i += 256) z[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    uint64_t key[kItems];
    uint32_t dig[kItems], aux[kItems], rank[kItems], val[kItems];
    const uint64_t g0 = tile_off + sub;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = (uint32_t)w * (32 * kItems) + (uint32_t)k * 32 + (uint32_t)l;
      const bool v = li < nsub;
      key[k] = v ? ld_nc(src + g0 + li) : 0ull;
      if (PAIRS) val[k] = v ? __ldg(src_v + g0 + li) : 0u;
      if (PASS == 2) dig[k] = v ? (uint32_t)__ldg(src_aux + g0 + li) : 0u;
    }
    if (PASS == 1) {
      // the bucket id j of every key was stored by the histogram pass
#pragma unroll
      for (int k = 0; k < kItems; ++k) {
        const uint32_t li = (uint32_t)w * (32 * kItems) + (uint32_t)k * 32 + (uint32_t)l;
        const uint32_t j = li < nsub ? __ldg(src_j + g0 + li) : 0u;
        dig[k] = j >> b2;
        aux[k] = j & low_mask;
      }
    }
    // per-warp counters, u16 in shared memory, updated with 32-bit atomics
    // on the aligned word holding them.  Key-value sorts rank stably: one
    // leader per digit per step (match.any), and shared atomics of one warp
    // apply in program order, so ranks follow input order.  Keys-only sorts
    // let every key take its rank from its own atomic: keys of one digit in
    // one step may then land in either order, which no result can show
    // (equal keys are indistinguishable, and every bucket is sorted later).
    uint16_t* my = sm.wcnt + (size_t)w * D;
    uint32_t* myw = reinterpret_cast<uint32_t*>(my);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = (uint32_t)w * (32 * kItems) + (uint32_t)k * 32 + (uint32_t)l;
      const bool v = li < nsub;
      if (!PAIRS) {
        uint32_t prior = 0;
        if (v) {
          const uint32_t sh = (dig[k] & 1u) * 16u;
          prior = (atomicAdd(&myw[dig[k] >> 1], 1u << sh) >> sh) & 0xFFFFu;
        }
        rank[k] = prior;
        continue;
      }
      const uint32_t peers = __match_any_sync(~0u, v ? dig[k] : 0xFFFFFFFFu);
      const int leader = __ffs(peers) - 1;
      uint32_t prior = 0;
      if (v && l == leader) {
        const uint32_t sh = (dig[k] & 1u) * 16u;
        prior = (atomicAdd(&myw[dig[k] >> 1], (uint32_t)__popc(peers) << sh) >> sh) & 0xFFFFu;
      }
      prior = __shfl_sync(~0u, prior, leader);
      rank[k] = prior + __popc(peers & lmask);
    }
    __syncthreads();
    // column prefix over warps, digit totals
    for (uint32_t d = tid; d < D; d += 256) {
      uint32_t run = 0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        uint32_t c = sm.wcnt[(size_t)ww * D + d];
        sm.wcnt[(size_t)ww * D + d] = (uint16_t)run;
        run += c;
      }
      sm.dtot[d] = (uint16_t)run;
    }
    __syncthreads();
    // exclusive scan of digit totals -> dbase (each thread a contiguous run)
    {
      __shared__ uint32_t sh8[8];
      const uint32_t per = (D + 255) / 256;
      const uint32_t d0 = min(D, (uint32_t)tid * per), d1 = min(D, d0 + per);
      uint32_t sum = 0;
      for (uint32_t d = d0; d < d1; ++d) sum += sm.dtot[d];
      uint32_t tot;
      uint32_t ex = block_excl_scan256(sum, sh8, &tot);
      for (uint32_t d = d0; d < d1; ++d) {
        sm.dbase[d] = (uint16_t)ex;
        ex += sm.dtot[d];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = (uint32_t)w * (32 * kItems) + (uint32_t)k * 32 + (uint32_t)l;
      if (li < nsub) {
        const uint32_t pos = sm.dbase[dig[k]] + my[dig[k]] + rank[k];
        if (!PCF_IN(pos, nsub, status)) continue;
        sm.skey[pos] = key[k];
        sm.sdig[pos] = (uint16_t)dig[k];
        if (PASS == 1) sm.saux[pos] = (uint16_t)aux[k];
        if (PAIRS) sm.sval[pos] = val[k];
      }
    }
    __syncthreads();
    // write-out in staged (digit) order; unrolled so that the shared loads
    // of all items are in flight together
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t pos = (uint32_t)tid + (uint32_t)k * 256u;
      if (pos < nsub) {
        const uint32_t d = sm.sdig[pos];
        const uint64_t o = (uint64_t)sm.gofs[d] + (pos - sm.dbase[d]);
        if (!PCF_IN_KEYS(o, status)) continue;
        dst[o] = sm.skey[pos];
        if (PASS == 1) dst_aux[o] = sm.saux[pos];
        if (PAIRS) dst_v[o] = sm.sval[pos];
      }
    }
    __syncthreads();
    for (uint32_t d = tid; d < D; d += 256) sm.gofs[d] += sm.dtot[d];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same stable scatter for keys-only sorts, with the sub-tiles staged by
// bulk copies.  Two stages alternate: while the CTA ranks and writes one
// sub-tile, the next one is already in flight into the other stage (one
// cp.async.bulk for the keys and one for the digit words, completing on the
// stage's mbarrier).  A consumed stage then serves as the staging area of
// the digit-sorted sub-tile (keys, and the digit / carried low digit as u16
// beside them) before the copy two sub-tiles ahead is issued into it.  The
// ranks and the order of the write-out are those of scatter_tile.
// ---------------------------------------------------------------------------
template <int PASS>
struct BulkStage {
  static constexpr uint32_t kKeySlots = kScatterSub + 2;  // +2: 16-byte alignment shift
  // digit words: pass 1 u32 bucket ids, pass 2 u16 low digits (+ shift slack)
  static constexpr uint32_t kWordBytes = PASS == 1 ? (kScatterSub + 4) * 4 : (kScatterSub + 8) * 2;
  static constexpr uint32_t kBytes = kKeySlots * 8 + ((kWordBytes + 15) & ~15u);
};

__host__ __device__ inline size_t scatter_bulk_smem_bytes(uint32_t D, int pass) {
  size_t b = (size_t)8 * D * 2 + (size_t)D * 2 * 2 + (size_t)D * 4;
  b = (b + 15) & ~(size_t)15;
  b += 2 * (size_t)(pass == 1 ? BulkStage<1>::kBytes : BulkStage<2>::kBytes);
  return b + 16;  // two mbarriers
}

// Issues the copy of keys [g0, g0 + n) and their digit words into stage st.
// The 16-byte-aligned middle of each array goes by bulk copy; the at most
// one key and three (pass 1) or seven (pass 2) words at the ragged ends are
// loaded by threads 32.. with plain loads.
template <int PASS>
__device__ __forceinline__ void bulk_stage_issue(uint8_t* st, uint64_t* bar, const uint64_t* keys,
                                                 const void* words, uint64_t g0, uint32_t n,
                                                 uint32_t tid) {
  constexpr uint32_t WB = PASS == 1 ? 4u : 2u;       // bytes per word
  constexpr uint32_t WA = 16u / WB;                  // words per 16 bytes
  uint64_t* K = reinterpret_cast<uint64_t*>(st);
  uint8_t* Wd = st + BulkStage<PASS>::kKeySlots * 8;
  const uint64_t kq = (reinterpret_cast<uintptr_t>(keys) >> 3) & 1u;
  const uint64_t wq = (reinterpret_cast<uintptr_t>(words) / WB) & (WA - 1);
  const uint64_t e = g0 + n;
  // keys: slot of key g0 + i is i + ks
  const uint32_t ks = (uint32_t)((g0 + kq) & 1u);
  const uint64_t ka0 = min(e, ((g0 + kq + 1) & ~(uint64_t)1) - kq);
  const uint64_t ka1 = max(ka0, ((e + kq) & ~(uint64_t)1) - kq);
  // words: slot of word g0 + i is i + ws
  const uint32_t ws = (uint32_t)((g0 + wq) & (WA - 1));
  const uint64_t wa0 = min(e, ((g0 + wq + (uint64_t)(WA - 1)) & ~(uint64_t)(WA - 1)) - wq);
  const uint64_t wa1 = max(wa0, ((e + wq) & ~(uint64_t)(WA - 1)) - wq);
  if (tid == 0) {
    const uint32_t kb = (uint32_t)(ka1 - ka0) * 8u, wb = (uint32_t)(wa1 - wa0) * WB;
    mbar_arrive_tx(bar, kb + wb);
    if (kb) bulk_g2s(K + (ka0 - g0 + ks), keys + ka0, kb, bar);
    if (wb)
      bulk_g2s(Wd + (size_t)(wa0 - g0 + ws) * WB,
               reinterpret_cast<const uint8_t*>(words) + wa0 * WB, wb, bar);
  }
  // ragged ends: thread 32 + h for h < 2 the keys, then the words
  if (tid >= 32 && tid < 32 + 2 + 2 * (WA - 1)) {
    const uint32_t h = tid - 32;
    if (h == 0) {
      if (ka0 > g0) K[ks] = __ldg(keys + g0);
    } else if (h == 1) {
      if (ka1 < e) K[ka1 - g0 + ks] = __ldg(keys + ka1);
    } else {
      const uint32_t u = h - 2;  // 0 .. 2 (WA - 1) - 1
      const uint64_t g = u < WA - 1 ? g0 + u : wa1 + (u - (WA - 1));
      const bool v = u < WA - 1 ? g < wa0 : g < e;
      if (v) {
        if (PASS == 1)
          reinterpret_cast<uint32_t*>(Wd)[g - g0 + ws] =
              __ldg(reinterpret_cast<const uint32_t*>(words) + g);
        else
          reinterpret_cast<uint16_t*>(Wd)[g - g0 + ws] =
              __ldg(reinterpret_cast<const uint16_t*>(words) + g);
      }
    }
  }
}

// One count tile of a keys-only scatter, sub-tiles staged by bulk copies.
// sm_stage: the two stages; bars: their mbarriers (initialised, phases in
// ph).  Returns false when a staging wait gave up (STATUS_TIMEOUT set).
template <int PASS>
__device__ bool scatter_tile_bulk(const ScatterSmem& sm, uint8_t* stages, uint64_t* bars,
                                  uint32_t D, uint64_t tile_off, uint32_t tile_n,
                                  const void* __restrict__ words, uint32_t b2,
                                  const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                                  uint16_t* __restrict__ dst_aux, uint32_t* status) {
  (void)status;
  const uint32_t tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const uint32_t low_mask = (1u << b2) - 1u;
  constexpr uint32_t WA = PASS == 1 ? 4u : 8u;
  const uint32_t nsubs = (tile_n + kScatterSub - 1) / kScatterSub;
  uint32_t ph = 0;  // bit b: the phase stage b waits for next
  // the first two sub-tiles
  for (uint32_t s = 0; s < 2 && s < nsubs; ++s)
    bulk_stage_issue<PASS>(stages + (size_t)s * BulkStage<PASS>::kBytes, bars + s, src, words,
                           tile_off + (uint64_t)s * kScatterSub,
                           min(kScatterSub, tile_n - s * kScatterSub), tid);
  for (uint32_t s = 0; s < nsubs; ++s) {
    const uint32_t b = s & 1u;
    uint8_t* st = stages + (size_t)b * BulkStage<PASS>::kBytes;
    uint64_t* K = reinterpret_cast<uint64_t*>(st);
    uint8_t* Wd = st + BulkStage<PASS>::kKeySlots * 8;
    const uint64_t g0 = tile_off + (uint64_t)s * kScatterSub;
    const uint32_t nsub = min(kScatterSub, tile_n - s * kScatterSub);
    const uint32_t ks = (uint32_t)((g0 + ((reinterpret_cast<uintptr_t>(src) >> 3) & 1u)) & 1u);
    const uint32_t ws = (uint32_t)((g0 + (reinterpret_cast<uintptr_t>(words) /
                                          (PASS == 1 ? 4u : 2u))) & (WA - 1));
    {
      uint4* z = reinterpret_cast<uint4*>(sm.wcnt);  // 8*D u16, D a power of two >= 1
      const uint32_t nz = (8 * D * 2 + 15) / 16;
      for (uint32_t i = tid; i < nz; i += 256) z[i] = make_uint4(0, 0, 0, 0);
    }
    const bool ok = mbar_wait(bars + b, (ph >> b) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(status, STATUS_TIMEOUT);
      // one more bounded wait for each copy in flight before leaving
      mbar_wait(bars + b, (ph >> b) & 1u);
      if (s + 1 < nsubs) mbar_wait(bars + (b ^ 1u), (ph >> (b ^ 1u)) & 1u);
      return false;
    }
    ph ^= 1u << b;
    uint64_t key[kItems];
    uint32_t dig[kItems], aux[kItems], rank[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = w * (32 * kItems) + (uint32_t)k * 32 + l;
      const bool v = li < nsub;
      key[k] = v ? K[li + ks] : 0ull;
      if (PASS == 1) {
        const uint32_t j = v ? reinterpret_cast<const uint32_t*>(Wd)[li + ws] : 0u;
        dig[k] = j >> b2;
        aux[k] = j & low_mask;
      } else {
        dig[k] = v ? (uint32_t)reinterpret_cast<const uint16_t*>(Wd)[li + ws] : 0u;
        aux[k] = 0u;
      }
    }
    uint16_t* my = sm.wcnt + (size_t)w * D;
    uint32_t* myw = reinterpret_cast<uint32_t*>(my);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = w * (32 * kItems) + (uint32_t)k * 32 + l;
      uint32_t prior = 0;
      if (li < nsub) {
        const uint32_t sh = (dig[k] & 1u) * 16u;
        prior = (atomicAdd(&myw[dig[k] >> 1], 1u << sh) >> sh) & 0xFFFFu;
      }
      rank[k] = prior;
    }
    __syncthreads();  // every thread holds its items: the stage is free
    for (uint32_t d = tid; d < D; d += 256) {
      uint32_t run = 0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        uint32_t c = sm.wcnt[(size_t)ww * D + d];
        sm.wcnt[(size_t)ww * D + d] = (uint16_t)run;
        run += c;
      }
      sm.dtot[d] = (uint16_t)run;
    }
    __syncthreads();
    {
      __shared__ uint32_t sh8[8];
      const uint32_t per = (D + 255) / 256;
      const uint32_t d0 = min(D, tid * per), d1 = min(D, d0 + per);
      uint32_t sum = 0;
      for (uint32_t d = d0; d < d1; ++d) sum += sm.dtot[d];
      uint32_t tot;
      uint32_t ex = block_excl_scan256(sum, sh8, &tot);
      for (uint32_t d = d0; d < d1; ++d) {
        sm.dbase[d] = (uint16_t)ex;
        ex += sm.dtot[d];
      }
    }
    __syncthreads();
    // the digit-sorted sub-tile in the consumed stage: keys in K, digit and
    // carried low digit as u16 in the word area
    uint16_t* sdig = reinterpret_cast<uint16_t*>(Wd);
    uint16_t* saux = sdig + kScatterSub;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t li = w * (32 * kItems) + (uint32_t)k * 32 + l;
      if (li < nsub) {
        const uint32_t pos = sm.dbase[dig[k]] + my[dig[k]] + rank[k];
        if (!PCF_IN(pos, nsub, status)) continue;
        K[pos] = key[k];
        sdig[pos] = (uint16_t)dig[k];
        if (PASS == 1) saux[pos] = (uint16_t)aux[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const uint32_t pos = tid + (uint32_t)k * 256u;
      if (pos < nsub) {
        const uint32_t d = sdig[pos];
        const uint64_t o = (uint64_t)sm.gofs[d] + (pos - sm.dbase[d]);
        if (!PCF_IN_KEYS(o, status)) continue;
        dst[o] = K[pos];
        if (PASS == 1) dst_aux[o] = saux[pos];
      }
    }
    __syncthreads();  // the stage is read out
    for (uint32_t d = tid; d < D; d += 256) sm.gofs[d] += sm.dtot[d];
    if (s + 2 < nsubs)
      bulk_stage_issue<PASS>(st, bars + b, src, words, g0 + 2ull * kScatterSub,
                             min(kScatterSub, tile_n - (s + 2) * kScatterSub), tid);
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------
// k_scatter1: pass 1 (src -> tmp), digit = high bits of the bucket id
// ---------------------------------------------------------------------------
template <bool PAIRS>
__global__ void __launch_bounds__(256, 2) k_scatter1(const Seg* segs, uint32_t S,
                                                  const uint32_t* tile_base, uint32_t tile_keys,
                                                  KeyBufs kb, const uint32_t* __restrict__ tpool,
                                                  const uint32_t* __restrict__ cmat,
                                                  uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(tile_base, S + 1, t) - 1;
  const Seg& g = segs[s];
  if (g.status != SEG_BUCKET) return;
  const uint32_t tt = t - tile_base[s];
  const uint32_t D = 1u << g.b1;
  const uint32_t seg_base = cmat[g.cbase1];  // exclusive prefix at the segment's first entry
  const uint64_t tile_off = g.off + (uint64_t)tt * tile_keys;
  const uint32_t tile_n = (uint32_t)min((uint64_t)tile_keys, g.off + g.n - tile_off);
  ScatterSmem sm = carve_scatter(smem_raw, D, PAIRS, true);
  for (uint32_t d = threadIdx.x; d < D; d += 256)
    sm.gofs[d] = (uint32_t)g.off + (cmat[g.cbase1 + (uint64_t)d * g.tiles1 + tt] - seg_base);
  __syncthreads();
  scatter_tile<1, PAIRS>(sm, D, tile_off, tile_n, kb.jbuf, g.b2, kb.src, kb.src_v, nullptr, kb.tmp,
                         kb.tmp_v, kb.tmp_aux, status);
}

// k_scatter1 for keys-only sorts with the sub-tiles staged by bulk copies
__global__ void __launch_bounds__(256, 2) k_scatter1_bulk(const Seg* segs, uint32_t S,
                                                        const uint32_t* tile_base,
                                                        uint32_t tile_keys, KeyBufs kb,
                                                        const uint32_t* __restrict__ cmat,
                                                        uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(tile_base, S + 1, t) - 1;
  const Seg& g = segs[s];
  if (g.status != SEG_BUCKET) return;
  const uint32_t tt = t - tile_base[s];
  const uint32_t D = 1u << g.b1;
  const uint32_t seg_base = cmat[g.cbase1];
  const uint64_t tile_off = g.off + (uint64_t)tt * tile_keys;
  const uint32_t tile_n = (uint32_t)min((uint64_t)tile_keys, g.off + g.n - tile_off);
  ScatterSmem sm = carve_scatter(smem_raw, D, false, false);
  uint8_t* stages = reinterpret_cast<uint8_t*>(sm.skey);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + 2 * (size_t)BulkStage<1>::kBytes);
  if (threadIdx.x == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
  }
  for (uint32_t d = threadIdx.x; d < D; d += 256)
    sm.gofs[d] = (uint32_t)g.off + (cmat[g.cbase1 + (uint64_t)d * g.tiles1 + tt] - seg_base);
  __syncthreads();
  scatter_tile_bulk<1>(sm, stages, bars, D, tile_off, tile_n, kb.jbuf, g.b2, kb.src, kb.tmp,
                       kb.tmp_aux, status);
}

// k_scatter2 for keys-only sorts with the sub-tiles staged by bulk copies
__global__ void __launch_bounds__(256, 2) k_scatter2_bulk(const Group* groups, uint32_t n_groups,
                                                        const Seg* segs,
                                                        const uint32_t* g_tile_scan,
                                                        const uint64_t* total_tiles,
                                                        uint32_t tile_keys, KeyBufs kb,
                                                        const uint32_t* __restrict__ cmat2,
                                                        uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t t = blockIdx.x;
  if (t >= *total_tiles) return;
  const uint32_t G = upper_bound_dev(g_tile_scan, n_groups, t) - 1;
  const Group gr = groups[G];
  if (segs[gr.seg].b2 == 0) return;  // one-digit id: copied, not scattered
  const uint32_t D = 1u << segs[gr.seg].b2;
  const uint32_t tt = t - g_tile_scan[G];
  const uint32_t gbase = cmat2[gr.cbase];
  const uint64_t tile_off = gr.off + (uint64_t)tt * tile_keys;
  const uint32_t tile_n = (uint32_t)min((uint64_t)tile_keys, gr.off + gr.n - tile_off);
  ScatterSmem sm = carve_scatter(smem_raw, D, false, false);
  uint8_t* stages = reinterpret_cast<uint8_t*>(sm.skey);
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + 2 * (size_t)BulkStage<2>::kBytes);
  if (threadIdx.x == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
  }
  for (uint32_t d = threadIdx.x; d < D; d += 256)
    sm.gofs[d] = (uint32_t)gr.off + (cmat2[gr.cbase + (uint64_t)d * gr.tiles + tt] - gbase);
  __syncthreads();
  scatter_tile_bulk<2>(sm, stages, bars, D, tile_off, tile_n, kb.tmp_aux, 0, kb.tmp, kb.out,
                       nullptr, status);
}

// ---------------------------------------------------------------------------
// k_groups: one thread per pass-1 group (segment s, high digit g): size,
// offset and number of pass-2 count tiles.
// ---------------------------------------------------------------------------
__global__ void k_groups(const Seg* segs, uint32_t S, const uint64_t* group_base_dev,
                         uint64_t n_groups, const uint32_t* cmat1, uint32_t tile_keys,
                         Group* groups, uint32_t* g_tiles, uint32_t* g_centries,
                         const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint64_t G = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= n_groups) return;
  const uint32_t s = upper_bound_dev(group_base_dev, S + 1, G) - 1;
  const Seg& sg = segs[s];
  const uint32_t g = (uint32_t)(G - sg.group_base);
  Group gr;
  gr.seg = s;
  gr.pad = 0;
  gr.n = 0;
  gr.off = sg.off;
  gr.key_prefix = 0;
  gr.cbase = 0;
  if (sg.status == SEG_BUCKET && sg.b2 == 0) {
    // no second digit: pass 2 is one copy of the whole segment
    if (g == 0) gr.n = (uint32_t)sg.n;
  } else if (sg.status == SEG_BUCKET) {
    const uint32_t D1 = 1u << sg.b1;
    const uint32_t seg_base = cmat1[sg.cbase1];
    const uint32_t a = cmat1[sg.cbase1 + (uint64_t)g * sg.tiles1] - seg_base;
    const uint32_t b = (g + 1 < D1) ? cmat1[sg.cbase1 + (uint64_t)(g + 1) * sg.tiles1] - seg_base
                                    : (uint32_t)sg.n;
    gr.off = sg.off + a;
    gr.n = b - a;
  }
  gr.tiles = (uint32_t)(((uint64_t)gr.n + tile_keys - 1) / tile_keys);
  groups[G] = gr;
  g_tiles[G] = gr.tiles;
  g_centries[G] = gr.tiles << sg.b2;
}

// cbase of every group from the scanned entry counts
__global__ void k_group_bases(Group* groups, uint64_t n_groups, const uint32_t* g_centries_scan,
                              const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint64_t G = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= n_groups) return;
  groups[G].cbase = g_centries_scan[G];
}

// ---------------------------------------------------------------------------
// k_hist2 / k_scatter2: pass 2 within each group, digit = carried low bits
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_hist2(const Group* groups, uint32_t n_groups,
                                               const Seg* segs, const uint32_t* g_tile_scan,
                                               const uint64_t* total_tiles, uint32_t tile_keys,
                                               const uint16_t* __restrict__ aux,
                                               uint32_t* cmat2, const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  extern __shared__ uint32_t hist[];
  const uint32_t t = blockIdx.x;
  if (t >= *total_tiles) return;
  const uint32_t G = upper_bound_dev(g_tile_scan, n_groups, t) - 1;
  const Group gr = groups[G];
  if (segs[gr.seg].b2 == 0) return;  // one-digit id: copied, not scattered
  const uint32_t D = 1u << segs[gr.seg].b2;
  const bool agg = D <= 64;
  const uint32_t tt = t - g_tile_scan[G];
  for (uint32_t d = threadIdx.x; d < D; d += 256) hist[d] = 0;
  __syncthreads();
  const uint64_t base = gr.off + (uint64_t)tt * tile_keys;
  const uint64_t end = min(gr.off + gr.n, base + tile_keys);
  // 16-byte loads of eight digits over the aligned middle, single digits
  // at the ragged ends
  const uint64_t a0 = min(end, (base + 7) & ~(uint64_t)7), a1 = max(a0, end & ~(uint64_t)7);
  {
    // fewer than 8 digits at each end: threads 0-7 the head, 8-15 the tail
    // (every lane takes part, as the warp-aggregated increment needs)
    const uint64_t i = threadIdx.x < 8 ? base + threadIdx.x : a1 + (threadIdx.x - 8);
    const bool v = threadIdx.x < 8 ? i < a0 : (threadIdx.x < 16 && i < end);
    hist_inc(hist, v ? (uint32_t)__ldg(aux + i) : 0u, v, agg);
  }
  const uint4* v4 = reinterpret_cast<const uint4*>(aux + a0);
  const uint32_t n4 = (uint32_t)((a1 - a0) >> 3);
  constexpr int U = 2;
  for (uint32_t q0 = 0; q0 < n4; q0 += 256 * U) {
    uint4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t q = q0 + (uint32_t)u * 256 + threadIdx.x;
      w[u] = q < n4 ? __ldg(v4 + q) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool v = q0 + (uint32_t)u * 256 + threadIdx.x < n4;
      const uint32_t ws[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        hist_inc(hist, ws[h] & 0xFFFFu, v, agg);
        hist_inc(hist, ws[h] >> 16, v, agg);
      }
    }
  }
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < D; d += 256)
    cmat2[gr.cbase + (uint64_t)d * gr.tiles + tt] = hist[d];
}

template <bool PAIRS>
__global__ void __launch_bounds__(256, 2) k_scatter2(const Group* groups, uint32_t n_groups,
                                                  const Seg* segs, const uint32_t* g_tile_scan,
                                                  const uint64_t* total_tiles, uint32_t tile_keys,
                                                  KeyBufs kb, const uint32_t* __restrict__ cmat2,
                                                  uint32_t* status) {
  if (pcf_aborted(status)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const uint32_t t = blockIdx.x;
  if (t >= *total_tiles) return;
  const uint32_t G = upper_bound_dev(g_tile_scan, n_groups, t) - 1;
  const Group gr = groups[G];
  if (segs[gr.seg].b2 == 0) return;  // one-digit id: copied, not scattered
  const uint32_t D = 1u << segs[gr.seg].b2;
  const uint32_t tt = t - g_tile_scan[G];
  const uint32_t gbase = cmat2[gr.cbase];
  const uint64_t tile_off = gr.off + (uint64_t)tt * tile_keys;
  const uint32_t tile_n = (uint32_t)min((uint64_t)tile_keys, gr.off + gr.n - tile_off);
  ScatterSmem sm = carve_scatter(smem_raw, D, PAIRS, false);
  for (uint32_t d = threadIdx.x; d < D; d += 256)
    sm.gofs[d] = (uint32_t)gr.off + (cmat2[gr.cbase + (uint64_t)d * gr.tiles + tt] - gbase);
  __syncthreads();
  scatter_tile<2, PAIRS>(sm, D, tile_off, tile_n, nullptr, 0, kb.tmp, kb.tmp_v, kb.tmp_aux, kb.out,
                         kb.out_v, nullptr, status);
}

// ---------------------------------------------------------------------------
// k_buckets: Alg. 1's loop over buckets.  For bucket j of segment s:
// |c_j| >= delta -> standard sort; |c_j| <= leaf_cap -> shared-memory kernel
// (which itself applies n < tau); otherwise Learned-Sort at the next level.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
  const uint32_t m = __ballot_sync(~0u, want);
  if (!m) return 0;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(~0u, base, leader);
  return base + __popc(m & lanemask_lt());
}

constexpr uint32_t kTiny = 16;  // buckets this small are sorted by one thread

template <bool PAIRS>
__global__ void __launch_bounds__(256) k_buckets(const Seg* segs, uint32_t S, uint64_t n_buckets,
                                                 const uint64_t* bucket_base, const Group* groups,
                                                 const uint32_t* __restrict__ cmat1,
                                                 const uint32_t* __restrict__ cmat2, int two_pass,
                                                 uint32_t leaf_cap, uint32_t tau, uint32_t kt,
                                                 const uint64_t* __restrict__ X,
                                                 const uint32_t* __restrict__ Xv, uint64_t* out_k,
                                                 uint32_t* out_v, BRec* brec, uint32_t* next_flag,
                                                 FbItem* fb, LevelOut* lo, uint32_t max_items,
                                                 uint2* leaf_lists, uint32_t* leaf_counts,
                                                 uint32_t leaf_classes, uint32_t* mid_list,
                                                 uint32_t* mid_count, uint32_t* status) {
  if (pcf_aborted(status)) return;
  // [kTiny][256] (transposed: thread t owns column t, so accesses are
  // conflict-free)
  __shared__ uint64_t tk[kTiny][256];
  __shared__ uint32_t tv[PAIRS ? kTiny : 1][PAIRS ? 256 : 1];
  const uint64_t B = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = B < n_buckets;
  // the segments this block's buckets fall in: one search per bound, then
  // each thread searches that short window
  __shared__ uint32_t s_win[2];
  {
    const uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x;
    if (threadIdx.x == 0) s_win[0] = upper_bound_dev(bucket_base, S + 1, b0) - 1;
    if (threadIdx.x == 32)
      s_win[1] = upper_bound_dev(bucket_base, S + 1, min(b0 + blockDim.x, n_buckets) - 1);
  }
  __syncthreads();
  uint32_t s = 0, size = 0;
  uint64_t off = 0;  // start of the bucket, also when empty (records stay ordered)
  bool v = false;
  if (in) {
    s = s_win[0] + upper_bound_dev(bucket_base + s_win[0], s_win[1] - s_win[0] + 1, B) - 1;
    const Seg& sg = segs[s];
    off = sg.off;
    if (sg.status == SEG_BUCKET && sg.b2 == 0) {
      // bucket j is pass-1 digit j (positions kept by the pass-2 copy)
      const uint32_t j = (uint32_t)(B - sg.bucket_base);
      const uint32_t base = cmat1[sg.cbase1];
      const uint32_t a = cmat1[sg.cbase1 + (uint64_t)j * sg.tiles1] - base;
      const uint32_t b = (j + 1 < (1u << sg.b1)) ? cmat1[sg.cbase1 + (uint64_t)(j + 1) * sg.tiles1] - base
                                                 : (uint32_t)sg.n;
      size = b - a;
      off = sg.off + a;
    } else if (sg.status == SEG_BUCKET) {
      const uint32_t j = (uint32_t)(B - sg.bucket_base);
      const uint32_t g = j >> sg.b2, d = j & ((1u << sg.b2) - 1u);
      const Group gr = groups[sg.group_base + g];
      off = gr.off;
      if (gr.n > 0) {
        const uint32_t gbase = cmat2[gr.cbase];
        const uint32_t a = cmat2[gr.cbase + (uint64_t)d * gr.tiles] - gbase;
        const uint32_t b = (d + 1 < (1u << sg.b2))
                               ? cmat2[gr.cbase + (uint64_t)(d + 1) * gr.tiles] - gbase
                               : gr.n;
        size = b - a;
        off = gr.off + a;
      }
    }
    v = sg.status == SEG_BUCKET && size > 0;
  }
  const Seg* sg = v ? &segs[s] : nullptr;
  // Alg. 1's failure guard, counted per warp (the decision record)
  {
    const bool guard = v && size >= sg->delta;
    const uint32_t gb = __ballot_sync(~0u, guard);
    const uint32_t gk = __reduce_add_sync(~0u, guard ? size : 0u);
    if (gb && (threadIdx.x & 31) == 0) {
      atomicAdd(&pcf_counters(status)->guard_buckets, (unsigned long long)__popc(gb));
      atomicAdd(&pcf_counters(status)->guard_keys, (unsigned long long)gk);
    }
  }
  // A run of small leaf buckets (block-local leaf sort only): when this
  // warp's 32 buckets belong to one bucketed (sub)array and each of them is
  // a leaf of at most kRunBucket keys, they are listed as one leaf record of
  // their total size.  Buckets are ordered (every key of bucket j precedes
  // every key of bucket j + 1, Sec. 3.2), so the run sorted as one piece is
  // the buckets sorted one after another.
  bool run = false;
  uint32_t run_n = 0;
  if (leaf_lists) {
    const uint32_t s0 = __shfl_sync(~0u, s, 0);
    const bool small = in && s == s0 && segs[s].status == SEG_BUCKET && size <= kRunBucket &&
                       size <= leaf_cap &&
                       !(size >= segs[s].delta && size > guard_leaf_max(leaf_cap, true));
    run_n = __reduce_add_sync(~0u, in ? size : 0u);
    run = __all_sync(~0u, small) && run_n <= leaf_cap;
  }
  // Standard-Sort (|c| >= delta, or |c| < tau inside the recursive call) of a
  // tiny bucket: insertion sort by this thread, X -> out
  const bool std_sort = v && (size >= sg->delta || size < tau);
  if (std_sort && size <= kTiny && !run) {
    const uint32_t t = threadIdx.x;
    for (uint32_t i = 0; i < size; ++i) {
      const uint64_t key = X[off + i];
      const uint64_t ok = ord_of(key, kt);
      const uint32_t val = PAIRS ? Xv[off + i] : 0u;
      uint32_t q = i;
      while (q > 0 && ord_of(tk[q - 1][t], kt) > ok) {
        tk[q][t] = tk[q - 1][t];
        if (PAIRS) tv[q][t] = tv[q - 1][t];
        --q;
      }
      tk[q][t] = key;
      if (PAIRS) tv[q][t] = val;
    }
    for (uint32_t i = 0; i < size; ++i) {
      if (!PCF_IN_KEYS(off + i, status)) break;
      out_k[off + i] = tk[i][t];
      if (PAIRS) out_v[off + i] = tv[i][t];
    }
    v = false;
  }
  // a failure-guard bucket is sorted on chip only up to guard_leaf_max keys
  // (leaf_cap for the block-local sort, else kStdLeafMax: one warp runs the
  // Standard-Sort); larger ones go to the fallback
  const bool is_fb =
      v && size >= sg->delta && size > guard_leaf_max(leaf_cap, leaf_lists != nullptr);
  const bool is_leaf = v && !is_fb && size <= leaf_cap;
  const bool is_next = v && !is_fb && !is_leaf;
  // the records are read for next-level buckets (the planner, k_mid) and,
  // without the block-local sort's lists, for the on-chip kernels' lists
  if (in && (is_next || !leaf_lists)) {
    BRec r;
    r.off = (uint32_t)off;
    r.n = size;
    r.kind = is_leaf && !run ? (BK_LEAF | (std_sort ? BK_STD : 0u)) : 0u;
    r.depth = sg ? sg->depth + 1 : 0u;
    r.start = sg ? sg->start + (off - sg->off) : 0ull;
    r.seed = sg ? sg->seed : 0ull;
    brec[B] = r;
  }
  // a next-level bucket of at most kMidCap keys goes to k_mid first (its
  // flag stays clear unless k_mid leaves it to the next level)
  const bool is_mid = is_next && mid_list && size <= kMidCap;
  if (in) next_flag[B] = is_next && !is_mid ? 1u : 0u;
  if (mid_list) {
    const uint32_t i_mid = warp_append(mid_count, is_mid);
    if (is_mid) mid_list[i_mid] = (uint32_t)B;
  }
  warp_append(&lo->n_flag, is_next && !is_mid);
  const uint32_t i_leaf = warp_append(&lo->n_leaf, is_leaf);
  (void)i_leaf;
  // the block-local sort's class lists, (offset, size) per leaf bucket, or
  // one record per run (lane 0: the run's first offset and its size)
  if (leaf_lists) {
    const bool lane0 = (threadIdx.x & 31) == 0;
    const uint32_t ln = run ? run_n : size;
    const uint32_t cls = (run ? lane0 && run_n > 0 : is_leaf)
                             ? min(leaf_size_class(ln), leaf_classes - 1)
                             : kMaxLeafClasses;
#pragma unroll
    for (uint32_t k = 0; k < kMaxLeafClasses; ++k) {
      const uint32_t bal = __ballot_sync(~0u, cls == k);
      if (!bal) continue;
      const int leader = __ffs(bal) - 1;
      uint32_t base = 0;
      if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&leaf_counts[k], (uint32_t)__popc(bal));
      base = __shfl_sync(~0u, base, leader);
      if (cls == k)
        leaf_lists[(size_t)k * n_buckets + base + __popc(bal & lanemask_lt())] =
            make_uint2((uint32_t)off, ln);
    }
  }
  const uint32_t i_next = warp_append(&lo->n_next, is_next);
  (void)i_next;
  const uint32_t i_fb = warp_append(&lo->n_fb, is_fb);
  if (is_fb) {
    if (i_fb < max_items) {
      fb[i_fb].off = off;
      fb[i_fb].n = size;
      atomicMax(&lo->max_fb_n, size);
    } else {
      atomicOr(status, STATUS_INTERNAL);
    }
  }
}

// ---------------------------------------------------------------------------
// Device-side plan of the next level.  Every bucket flagged "next" (larger
// than the on-chip kernel takes, below delta) is one Learned-Sort call of the
// next level (Alg. 1).  An exclusive scan of the flags numbers them in bucket
// order, which is memory order, so the next level's (sub)arrays need no sort;
// a thread per flagged bucket writes its Seg and its per-segment counts, and
// a column scan of the counts gives every base the level's kernels read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bits_of_dev(uint32_t v) { return v ? 32u - __clz(v) : 0u; }

__global__ void k_plan_gate(LevelOut* lo, uint64_t n_buckets, uint64_t* n_flagged,
                            const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  lo->flag_n = lo->n_flag ? n_buckets : 0ull;
  *n_flagged = 0ull;
}

__global__ void k_next_segs(const BRec* __restrict__ brec, const uint32_t* __restrict__ pos,
                            const uint64_t* __restrict__ n_flagged, uint64_t n_buckets, Policy P,
                            uint32_t dbits, uint32_t tile_keys, Seg* nsegs, uint32_t* cols,
                            uint32_t s_max, LevelOut* lo, uint32_t* status) {
  if (pcf_aborted(status)) return;
  const uint64_t B = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= n_buckets || *n_flagged == 0) return;
  const uint32_t s = pos[B];
  const uint32_t s_end = B + 1 < n_buckets ? pos[B + 1] : (uint32_t)*n_flagged;
  if (s_end == s) return;
  if (s >= s_max) {
    atomicOr(status, STATUS_INTERNAL);
    return;
  }
  const BRec r = brec[B];
  Seg g;
  memset(&g, 0, sizeof g);
  g.off = r.off;
  g.n = r.n;
  g.start = r.start;
  g.seed = r.seed;
  g.depth = r.depth;
  const Params pr = params_of(P, r.n);
  g.alpha = pr.alpha;
  g.beta = pr.beta;
  g.gamma = pr.gamma;
  g.delta = pr.delta;
  // bucket-id digits as on the host: one digit when it fits, else the low
  // digit as wide as allowed
  const uint32_t jb = max(1u, bits_of_dev(pr.gamma));
  uint32_t b1 = jb;
  if (jb > dbits) {
    const uint32_t b2 = min(dbits, jb - 1);
    b1 = min(jb - b2, kMaxDigitBits);
    atomicOr(&lo->plan.two_pass, 1u);
  }
  g.b1 = b1;
  g.b2 = jb - b1;
  g.tiles1 = (uint32_t)((r.n + tile_keys - 1) / tile_keys);
  g.ord_lo = ~0ull;
  g.ord_hi = 0;
  g.status = SEG_BUCKET;
  nsegs[s] = g;
  const uint32_t ng = g.b2 ? (1u << g.b1) : 1u;
  cols[PC_RANGE * s_max + s] = (r.n + kRangeTile - 1) / kRangeTile;
  cols[PC_K1 * s_max + s] = (pr.alpha + kSamplesPerCta - 1) / kSamplesPerCta;
  cols[PC_TILES1 * s_max + s] = g.tiles1;
  cols[PC_GROUPS * s_max + s] = ng;
  cols[PC_BUCKETS * s_max + s] = pr.gamma + 1;
  cols[PC_TPOOL * s_max + s] = pr.beta + 1;
  cols[PC_CMAT1 * s_max + s] = g.tiles1 << g.b1;
  cols[PC_CMAT2 * s_max + s] = (g.tiles1 + ng) << g.b2;
  cols[PC_TILES2 * s_max + s] = g.tiles1 + ng;
  atomicMax(&lo->plan.dmax1, 1u << g.b1);
  atomicMax(&lo->plan.dmax2, 1u << g.b2);
  atomicAdd((unsigned long long*)&lo->plan.n_keys, (unsigned long long)r.n);
}

// Exclusive scan of the PC_NCOL count columns over the S rows: per-block
// sums, a scan of the block sums, then the rows.
constexpr uint32_t kColRows = 2048;

__global__ void __launch_bounds__(256) k_cols_reduce(const uint32_t* __restrict__ cols,
                                                     uint32_t s_max, const uint64_t* n_rows,
                                                     uint32_t* block_sums, uint32_t n_blocks,
                                                     const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t S = (uint32_t)(*n_rows < s_max ? *n_rows : (uint64_t)s_max);
  const uint32_t r0 = blockIdx.x * kColRows, r1 = min(S, r0 + kColRows);
  __shared__ uint32_t sh8[8];
  for (uint32_t c = 0; c < PC_NCOL; ++c) {
    uint32_t sum = 0;
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += 256) sum += cols[c * s_max + r];
    uint32_t tot;
    block_excl_scan256(sum, sh8, &tot);
    if (threadIdx.x == 0) block_sums[c * n_blocks + blockIdx.x] = tot;
  }
}

// One warp per column scans the block sums (exclusive, in place); the
// totals and the end entries [S] of the base arrays are written here.
__global__ void __launch_bounds__(32 * PC_NCOL) k_cols_scan(uint32_t* block_sums,
                                                            uint32_t n_blocks,
                                                            const uint64_t* n_rows,
                                                            uint32_t s_max, const Seg* nsegs,
                                                            DevPlan dp, LevelOut* lo,
                                                            const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t S = (uint32_t)(*n_rows < s_max ? *n_rows : (uint64_t)s_max);
  uint64_t carry = 0;
  for (uint32_t b0 = 0; b0 < n_blocks; b0 += 32) {
    const uint32_t b = b0 + lane;
    const uint32_t v = b < n_blocks ? block_sums[c * n_blocks + b] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(~0u, inc, d);
      if (lane >= (uint32_t)d) inc += u;
    }
    if (b < n_blocks) block_sums[c * n_blocks + b] = (uint32_t)carry + inc - v;
    carry += __shfl_sync(~0u, inc, 31);
  }
  if (lane != 0) return;
  lo->plan.col[c] = carry;
  if (c == PC_RANGE) dp.rb[S] = (uint32_t)carry;
  if (c == PC_K1) dp.k1[S] = (uint32_t)carry;
  if (c == PC_TILES1) dp.t1[S] = (uint32_t)carry;
  if (c == PC_GROUPS) dp.gb[S] = carry;
  if (c == PC_BUCKETS) dp.bb[S] = carry;
  if (c == 0) {
    lo->plan.S = S;
    lo->plan.lo = S ? nsegs[0].off : 0;
    lo->plan.hi = S ? nsegs[S - 1].off + nsegs[S - 1].n : 0;
  }
}

__global__ void __launch_bounds__(256) k_cols_apply(const uint32_t* __restrict__ cols,
                                                    uint32_t s_max, const uint64_t* n_rows,
                                                    const uint32_t* __restrict__ block_sums,
                                                    uint32_t n_blocks, DevPlan dp,
                                                    const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t S = (uint32_t)(*n_rows < s_max ? *n_rows : (uint64_t)s_max);
  const uint32_t r0 = blockIdx.x * kColRows, r1 = min(S, r0 + kColRows);
  __shared__ uint32_t sh8[8];
  constexpr uint32_t kPer = kColRows / 256;  // rows per thread, consecutive
  for (uint32_t c = 0; c < PC_TILES2; ++c) {
    if (c == PC_CMAT2) continue;
    uint32_t v[kPer], sum = 0;
    const uint32_t rt = r0 + threadIdx.x * kPer;
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      v[i] = rt + i < r1 ? cols[c * s_max + rt + i] : 0u;
      sum += v[i];
    }
    uint32_t tot;
    uint32_t run = block_sums[c * n_blocks + blockIdx.x] + block_excl_scan256(sum, sh8, &tot);
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i) {
      const uint32_t r = rt + i;
      if (r < r1) {
        switch (c) {
          case PC_RANGE: dp.rb[r] = run; break;
          case PC_K1: dp.k1[r] = run; break;
          case PC_TILES1: dp.t1[r] = run; break;
          case PC_GROUPS: dp.gb[r] = run; dp.segs[r].group_base = run; break;
          case PC_BUCKETS: dp.bb[r] = run; dp.segs[r].bucket_base = run; break;
          case PC_TPOOL: dp.segs[r].T_off = run; break;
          case PC_CMAT1: dp.segs[r].cbase1 = run; break;
          default: break;
        }
      }
      run += v[i];
    }
  }
}


// Segments whose range is degenerate go to the standard sort as a whole.
__global__ void k_seg_status_lists(const Seg* segs, uint32_t S, FbItem* fb, LevelOut* lo,
                                   uint32_t max_items, uint32_t* status) {
  if (pcf_aborted(status)) return;
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  if (segs[s].status != SEG_DEGEN) return;
  uint32_t i = atomicAdd(&lo->n_fb, 1u);
  if (i < max_items) {
    fb[i].off = segs[s].off;
    fb[i].n = segs[s].n;
    atomicMax(&lo->max_fb_n, (uint32_t)segs[s].n);
  } else {
    atomicOr(status, STATUS_INTERNAL);
  }
}

// Out-of-place level 0: segments that are not bucketed (one value, or a
// degenerate range) are copied to the output as they are.
__global__ void __launch_bounds__(256) k_copy_segs(const Seg* segs, uint32_t S,
                                                   const uint32_t* range_base,
                                                   const uint64_t* __restrict__ src, uint64_t* dst,
                                                   const uint32_t* __restrict__ src_v,
                                                   uint32_t* dst_v, uint32_t status_mask,
                                                   const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(range_base, S + 1, t) - 1;
  const Seg& g = segs[s];
  const bool sel = (status_mask & kCopyOneDigit) ? (g.status == SEG_BUCKET && g.b2 == 0)
                                                 : ((status_mask >> g.status) & 1u) != 0;
  if (!sel) return;
  const uint64_t base = g.off + (uint64_t)(t - range_base[s]) * kRangeTile;
  const uint64_t end = min(g.off + g.n, base + kRangeTile);
  uint64_t i = base + threadIdx.x;
  for (; i + 3 * 256 < end; i += 4 * 256) {
    const uint64_t a = ld_nc(src + i), b = ld_nc(src + i + 256), c = ld_nc(src + i + 512),
                   d = ld_nc(src + i + 768);
    dst[i] = a;
    dst[i + 256] = b;
    dst[i + 512] = c;
    dst[i + 768] = d;
  }
  for (; i < end; i += 256) dst[i] = src[i];
  if (dst_v)
    for (uint64_t q = base + threadIdx.x; q < end; q += 256) dst_v[q] = src_v[q];
}

// A replayed sort graph's check at the end of a level: the host decisions the
// graph was captured with (the next level's plan, and that no bucket went to
// the standard sort) against what this run's device computed.  Any
// difference sets STATUS_REPLAN, which gates every later kernel; the host
// then sorts the input again without the graph.
__global__ void k_guard(const LevelOut* dev, const LevelOut* rec, uint32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const PlanTotals& a = dev->plan;
  const PlanTotals& b = rec->plan;
  bool same = dev->n_fb == rec->n_fb && dev->max_fb_n == rec->max_fb_n && a.n_keys == b.n_keys &&
              a.lo == b.lo && a.hi == b.hi && a.S == b.S && a.dmax1 == b.dmax1 &&
              a.dmax2 == b.dmax2 && a.two_pass == b.two_pass;
  for (int k = 0; k < PC_NCOL; ++k) same = same && a.col[k] == b.col[k];
  if (!same) atomicOr(status, STATUS_REPLAN);
}

// ... and of a level's standard-sort list, which the device builds in any
// order: every one of its n items must be one of the recorded items (kept
// sorted by offset; the items are disjoint, so equal counts and every item
// found make the same set).
__global__ void k_guard_list(const FbItem* dev, const FbItem* rec, uint32_t n, uint32_t* status) {
  if (pcf_aborted(status)) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const FbItem d = dev[i];
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t m = (lo + hi) >> 1;
    if (rec[m].off < d.off) lo = m + 1;
    else hi = m;
  }
  if (lo >= n || rec[lo].off != d.off || rec[lo].n != d.n) atomicOr(status, STATUS_REPLAN);
}

// ... and of a buffer the host read back during the standard sort's rounds
// (ranges, pivots, split decisions, part sizes): word for word.
__global__ void k_guard_words(const uint32_t* dev, const uint32_t* rec, uint64_t n,
                              uint32_t* status) {
  if (pcf_aborted(status)) return;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (dev[i] != rec[i]) {
      atomicOr(status, STATUS_REPLAN);
      return;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_guard_list(const LaunchCfg& c, const FbItem* dev, const FbItem* rec,
                              uint32_t n) {
  if (!n) return cudaSuccess;
  k_guard_list<<<(n + 255) / 256, 256, 0, c.stream>>>(dev, rec, n, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_guard_words(const LaunchCfg& c, const void* dev, const void* rec,
                               uint64_t n_words) {
  if (!n_words) return cudaSuccess;
  const uint64_t blocks = (n_words + 255) / 256;
  const uint32_t grid = (uint32_t)(blocks < 256 ? blocks : 256);
  k_guard_words<<<grid, 256, 0, c.stream>>>((const uint32_t*)dev, (const uint32_t*)rec, n_words,
                                            c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_guard(const LaunchCfg& c, const LevelOut* dev, const LevelOut* rec) {
  k_guard<<<1, 32, 0, c.stream>>>(dev, rec, c.status);
  count_launch(c);
  return cudaGetLastError();
}

static inline uint32_t cdiv(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

cudaError_t launch_range(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* range_base,
                         uint32_t n_tiles, const uint64_t* keys, bool check_nan,
                         uint32_t only_status) {
  if (!n_tiles) return cudaSuccess;
  k_range<<<n_tiles, 256, 0, c.stream>>>(segs, S, range_base, keys, c.kt, check_nan ? 1 : 0,
                                         c.status, only_status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_sample_range(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* k1_base,
                                uint32_t n_ctas, const uint64_t* keys) {
  if (!n_ctas) return cudaSuccess;
  k_sample_range<<<n_ctas, 256, 0, c.stream>>>(segs, S, k1_base, keys, c.kt, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_model(const LaunchCfg& c, Seg* segs, uint32_t S, uint32_t pass) {
  if (!S) return cudaSuccess;
  k_model<<<cdiv(S, 128), 128, 0, c.stream>>>(segs, S, c.kt, c.model, pass, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_sample(const LaunchCfg& c, Seg* segs, uint32_t S, const uint32_t* k1_base,
                          uint32_t n_ctas, const uint64_t* keys, uint32_t* tpool) {
  if (!n_ctas) return cudaSuccess;
  k_sample<<<n_ctas, 256, 0, c.stream>>>(segs, S, k1_base, keys, c.kt, tpool, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_table(const LaunchCfg& c, Seg* segs, uint32_t S, uint32_t* tpool,
                         uint64_t pool_n, uint64_t* status_words, uint32_t* tile_counter,
                         uint64_t spin_limit) {
  cudaError_t e = launch_scan(c, tpool, pool_n, nullptr, status_words, tile_counter, 0xFFFFFFFFu,
                              spin_limit, nullptr, true);
  if (e) return e;
  k_seg_base<<<cdiv(S, 128), 128, 0, c.stream>>>(segs, S, tpool, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_hist1(const LaunchCfg& c, const Seg* segs, uint32_t S, const uint32_t* tile_base,
                         uint32_t n_tiles, uint32_t tile_keys, const uint64_t* keys,
                         const uint32_t* tpool, uint32_t* cmat, uint32_t dmax, uint32_t* jout,
                         bool check_nan) {
  if (!n_tiles) return cudaSuccess;
  k_hist1<<<n_tiles, 256, dmax * 4, c.stream>>>(segs, S, tile_base, tile_keys, keys, c.kt, tpool,
                                                cmat, jout, check_nan ? 1 : 0, c.status);
  count_launch(c);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Level-0 bucket sizes only (the bucketing-failure experiment of Sec. 4.2):
// every key's bucket id j (stored by k_hist1) counted per segment, then the
// largest count of each segment.  Few buckets: a shared-memory histogram per
// tile first (the counters would otherwise be hot); many: global atomics.
// ---------------------------------------------------------------------------
constexpr uint32_t kSizeBinsSmem = 8192;

__global__ void __launch_bounds__(256) k_bucket_sizes(const Seg* segs, uint32_t S,
                                                      const uint32_t* tile_base,
                                                      uint32_t tile_keys,
                                                      const uint32_t* __restrict__ jbuf,
                                                      uint32_t* counts) {
  __shared__ uint32_t h[kSizeBinsSmem];
  const uint32_t t = blockIdx.x;
  const uint32_t s = upper_bound_dev(tile_base, S + 1, t) - 1;
  const Seg& g = segs[s];
  if (g.status != SEG_BUCKET) return;  // uniform across the block
  const uint32_t nb = g.gamma + 1;
  uint32_t* c = counts + g.bucket_base;
  const uint64_t base = g.off + (uint64_t)(t - tile_base[s]) * tile_keys;
  const uint64_t end = min(g.off + g.n, base + tile_keys);
  if (nb <= kSizeBinsSmem) {
    for (uint32_t k = threadIdx.x; k < nb; k += 256) h[k] = 0;
    __syncthreads();
    for (uint64_t i = base + threadIdx.x; i < end; i += 256) atomicAdd(&h[jbuf[i]], 1u);
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nb; k += 256)
      if (h[k]) atomicAdd(&c[k], h[k]);
  } else {
    for (uint64_t i = base + threadIdx.x; i < end; i += 256) atomicAdd(&c[jbuf[i]], 1u);
  }
}

// a block per segment: max_j |c_j|, or n when the segment was not bucketed
__global__ void __launch_bounds__(256) k_bucket_max(const Seg* segs, const uint32_t* counts,
                                                    uint64_t* out) {
  __shared__ uint32_t wm[8];
  const Seg& g = segs[blockIdx.x];
  if (g.status != SEG_BUCKET) {
    if (threadIdx.x == 0) out[blockIdx.x] = g.n;
    return;
  }
  const uint32_t* c = counts + g.bucket_base;
  uint32_t m = 0;
  for (uint32_t k = threadIdx.x; k <= g.gamma; k += 256) m = max(m, c[k]);
  for (int d = 16; d; d >>= 1) m = max(m, __shfl_xor_sync(~0u, m, d));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = max(m, wm[w]);
    out[blockIdx.x] = m;
  }
}

cudaError_t launch_bucket_sizes(const LaunchCfg& c, const Seg* segs, uint32_t S,
                                const uint32_t* tile_base, uint32_t n_tiles, uint32_t tile_keys,
                                const uint32_t* jbuf, uint32_t* counts, uint64_t* out_max) {
  if (n_tiles) {
    k_bucket_sizes<<<n_tiles, 256, 0, c.stream>>>(segs, S, tile_base, tile_keys, jbuf, counts);
    count_launch(c);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
  }
  k_bucket_max<<<S, 256, 0, c.stream>>>(segs, counts, out_max);
  count_launch(c);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Copy bandwidth probe: the same 16-byte, grid-stride, read-once write-once
// access pattern as the passes, over device buffers (a roofline reference
// measured beside the sort; the reported peak stays the pool's measurement).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_copy128(const uint4* __restrict__ src,
                                                 uint4* __restrict__ dst, uint64_t n16) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = t;
  for (; i + 3 * nt < n16; i += 4 * nt) {
    const uint4 a = __ldg(src + i), b = __ldg(src + i + nt), c = __ldg(src + i + 2 * nt),
                d = __ldg(src + i + 3 * nt);
    dst[i] = a;
    dst[i + nt] = b;
    dst[i + 2 * nt] = c;
    dst[i + 3 * nt] = d;
  }
  for (; i < n16; i += nt) dst[i] = __ldg(src + i);
}

cudaError_t launch_copy128(cudaStream_t st, const void* src, void* dst, uint64_t n16,
                           uint32_t grid) {
  if (!n16) return cudaSuccess;
  k_copy128<<<grid, 256, 0, st>>>((const uint4*)src, (uint4*)dst, n16);
  return cudaGetLastError();
}

// Byte copy by the SMs (one side pinned host memory, seen through its
// device pointer): 16-byte words when both ends allow it.
__global__ void k_xfer(uint8_t* __restrict__ dst, const uint8_t* __restrict__ src, size_t n,
                       int wide) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nt = (size_t)gridDim.x * blockDim.x;
  if (wide) {
    const size_t nw = n / 16;
    for (size_t i = t; i < nw; i += nt)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    for (size_t i = nw * 16 + t; i < n; i += nt) dst[i] = src[i];
  } else {
    for (size_t i = t; i < n; i += nt) dst[i] = src[i];
  }
}

cudaError_t launch_xfer(cudaStream_t st, void* dst, const void* src, size_t bytes) {
  if (!bytes) return cudaSuccess;
  const int wide = (((uintptr_t)dst | (uintptr_t)src) & 15) == 0;
  const size_t units = wide ? bytes / 16 + 1 : bytes;
  const size_t blocks = (units + 255) / 256;
  const uint32_t grid = (uint32_t)(blocks < 256 ? blocks : 256);
  k_xfer<<<grid, 256, 0, st>>>((uint8_t*)dst, (const uint8_t*)src, bytes, wide);
  return cudaGetLastError();
}

cudaError_t launch_scan(const LaunchCfg& c, uint32_t* data, uint64_t n, const uint64_t* n_dev,
                        uint64_t* status_words, uint32_t* tile_counter, uint32_t withhold,
                        uint64_t spin_limit, uint64_t* total_out, bool inclusive) {
  if (!n) return cudaSuccess;
  const uint32_t tiles = cdiv(n, kScanTile);
  cudaError_t e = cudaMemsetAsync(status_words, 0, (size_t)tiles * 8, c.stream);
  if (e) return e;
  e = cudaMemsetAsync(tile_counter, 0, 4, c.stream);
  if (e) return e;
  k_scan<<<tiles, 256, 0, c.stream>>>(data, n, n_dev, status_words, tile_counter, withhold,
                                      spin_limit, total_out, c.status, inclusive ? 1 : 0);
  count_launch(c);
  return cudaGetLastError();
}

// The bulk-staged scatters run where two CTAs still fit an SM's shared
// memory (228 KB, 1 KB of it reserved per CTA)
constexpr size_t kBulkSmemMax = 113 * 1024;

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return allow_max_smem((const void*)kernel);
}

cudaError_t launch_scatter1(const LaunchCfg& c, const Seg* segs, uint32_t S,
                            const uint32_t* tile_base, uint32_t n_tiles, uint32_t tile_keys,
                            const KeyBufs& kb, const uint32_t* tpool, const uint32_t* cmat,
                            uint32_t dmax) {
  if (!n_tiles) return cudaSuccess;
  const size_t sm = scatter_smem_bytes(dmax, c.pairs, true);
  cudaError_t e;
  if (c.pairs) {
    if ((e = set_smem(k_scatter1<true>, sm))) return e;
    k_scatter1<true><<<n_tiles, 256, sm, c.stream>>>(segs, S, tile_base, tile_keys, kb, tpool, cmat,
                                                      c.status);
    count_launch(c);
  } else if (scatter_bulk_smem_bytes(dmax, 1) <= kBulkSmemMax) {
    const size_t smb = scatter_bulk_smem_bytes(dmax, 1);
    if ((e = set_smem(k_scatter1_bulk, smb))) return e;
    k_scatter1_bulk<<<n_tiles, 256, smb, c.stream>>>(segs, S, tile_base, tile_keys, kb, cmat,
                                                     c.status);
    count_launch(c);
  } else {
    if ((e = set_smem(k_scatter1<false>, sm))) return e;
    k_scatter1<false><<<n_tiles, 256, sm, c.stream>>>(segs, S, tile_base, tile_keys, kb,
                                                                tpool, cmat, c.status);
    count_launch(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_groups(const LaunchCfg& c, const Seg* segs, uint32_t S,
                          const uint64_t* group_base_dev, uint64_t n_groups, const uint32_t* cmat1,
                          uint32_t tile_keys, Group* groups, uint32_t* g_tiles,
                          uint32_t* g_centries) {
  if (!n_groups) return cudaSuccess;
  k_groups<<<cdiv(n_groups, 256), 256, 0, c.stream>>>(segs, S, group_base_dev, n_groups, cmat1,
                                                      tile_keys, groups, g_tiles, g_centries,
                                                      c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_group_bases(const LaunchCfg& c, Group* groups, uint64_t n_groups,
                               const uint32_t* g_centries_scan) {
  if (!n_groups) return cudaSuccess;
  k_group_bases<<<cdiv(n_groups, 256), 256, 0, c.stream>>>(groups, n_groups, g_centries_scan,
                                                           c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_hist2(const LaunchCfg& c, const Group* groups, uint32_t n_groups,
                         const Seg* segs, const uint32_t* g_tile_scan, const uint64_t* total_tiles,
                         uint32_t n_tiles_bound, uint32_t tile_keys, const uint16_t* aux,
                         uint32_t* cmat2, uint32_t dmax) {
  if (!n_tiles_bound) return cudaSuccess;
  k_hist2<<<n_tiles_bound, 256, dmax * 4, c.stream>>>(groups, n_groups, segs, g_tile_scan,
                                                      total_tiles, tile_keys, aux, cmat2,
                                                      c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_scatter2(const LaunchCfg& c, const Group* groups, uint32_t n_groups,
                            const Seg* segs, const uint32_t* g_tile_scan,
                            const uint64_t* total_tiles, uint32_t n_tiles_bound,
                            uint32_t tile_keys, const KeyBufs& kb, const uint32_t* cmat2,
                            uint32_t dmax) {
  if (!n_tiles_bound) return cudaSuccess;
  const size_t sm = scatter_smem_bytes(dmax, c.pairs, false);
  cudaError_t e;
  if (c.pairs) {
    if ((e = set_smem(k_scatter2<true>, sm))) return e;
    k_scatter2<true><<<n_tiles_bound, 256, sm, c.stream>>>(groups, n_groups, segs, g_tile_scan,
                                                           total_tiles, tile_keys, kb, cmat2,
                                                           c.status);
    count_launch(c);
  } else if (scatter_bulk_smem_bytes(dmax, 2) <= kBulkSmemMax) {
    const size_t smb = scatter_bulk_smem_bytes(dmax, 2);
    if ((e = set_smem(k_scatter2_bulk, smb))) return e;
    k_scatter2_bulk<<<n_tiles_bound, 256, smb, c.stream>>>(
        groups, n_groups, segs, g_tile_scan, total_tiles, tile_keys, kb, cmat2, c.status);
    count_launch(c);
  } else {
    if ((e = set_smem(k_scatter2<false>, sm))) return e;
    k_scatter2<false><<<n_tiles_bound, 256, sm, c.stream>>>(
        groups, n_groups, segs, g_tile_scan, total_tiles, tile_keys, kb, cmat2, c.status);
    count_launch(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_buckets(const LaunchCfg& c, const Seg* segs, uint32_t S, uint64_t n_buckets,
                           const uint64_t* bucket_base, const Group* groups, const uint32_t* cmat1,
                           const uint32_t* cmat2, bool two_pass, uint32_t leaf_cap, uint32_t tau,
                           const uint64_t* X, const uint32_t* Xv, uint64_t* out_k, uint32_t* out_v,
                           BRec* brec, uint32_t* next_flag, FbItem* fb, LevelOut* lo,
                           uint32_t max_items, uint2* leaf_lists, uint32_t* leaf_counts,
                           uint32_t leaf_classes, uint32_t* mid_list, uint32_t* mid_count) {
  if (!n_buckets) return cudaSuccess;
  if (c.pairs)
    k_buckets<true><<<cdiv(n_buckets, 256), 256, 0, c.stream>>>(
        segs, S, n_buckets, bucket_base, groups, cmat1, cmat2, two_pass ? 1 : 0, leaf_cap, tau,
        c.kt, X, Xv, out_k, out_v, brec, next_flag, fb, lo, max_items, nullptr, nullptr, 0,
        nullptr, nullptr, c.status);
  else
    k_buckets<false><<<cdiv(n_buckets, 256), 256, 0, c.stream>>>(
        segs, S, n_buckets, bucket_base, groups, cmat1, cmat2, two_pass ? 1 : 0, leaf_cap, tau,
        c.kt, X, Xv, out_k, out_v, brec, next_flag, fb, lo, max_items, leaf_lists, leaf_counts,
        leaf_classes, leaf_lists ? mid_list : nullptr, mid_count, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_seg_status_lists(const LaunchCfg& c, const Seg* segs, uint32_t S, FbItem* fb,
                                    LevelOut* lo, uint32_t max_items) {
  if (!S) return cudaSuccess;
  k_seg_status_lists<<<cdiv(S, 128), 128, 0, c.stream>>>(segs, S, fb, lo, max_items, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_copy_segs(const LaunchCfg& c, const Seg* segs, uint32_t S,
                             const uint32_t* range_base, uint32_t n_tiles, const uint64_t* src,
                             uint64_t* dst, const uint32_t* src_v, uint32_t* dst_v,
                             uint32_t status_mask) {
  if (!n_tiles) return cudaSuccess;
  k_copy_segs<<<n_tiles, 256, 0, c.stream>>>(segs, S, range_base, src, dst, src_v, dst_v,
                                             status_mask, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_plan_next(const LaunchCfg& c, const BRec* brec, uint32_t* next_flag,
                             uint64_t n_buckets, uint32_t s_max, Policy P, uint32_t dbits,
                             uint32_t tile_keys, const DevPlan& out, uint32_t* cols,
                             uint32_t* block_sums, LevelOut* lo, uint64_t* sw,
                             uint32_t* tile_counter, uint64_t spin_limit, uint64_t* n_flagged) {
  if (!n_buckets) return cudaSuccess;
  // no bucket flagged (every one finished this level): the flag scan takes
  // no tiles and the next level's plan stays empty
  k_plan_gate<<<1, 1, 0, c.stream>>>(lo, n_buckets, n_flagged, c.status);
  count_launch(c);
  cudaError_t e = launch_scan(c, next_flag, n_buckets, &lo->flag_n, sw, tile_counter,
                              0xFFFFFFFFu, spin_limit, n_flagged);
  if (e) return e;
  k_next_segs<<<cdiv(n_buckets, 256), 256, 0, c.stream>>>(brec, next_flag, n_flagged, n_buckets,
                                                          P, dbits, tile_keys, out.segs, cols,
                                                          s_max, lo, c.status);
  count_launch(c);
  const uint32_t nb = cdiv(s_max, kColRows);
  k_cols_reduce<<<nb, 256, 0, c.stream>>>(cols, s_max, n_flagged, block_sums, nb, c.status);
  count_launch(c);
  k_cols_scan<<<1, 32 * PC_NCOL, 0, c.stream>>>(block_sums, nb, n_flagged, s_max, out.segs, out, lo,
                                                c.status);
  count_launch(c);
  k_cols_apply<<<nb, 256, 0, c.stream>>>(cols, s_max, n_flagged, block_sums, nb, out, c.status);
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace pcf

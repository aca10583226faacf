// pcf_fallback.cu -- the standard sort of buckets too large for the
// on-chip kernels: |c| >= delta (Algorithm 1's failure guard, Sato & Matsui,
// TMLR 2025) or a degenerate range.  A stable merge sort: block-local sorted
// runs of kMergeTile keys, then merge passes split by merge-path
// partitioning, one CTA per kMergeTile outputs.  Before it, a bucket that
// one value dominates is split stably into below / equal / above that value
// (k_fb_mode, k_fb_part_count, k_fb_part_scatter; the host driver runs the
// rounds).
#include "pcf_internal.h"

namespace pcf {

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

// exclusive scan of one u64 per thread over a 256-thread block
__device__ __forceinline__ uint64_t block_excl_scan256_u64(uint64_t v, uint64_t* sh8,
                                                          uint64_t* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t u = (uint64_t)__shfl_up_sync(~0u, (unsigned long long)inc, d);
    if (l >= d) inc += u;
  }
  if (l == 31) sh8[w] = inc;
  __syncthreads();
  uint64_t wsum = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t x = sh8[k];
    if (k < w) wsum += x;
    tot += x;
  }
  __syncthreads();
  *total = tot;
  return wsum + inc - v;
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


// ---------------------------------------------------------------------------
// Fallback standard sort of large buckets: stable merge sort
// ---------------------------------------------------------------------------
// per item range -> ord_lohi[2i], [2i+1]; tiles of kRangeTile
__global__ void __launch_bounds__(256) k_fb_range(const FbItem* items, uint32_t n_items,
                                                  const uint32_t* tile_base,
                                                  const uint64_t* __restrict__ keys, uint32_t kt,
                                                  uint64_t* ord_lohi,
                                                  const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
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
                                                       uint32_t* vals, uint32_t kt,
                                                       const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
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
                                                  uint32_t* dst_v, uint32_t kt,
                                                  const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
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

// copy tmp -> out for items that were merged an odd number of times (with
// ord_lohi null: every item, src -> dst)
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_fb_copy(const FbItem* items, uint32_t n_items,
                                                 const uint32_t* tile_base,
                                                 const uint64_t* ord_lohi, const uint64_t* src,
                                                 uint64_t* dst, const uint32_t* src_v,
                                                 uint32_t* dst_v, const uint64_t* orig,
                                                 const uint32_t* orig_v,
                                                 const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  const uint32_t t = blockIdx.x;
  const uint32_t i = ub_dev(tile_base, n_items + 1, t) - 1;
  if (ord_lohi && ord_lohi[2 * i] == ord_lohi[2 * i + 1]) {  // never moved: copy from there
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
// Duplicate-heavy items.  The standard sort may be any sort (Sec. 3.1); an
// item that one value dominates is first split stably three ways around it
// (as in three-way partitioning quicksort): the equal part is final, and
// the parts below and above go round again.
// ---------------------------------------------------------------------------
// a CTA per item: kModeSample evenly spaced keys, the most frequent of them
__global__ void __launch_bounds__(kModeSample) k_fb_mode(const FbItem* items, uint32_t n_items,
                                                         const uint64_t* __restrict__ keys,
                                                         uint32_t kt,
                                                         const uint64_t* ord_lohi,
                                                         uint64_t* pivot, uint32_t* dom,
                                                         const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  __shared__ uint64_t s[kModeSample];
  __shared__ uint32_t best_c[kModeSample / 32];
  __shared__ uint64_t best_v[kModeSample / 32];
  const uint32_t i = blockIdx.x, t = threadIdx.x;
  if (i >= n_items) return;
  const FbItem it = items[i];
  if (it.n < 2 || ord_lohi[2 * i] == ord_lohi[2 * i + 1]) {  // one value: nothing to split
    if (t == 0) {
      dom[i] = 0;
      pivot[i] = 0;  // defined, so that a replayed sort graph can compare it
    }
    return;
  }
  s[t] = ord_of(__ldg(keys + it.off + (uint64_t)t * it.n / kModeSample), kt);
  __syncthreads();
  const uint64_t v = s[t];
  uint32_t cnt = 0;
  for (uint32_t j = 0; j < kModeSample; ++j) cnt += s[j] == v ? 1u : 0u;
  uint64_t bv = v;
  uint32_t bc = cnt;
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    const uint32_t oc = __shfl_xor_sync(~0u, bc, d);
    const uint64_t ov = (uint64_t)__shfl_xor_sync(~0u, (unsigned long long)bv, d);
    if (oc > bc || (oc == bc && ov < bv)) {
      bc = oc;
      bv = ov;
    }
  }
  if ((t & 31) == 0) {
    best_c[t >> 5] = bc;
    best_v[t >> 5] = bv;
  }
  __syncthreads();
  if (t == 0) {
    for (uint32_t w = 1; w < kModeSample / 32; ++w)
      if (best_c[w] > bc || (best_c[w] == bc && best_v[w] < bv)) {
        bc = best_c[w];
        bv = best_v[w];
      }
    dom[i] = bc >= kModeSample / 4 ? 1u : 0u;
    pivot[i] = bv;
  }
}

__device__ __forceinline__ uint32_t fb_item_of(const uint32_t* mtile_base, uint32_t n_items,
                                               uint32_t t) {
  return ub_dev(mtile_base, n_items + 1, t) - 1;
}

// per tile: keys below, equal to and above the item's pivot
__global__ void __launch_bounds__(256) k_fb_part_count(const FbItem* items, uint32_t n_items,
                                                       const uint32_t* mtile_base,
                                                       uint32_t n_mtiles,
                                                       const uint64_t* __restrict__ keys,
                                                       uint32_t kt, const uint64_t* pivot,
                                                       uint32_t* cnt,
                                                       unsigned long long* item_cnt,
                                                       const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  __shared__ uint32_t s3[3];
  const uint32_t t = blockIdx.x;
  const uint32_t i = fb_item_of(mtile_base, n_items, t);
  const FbItem it = items[i];
  const uint64_t a = (uint64_t)(t - mtile_base[i]) * kMergeTile;
  const uint32_t m = (uint32_t)min((uint64_t)kMergeTile, it.n - a);
  const uint64_t pv = pivot[i];
  if (threadIdx.x < 3) s3[threadIdx.x] = 0;
  __syncthreads();
  uint32_t lt = 0, eq = 0;
  for (uint32_t q = threadIdx.x; q < m; q += 256) {
    const uint64_t o = ord_of(__ldg(keys + it.off + a + q), kt);
    lt += o < pv ? 1u : 0u;
    eq += o == pv ? 1u : 0u;
  }
  atomicAdd(&s3[0], lt);
  atomicAdd(&s3[1], eq);
  __syncthreads();
  if (threadIdx.x == 0) {
    cnt[t] = s3[0];
    cnt[(n_mtiles + 1) + t] = s3[1];
    cnt[2 * (n_mtiles + 1) + t] = m - s3[0] - s3[1];
    atomicAdd(&item_cnt[3 * i], (unsigned long long)s3[0]);
    atomicAdd(&item_cnt[3 * i + 1], (unsigned long long)s3[1]);
    atomicAdd(&item_cnt[3 * i + 2], (unsigned long long)(m - s3[0] - s3[1]));
    if (t == 0) {  // the zero last column, scanned into the totals
      cnt[n_mtiles] = 0;
      cnt[(n_mtiles + 1) + n_mtiles] = 0;
      cnt[2 * (n_mtiles + 1) + n_mtiles] = 0;
    }
  }
}

// per tile: each thread takes 8 consecutive keys, so that one exclusive scan
// of the packed (below, equal, above) counts gives stable positions
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_fb_part_scatter(const FbItem* items, uint32_t n_items,
                                                         const uint32_t* mtile_base,
                                                         uint32_t n_mtiles,
                                                         const uint64_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ vals,
                                                         uint32_t kt, const uint64_t* pivot,
                                                         const uint32_t* cnt_ex, uint64_t* dst,
                                                         uint32_t* dst_v,
                                                         const uint32_t* gate) {
  if (pcf_aborted(gate)) return;
  static_assert(kMergeTile == 256 * 8, "one tile is 256 threads x 8 keys");
  __shared__ uint64_t sh8[8];
  const uint32_t t = blockIdx.x;
  const uint32_t i = fb_item_of(mtile_base, n_items, t);
  const FbItem it = items[i];
  const uint64_t a = (uint64_t)(t - mtile_base[i]) * kMergeTile;
  const uint32_t m = (uint32_t)min((uint64_t)kMergeTile, it.n - a);
  const uint64_t pv = pivot[i];
  const uint32_t t0 = mtile_base[i], t1 = mtile_base[i + 1];
  const uint32_t* lt_ex = cnt_ex;
  const uint32_t* eq_ex = cnt_ex + (n_mtiles + 1);
  const uint32_t* gt_ex = cnt_ex + 2 * (n_mtiles + 1);
  const uint64_t n_lt = lt_ex[t1] - lt_ex[t0], n_eq = eq_ex[t1] - eq_ex[t0];
  // where this tile's keys of each part start within the item
  const uint64_t base_lt = lt_ex[t] - lt_ex[t0];
  const uint64_t base_eq = n_lt + (eq_ex[t] - eq_ex[t0]);
  const uint64_t base_gt = n_lt + n_eq + (gt_ex[t] - gt_ex[t0]);
  const uint32_t q0 = threadIdx.x * 8u;
  uint64_t k[8];
  uint32_t v[8], c[8];
  uint64_t packed = 0;  // below | equal << 21 | above << 42
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const uint32_t q = q0 + u;
    c[u] = 3;
    if (q < m) {
      k[u] = keys[it.off + a + q];
      if (PAIRS) v[u] = vals[it.off + a + q];
      const uint64_t o = ord_of(k[u], kt);
      c[u] = o < pv ? 0u : (o == pv ? 1u : 2u);
      packed += 1ull << (21 * c[u]);
    }
  }
  uint64_t tot;
  uint64_t ex = block_excl_scan256_u64(packed, sh8, &tot);
  // next position of each part (register selects: no local-memory arrays)
  uint64_t p_lt = it.off + base_lt + (ex & 0x1FFFFFull);
  uint64_t p_eq = it.off + base_eq + ((ex >> 21) & 0x1FFFFFull);
  uint64_t p_gt = it.off + base_gt + (ex >> 42);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (c[u] < 3) {
      const uint64_t pos = c[u] == 0 ? p_lt++ : (c[u] == 1 ? p_eq++ : p_gt++);
      dst[pos] = k[u];
      if (PAIRS) dst_v[pos] = v[u];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_fb_range(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                            const uint32_t* tile_base, uint32_t n_tiles, const uint64_t* keys,
                            uint64_t* ord_lohi) {
  if (!n_tiles) return cudaSuccess;
  k_fb_range<<<n_tiles, 256, 0, c.stream>>>(items, n_items, tile_base, keys, c.kt, ord_lohi,
                                            c.status);
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
                                                          keys, vals, c.kt, c.status);
  } else {
    k_fb_block_sort<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi,
                                                           keys, vals, c.kt, c.status);
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
                                                       B, Av, Bv, c.kt, c.status);
    } else {
      k_fb_merge<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, w, A,
                                                        B, Av, Bv, c.kt, c.status);
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
                                                      final_k, Av, final_v, keys, vals, c.status);
    } else {
      k_fb_copy<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, ord_lohi, A,
                                                       final_k, nullptr, nullptr, keys, nullptr,
                                                       c.status);
    }
    count_launch(c);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fb_move(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint32_t* mtile_base, uint32_t n_mtiles, const uint64_t* src,
                           uint64_t* dst, const uint32_t* src_v, uint32_t* dst_v) {
  if (!n_mtiles || src == dst) return cudaSuccess;
  if (c.pairs)
    k_fb_copy<true><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, nullptr, src, dst,
                                                    src_v, dst_v, nullptr, nullptr, c.status);
  else
    k_fb_copy<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, nullptr, src,
                                                     dst, nullptr, nullptr, nullptr, nullptr,
                                                     c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_fb_mode(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                           const uint64_t* keys, const uint64_t* ord_lohi, uint64_t* pivot,
                           uint32_t* dom) {
  if (!n_items) return cudaSuccess;
  k_fb_mode<<<n_items, kModeSample, 0, c.stream>>>(items, n_items, keys, c.kt, ord_lohi, pivot,
                                                   dom, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_fb_part_count(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                                 const uint32_t* mtile_base, uint32_t n_mtiles,
                                 const uint64_t* keys, const uint64_t* pivot, uint32_t* cnt,
                                 uint64_t* item_cnt) {
  if (!n_mtiles) return cudaSuccess;
  k_fb_part_count<<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, n_mtiles, keys,
                                                  c.kt, pivot, cnt,
                                                  (unsigned long long*)item_cnt, c.status);
  count_launch(c);
  return cudaGetLastError();
}

cudaError_t launch_fb_part_scatter(const LaunchCfg& c, const FbItem* items, uint32_t n_items,
                                   const uint32_t* mtile_base, uint32_t n_mtiles,
                                   const uint64_t* keys, const uint32_t* vals,
                                   const uint64_t* pivot, const uint32_t* cnt_ex, uint64_t* dst,
                                   uint32_t* dst_v) {
  if (!n_mtiles) return cudaSuccess;
  if (c.pairs)
    k_fb_part_scatter<true><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base, n_mtiles,
                                                            keys, vals, c.kt, pivot, cnt_ex, dst,
                                                            dst_v, c.status);
  else
    k_fb_part_scatter<false><<<n_mtiles, 256, 0, c.stream>>>(items, n_items, mtile_base,
                                                             n_mtiles, keys, vals, c.kt, pivot,
                                                             cnt_ex, dst, dst_v, c.status);
  count_launch(c);
  return cudaGetLastError();
}

}  // namespace pcf

/*
 * pcf_oracle.c -- plain, slow, single-threaded CPU PCF Learned Sort.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the CUDA
 * library.  Only the test suite, the package smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product sort path never calls it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Sato & Matsui, "PCF Learned Sort", TMLR 2025):
 *   Algorithm 1 (Learned-Sort) with the PCF CDF model of Sec. 3.3:
 *     - n < tau                        -> Standard-Sort            (Alg. 1, small bucket)
 *     - x_min, x_max over the (sub)array                            (Sec. 3.3)
 *     - alpha samples a_j from x                                    (Sec. 3.3)
 *     - bin i(x) = floor((x - x_min) beta / (x_max - x_min)) + 1    (Sec. 3.3)
 *     - b_i = |{ j : i(a_j) <= i }|, i = 1..beta+1                  (Sec. 3.3)
 *     - F(x) = b_{i(x)} / alpha                                     (Sec. 3.3)
 *     - bucket j = floor(F(x) gamma) + 1, Append in input order     (Alg. 1)
 *     - |c_j| >= delta -> Standard-Sort, else recurse               (Alg. 1, failure guard)
 *     - alpha = beta = gamma = delta = floor(n^{3/4}), tau = 100     (Thm. pcf nlogn, Sec. 4 setup)
 *
 * Readings of points the paper leaves open (all 0-based here):
 *   R1 floor(n^{p/q}) is the largest integer m with m^q <= n^p, computed in
 *      exact big-integer arithmetic (no pow()).
 *   R2 Samples are drawn uniformly WITH replacement (the Chernoff argument in
 *      the proof of Lemma pcf-divide-success-prob treats them as independent
 *      draws).  Sample j of the sub-array (seed, depth, start, n) is element
 *      floor(r_j * n / 2^64) where r_j is the j-th output of a SplitMix64
 *      stream (Steele, Lea & Flood 2014) whose state is keyed by those four
 *      values; see sample_state() below.
 *   R3 bin(x) = clamp(floor(RN(RN(x - lo) * s)), 0, beta) with
 *      s = RN(beta / RN(hi - lo)): IEEE-754 binary64, round-to-nearest, no
 *      fused multiply-add (build with -ffp-contract=off).  u64 keys use
 *      (double)(x - lo) with exact unsigned subtraction.  0-based bins 0..beta.
 *   R4 A sub-array whose min and max have identical bits is already sorted
 *      (single value; the paper notes such buckets end early, Sec. 4.1).
 *   R5 A range that is zero, not finite, or gives a non-normal scale s goes
 *      to Standard-Sort (the bin formula is undefined there).
 *   R6 Bucket id floor(b * gamma / alpha) in exact integer arithmetic.
 *   R7 Standard-Sort = stable merge sort on the IEEE-754 total order
 *      (-0 < +0); u64 keys compare as unsigned.
 *   R8 The fallback test is |c_j| >= delta with the parent's delta (Alg. 1).
 *   R9 NaN keys are rejected (the paper's domain is a subset of the reals).
 *
 * Spline Learned Sort (App. A.5, policy model 1): the same training (b as
 * above); a key in bin k at relative position f in [t_k, t_{k+1}) gets
 * F(x) = (b_{k-1} + f (b_k - b_{k-1})) / alpha with b_{-1} = 0.
 *   R13 In binary64, round-to-nearest, no contraction, in this order:
 *      p = RN(RN(x - lo) * s) (R3's value), k = clamp(floor(p), 0, beta),
 *      f = p - k when 0 < p < beta (exact), else 0;
 *      y = RN(b_{k-1} + RN(f * (b_k - b_{k-1})));
 *      bucket = min(floor(RN(y * g)), gamma) with g = RN(gamma / alpha)
 *      (floor(F gamma) of Alg. 1 with one division per model, not per key).
 *
 * Sample range (policy range_mode 1: a cheaper variant of Sec. 3.3's
 * whole-array range, not one the paper uses):
 *   R14 lo, hi = the minimum and maximum of the alpha sampled keys (R2's
 *      indices).  If they are equal, or R5 finds that range degenerate, the
 *      (sub)array's own range is used instead, with R4 and R5 as usual.  A
 *      key below lo gets bin 0 (and, in the spline, position 0); a key above
 *      hi gets R3's value (RN(x - lo) is then at least RN(hi - lo), so the
 *      clamp at beta keeps bins monotone).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_KEY_F64 0
#define ORC_KEY_U64 1

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NAN 2
#define ORC_ERR_OOM 3

typedef struct {
  uint32_t a_num, b_num, c_num, d_num; /* exponents of alpha, beta, gamma, delta ... */
  uint32_t den;                        /* ... as a_num/den etc.                        */
  uint64_t tau;                        /* small-input threshold                        */
  uint32_t model;                      /* CDF model: 0 PCF (Sec. 3.3), 1 spline (A.5)  */
  uint32_t range_mode;                 /* 0: the (sub)array's range; 1: the sample's (R14) */
} orc_policy;

typedef struct {
  uint64_t max_depth;        /* deepest recursion level reached (0 = top call)   */
  uint64_t n_bucketings;     /* model-based bucketing steps performed            */
  uint64_t n_small;          /* Standard-Sort calls for n < tau                  */
  uint64_t n_fallback;       /* Standard-Sort calls for |c_j| >= delta           */
  uint64_t fallback_keys;    /* keys sorted by those calls                       */
  uint64_t n_single;         /* sub-arrays ended early: one distinct value (R4)  */
  uint64_t n_degenerate;     /* sub-arrays sent to Standard-Sort by R5           */
  uint64_t recursed_violations; /* recursed buckets not smaller than parent delta */
} orc_stats;

/* ------------------------------------------------------------------ */
/* R1: exact floor(n^{p/q})                                            */
/* ------------------------------------------------------------------ */
#define BIG_LIMBS 80 /* 80 x 32 bits: enough for (2^40)^64 */

static void big_set(uint32_t* a, uint64_t v) {
  memset(a, 0, sizeof(uint32_t) * BIG_LIMBS);
  a[0] = (uint32_t)v;
  a[1] = (uint32_t)(v >> 32);
}
/* a *= v (v < 2^32); returns 1 on overflow */
static int big_mul32(uint32_t* a, uint32_t v) {
  uint64_t carry = 0;
  for (int i = 0; i < BIG_LIMBS; ++i) {
    uint64_t t = (uint64_t)a[i] * v + carry;
    a[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return carry != 0;
}
/* a *= v for any 64-bit v: a*v = a*lo + (a*hi) << 32 */
static int big_mul64(uint32_t* a, uint64_t v) {
  uint32_t lo[BIG_LIMBS], hi[BIG_LIMBS];
  memcpy(lo, a, sizeof(lo));
  memcpy(hi, a, sizeof(hi));
  int ov = big_mul32(lo, (uint32_t)v) | big_mul32(hi, (uint32_t)(v >> 32));
  if (hi[BIG_LIMBS - 1]) ov = 1;
  uint64_t carry = 0;
  for (int i = 0; i < BIG_LIMBS; ++i) {
    uint64_t t = (uint64_t)lo[i] + (i > 0 ? hi[i - 1] : 0) + carry;
    a[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return ov | (carry != 0);
}
static int big_cmp(const uint32_t* a, const uint32_t* b) {
  for (int i = BIG_LIMBS - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  }
  return 0;
}
static void big_pow(uint32_t* out, uint64_t base, uint32_t e) {
  big_set(out, 1);
  for (uint32_t i = 0; i < e; ++i) big_mul64(out, base);
}

/* largest m with m^q <= n^p (binary search over [0, n]); requires p <= q */
uint64_t orc_root_floor(uint64_t n, uint32_t p, uint32_t q) {
  if (q == 0 || p == 0) return p == 0 ? 1 : 0;
  uint32_t np[BIG_LIMBS], mq[BIG_LIMBS];
  big_pow(np, n, p);
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo + 1) / 2;
    big_pow(mq, mid, q);
    if (big_cmp(mq, np) <= 0) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* ------------------------------------------------------------------ */
/* R2: sampling                                                         */
/* ------------------------------------------------------------------ */
#define GOLDEN 0x9E3779B97F4A7C15ULL

/* SplitMix64 output function (Steele, Lea & Flood 2014). */
uint64_t orc_splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* State of the sample stream of one sub-array: each key component is
 * folded in by adding it to the previous mix and mixing again. */
uint64_t orc_sample_state(uint64_t seed, uint64_t depth, uint64_t start, uint64_t n) {
  uint64_t h = orc_splitmix64_mix(seed + GOLDEN * (depth + 1));
  h = orc_splitmix64_mix(h + start);
  h = orc_splitmix64_mix(h + n);
  return h;
}

/* j-th element index: r_j = mix(state + (j+1) * GOLDEN) is the j-th output of
 * SplitMix64 started at `state`; index = floor(r_j * n / 2^64). */
uint64_t orc_sample_index(uint64_t state, uint64_t j, uint64_t n) {
  uint64_t r = orc_splitmix64_mix(state + GOLDEN * (j + 1));
  return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

/* ------------------------------------------------------------------ */
/* keys: IEEE-754 total order                                          */
/* ------------------------------------------------------------------ */
static uint64_t ord_key(uint64_t bits, int kt) {
  if (kt == ORC_KEY_U64) return bits;
  /* negative: flip all bits; non-negative: flip the sign bit */
  return (bits >> 63) ? ~bits : (bits | 0x8000000000000000ULL);
}
static double as_double(uint64_t bits) {
  double d;
  memcpy(&d, &bits, sizeof d);
  return d;
}

/* ------------------------------------------------------------------ */
/* R3: the bin function of Sec. 3.3                                    */
/* ------------------------------------------------------------------ */
typedef struct {
  int kt;
  uint64_t lo_bits;
  uint64_t lo_ord; /* lo in the total order: keys below it get bin 0 (R14) */
  double lo; /* f64 keys only */
  double s;  /* beta / range */
  uint64_t beta;
} orc_binfn;

/* Returns 0 and fills f, or 1 when the range is degenerate (R5). */
static int binfn_make(orc_binfn* f, int kt, uint64_t lo_bits, uint64_t hi_bits, uint64_t beta) {
  double r;
  f->kt = kt;
  f->lo_bits = lo_bits;
  f->lo_ord = ord_key(lo_bits, kt);
  f->beta = beta;
  if (kt == ORC_KEY_F64) {
    f->lo = as_double(lo_bits);
    r = as_double(hi_bits) - f->lo;
  } else {
    f->lo = 0.0;
    r = (double)(hi_bits - lo_bits);
  }
  if (!(r > 0.0) || !isfinite(r)) return 1;
  f->s = (double)beta / r;
  if (!isfinite(f->s) || !(f->s >= 2.2250738585072014e-308)) return 1;
  return 0;
}

static uint64_t binfn_eval(const orc_binfn* f, uint64_t xbits) {
  if (ord_key(xbits, f->kt) < f->lo_ord) return 0; /* only with a sample range */
  double d;
  if (f->kt == ORC_KEY_F64) d = as_double(xbits) - f->lo;
  else d = (double)(xbits - f->lo_bits);
  double p = d * f->s;
  if (!(p < (double)f->beta)) return f->beta;
  if (!(p > 0.0)) return 0;
  return (uint64_t)floor(p);
}

/* Exported for the tests: bin of each x in xs under the model built from
 * (lo, hi, beta).  Returns 1 if the range is degenerate. */
int orc_bins(int kt, uint64_t lo_bits, uint64_t hi_bits, uint64_t beta,
             const uint64_t* xs, uint64_t m, uint64_t* out) {
  orc_binfn f;
  if (binfn_make(&f, kt, lo_bits, hi_bits, beta)) return 1;
  for (uint64_t i = 0; i < m; ++i) out[i] = binfn_eval(&f, xs[i]);
  return 0;
}

/* ------------------------------------------------------------------ */
/* R7: Standard-Sort = stable merge sort on the total order             */
/* ------------------------------------------------------------------ */
static void std_sort_rec(uint64_t* k, uint32_t* v, uint64_t* tk, uint32_t* tv, uint64_t n, int kt) {
  if (n <= 16) {
    for (uint64_t i = 1; i < n; ++i) {
      uint64_t key = k[i];
      uint32_t val = v ? v[i] : 0;
      uint64_t ok = ord_key(key, kt);
      uint64_t j = i;
      while (j > 0 && ord_key(k[j - 1], kt) > ok) {
        k[j] = k[j - 1];
        if (v) v[j] = v[j - 1];
        --j;
      }
      k[j] = key;
      if (v) v[j] = val;
    }
    return;
  }
  uint64_t h = n / 2;
  std_sort_rec(k, v, tk, tv, h, kt);
  std_sort_rec(k + h, v ? v + h : NULL, tk, tv, n - h, kt);
  /* merge: take from the left run on ties (stability) */
  memcpy(tk, k, h * sizeof(uint64_t));
  if (v) memcpy(tv, v, h * sizeof(uint32_t));
  uint64_t i = 0, j = h, o = 0;
  while (i < h && j < n) {
    if (ord_key(k[j], kt) < ord_key(tk[i], kt)) {
      k[o] = k[j];
      if (v) v[o] = v[j];
      ++j;
    } else {
      k[o] = tk[i];
      if (v) v[o] = tv[i];
      ++i;
    }
    ++o;
  }
  while (i < h) {
    k[o] = tk[i];
    if (v) v[o] = tv[i];
    ++i;
    ++o;
  }
}

int orc_std_sort(uint64_t* keys, uint32_t* vals, uint64_t n, int kt) {
  if (n < 2) return ORC_OK;
  uint64_t* tk = (uint64_t*)malloc((n / 2 + 1) * sizeof(uint64_t));
  uint32_t* tv = vals ? (uint32_t*)malloc((n / 2 + 1) * sizeof(uint32_t)) : NULL;
  if (!tk || (vals && !tv)) {
    free(tk);
    free(tv);
    return ORC_ERR_OOM;
  }
  std_sort_rec(keys, vals, tk, tv, n, kt);
  free(tk);
  free(tv);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* One model-based bucketing step (Alg. 1 + Sec. 3.3)                 */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t alpha, beta, gamma, delta;
  uint64_t lo_bits, hi_bits;
  int status;           /* 0 bucketed, 1 single value (R4), 2 degenerate (R5) */
  uint64_t* sample_idx; /* alpha                                               */
  uint64_t* b;          /* beta + 1: cumulative counts b[k] = #{bin(a_j) <= k} */
  uint64_t* T;          /* beta + 1: bucket id of bin k                        */
  uint64_t* counts;     /* gamma + 1: bucket sizes                             */
} orc_level;

static void level_free(orc_level* L) {
  free(L->sample_idx);
  free(L->b);
  free(L->T);
  free(L->counts);
  memset(L, 0, sizeof *L);
}

static void policy_params(const orc_policy* P, uint64_t n, orc_level* L) {
  L->alpha = orc_root_floor(n, P->a_num, P->den);
  L->beta = orc_root_floor(n, P->b_num, P->den);
  L->gamma = orc_root_floor(n, P->c_num, P->den);
  L->delta = orc_root_floor(n, P->d_num, P->den);
  if (L->alpha < 1) L->alpha = 1;
  if (L->beta < 1) L->beta = 1;
}

/* Buckets keys[0..n) in place (stable), filling L.  aux/auxv: scratch of n.
 * fixed3: alpha, beta, gamma given (the bucketing-failure experiment of
 * Sec. 4.2), else the policy's (delta is then 0: unused by one step). */
static int bucketize_with(const orc_policy* P, const uint64_t* fixed3, uint32_t model,
                          uint64_t* keys, uint32_t* vals, uint64_t n, int kt, uint64_t seed,
                          uint64_t depth, uint64_t start, orc_level* L, uint64_t* aux,
                          uint32_t* auxv);

static int bucketize(const orc_policy* P, uint64_t* keys, uint32_t* vals, uint64_t n, int kt,
                     uint64_t seed, uint64_t depth, uint64_t start, orc_level* L,
                     uint64_t* aux, uint32_t* auxv) {
  return bucketize_with(P, NULL, P->model, keys, vals, n, kt, seed, depth, start, L, aux, auxv);
}

/* Spline model (App. A.5, R13): the bucket of key x from b (beta + 1). */
static uint64_t spline_bucket(const orc_binfn* f, uint64_t xbits, const uint64_t* b,
                              uint64_t gamma, double g) {
  const double d = f->kt == ORC_KEY_F64 ? as_double(xbits) - f->lo
                                        : (double)(xbits - f->lo_bits);
  const double p = d * f->s;
  uint64_t k;
  double fr;
  if (ord_key(xbits, f->kt) < f->lo_ord) { /* below a sample range (R14) */
    k = 0;
    fr = 0.0;
  } else if (!(p < (double)f->beta)) {
    k = f->beta;
    fr = 0.0;
  } else if (!(p > 0.0)) {
    k = 0;
    fr = 0.0;
  } else {
    k = (uint64_t)floor(p);
    fr = p - (double)k;
  }
  const uint64_t bkm1 = k ? b[k - 1] : 0;
  const double y = (double)bkm1 + fr * (double)(b[k] - bkm1);
  const double z = y * g;
  if (!(z < (double)gamma)) return gamma;
  return z > 0.0 ? (uint64_t)floor(z) : 0;
}

static int bucketize_with(const orc_policy* P, const uint64_t* fixed3, uint32_t model,
                          uint64_t* keys, uint32_t* vals, uint64_t n, int kt, uint64_t seed,
                          uint64_t depth, uint64_t start, orc_level* L, uint64_t* aux,
                          uint32_t* auxv) {
  memset(L, 0, sizeof *L);
  if (fixed3) {
    L->alpha = fixed3[0];
    L->beta = fixed3[1];
    L->gamma = fixed3[2];
    L->delta = 0;
  } else {
    policy_params(P, n, L);
  }
  orc_binfn f;
  uint64_t lo = keys[0], hi = keys[0];
  int have_model = 0;
  if (P && P->range_mode == 1) {
    /* R14: the range of the alpha samples */
    const uint64_t st0 = orc_sample_state(seed, depth, start, n);
    lo = hi = keys[orc_sample_index(st0, 0, n)];
    for (uint64_t j = 1; j < L->alpha; ++j) {
      const uint64_t x = keys[orc_sample_index(st0, j, n)];
      if (ord_key(x, kt) < ord_key(lo, kt)) lo = x;
      if (ord_key(x, kt) > ord_key(hi, kt)) hi = x;
    }
    have_model = lo != hi && !binfn_make(&f, kt, lo, hi, L->beta);
  }
  if (!have_model) {
    /* x_min, x_max over the whole (sub)array, Sec. 3.3 */
    lo = hi = keys[0];
    for (uint64_t i = 1; i < n; ++i) {
      if (ord_key(keys[i], kt) < ord_key(lo, kt)) lo = keys[i];
      if (ord_key(keys[i], kt) > ord_key(hi, kt)) hi = keys[i];
    }
  }
  L->lo_bits = lo;
  L->hi_bits = hi;
  if (!have_model) {
    if (lo == hi) {
      L->status = 1;
      return ORC_OK;
    }
    if (binfn_make(&f, kt, lo, hi, L->beta)) {
      L->status = 2;
      return ORC_OK;
    }
  }
  L->sample_idx = (uint64_t*)malloc(L->alpha * sizeof(uint64_t));
  L->b = (uint64_t*)calloc(L->beta + 1, sizeof(uint64_t));
  L->T = (uint64_t*)malloc((L->beta + 1) * sizeof(uint64_t));
  L->counts = (uint64_t*)calloc(L->gamma + 1, sizeof(uint64_t));
  if (!L->sample_idx || !L->b || !L->T || !L->counts) return ORC_ERR_OOM;

  /* training: sample alpha keys, count them per bin, accumulate */
  uint64_t st = orc_sample_state(seed, depth, start, n);
  for (uint64_t j = 0; j < L->alpha; ++j) {
    uint64_t idx = orc_sample_index(st, j, n);
    L->sample_idx[j] = idx;
    L->b[binfn_eval(&f, keys[idx])] += 1;
  }
  for (uint64_t k = 1; k <= L->beta; ++k) L->b[k] += L->b[k - 1];
  /* bucket of bin k: floor(F gamma) with F = b_k / alpha (R6) */
  for (uint64_t k = 0; k <= L->beta; ++k)
    L->T[k] = (uint64_t)(((unsigned __int128)L->b[k] * L->gamma) / L->alpha);

  /* inference (PCF: the table; spline: interpolated, R13) + Append: a
     stable counting scatter */
  const double g = (double)L->gamma / (double)L->alpha;
  uint64_t* jk = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* pos = (uint64_t*)malloc((L->gamma + 1) * sizeof(uint64_t));
  if (!jk || !pos) {
    free(jk);
    free(pos);
    return ORC_ERR_OOM;
  }
  for (uint64_t i = 0; i < n; ++i) {
    jk[i] = model ? spline_bucket(&f, keys[i], L->b, L->gamma, g) : L->T[binfn_eval(&f, keys[i])];
    L->counts[jk[i]] += 1;
  }
  uint64_t acc = 0;
  for (uint64_t j = 0; j <= L->gamma; ++j) {
    pos[j] = acc;
    acc += L->counts[j];
  }
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t j = jk[i];
    aux[pos[j]] = keys[i];
    if (vals) auxv[pos[j]] = vals[i];
    pos[j] += 1;
  }
  free(pos);
  free(jk);
  memcpy(keys, aux, n * sizeof(uint64_t));
  if (vals) memcpy(vals, auxv, n * sizeof(uint32_t));
  L->status = 0;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned-Sort (Alg. 1)                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_policy* P;
  int kt;
  uint64_t seed;
  uint64_t* aux;
  uint32_t* auxv;
  orc_stats* stats;
} orc_ctx;

static int learned_sort(orc_ctx* C, uint64_t* keys, uint32_t* vals, uint64_t n, uint64_t depth,
                        uint64_t start) {
  if (depth > C->stats->max_depth) C->stats->max_depth = depth;
  if (n < C->P->tau) {
    C->stats->n_small += 1;
    return orc_std_sort(keys, vals, n, C->kt);
  }
  orc_level L;
  int rc = bucketize(C->P, keys, vals, n, C->kt, C->seed, depth, start, &L, C->aux, C->auxv);
  if (rc) {
    level_free(&L);
    return rc;
  }
  if (L.status == 1) {
    C->stats->n_single += 1;
    level_free(&L);
    return ORC_OK;
  }
  if (L.status == 2) {
    C->stats->n_degenerate += 1;
    level_free(&L);
    return orc_std_sort(keys, vals, n, C->kt);
  }
  C->stats->n_bucketings += 1;
  uint64_t off = 0;
  for (uint64_t j = 0; j <= L.gamma && rc == ORC_OK; ++j) {
    uint64_t c = L.counts[j];
    if (c == 0) continue;
    if (c >= L.delta) {
      C->stats->n_fallback += 1;
      C->stats->fallback_keys += c;
      rc = orc_std_sort(keys + off, vals ? vals + off : NULL, c, C->kt);
    } else {
      if (c >= n) C->stats->recursed_violations += 1;
      rc = learned_sort(C, keys + off, vals ? vals + off : NULL, c, depth + 1, start + off);
    }
    off += c;
  }
  level_free(&L);
  return rc;
}

static int has_nan(const uint64_t* keys, uint64_t n, int kt) {
  if (kt != ORC_KEY_F64) return 0;
  for (uint64_t i = 0; i < n; ++i)
    if ((keys[i] & 0x7FFFFFFFFFFFFFFFULL) > 0x7FF0000000000000ULL) return 1;
  return 0;
}

/* Sorts keys (and vals, if non-NULL, stably) in place.  Keys are raw bits:
 * IEEE-754 binary64 for kt = ORC_KEY_F64, unsigned 64-bit for ORC_KEY_U64. */
int orc_sort(uint64_t* keys, uint32_t* vals, uint64_t n, int kt, uint64_t seed,
             const orc_policy* P, orc_stats* stats) {
  orc_stats local;
  if (!stats) stats = &local;
  memset(stats, 0, sizeof *stats);
  if (kt != ORC_KEY_F64 && kt != ORC_KEY_U64) return ORC_ERR_ARG;
  if (!P || P->den == 0 || P->a_num == 0 || P->a_num > P->den || P->b_num > P->den ||
      P->c_num > P->den || P->d_num == 0 || P->d_num >= P->den || P->model > 1 ||
      P->range_mode > 1)
    return ORC_ERR_ARG;
  if (n == 0) return ORC_OK;
  if (!keys) return ORC_ERR_ARG;
  if (has_nan(keys, n, kt)) return ORC_ERR_NAN;
  orc_ctx C;
  C.P = P;
  C.kt = kt;
  C.seed = seed;
  C.stats = stats;
  C.aux = (uint64_t*)malloc(n * sizeof(uint64_t));
  C.auxv = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
  if (!C.aux || (vals && !C.auxv)) {
    free(C.aux);
    free(C.auxv);
    return ORC_ERR_OOM;
  }
  int rc = learned_sort(&C, keys, vals, n, 0, 0);
  free(C.aux);
  free(C.auxv);
  return rc;
}

/* Level-0 intermediates of Learned-Sort on keys[0..n) (which are left
 * bucketed, not sorted): min/max bits, parameters, sample indices, b, T and
 * the bucket sizes.  Arrays must hold alpha, beta+1, beta+1 and gamma+1
 * entries (query the parameters with orc_root_floor first).  Returns the
 * level status through *status (0 bucketed, 1 single value, 2 degenerate). */
int orc_level0(uint64_t* keys, uint32_t* vals, uint64_t n, int kt, uint64_t seed,
               const orc_policy* P, uint64_t* params6, uint64_t* sample_idx, uint64_t* b,
               uint64_t* T, uint64_t* counts, int* status) {
  if (n < 2 || has_nan(keys, n, kt)) return ORC_ERR_ARG;
  uint64_t* aux = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint32_t* auxv = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
  orc_level L;
  int rc = bucketize(P, keys, vals, n, kt, seed, 0, 0, &L, aux, auxv);
  free(aux);
  free(auxv);
  if (rc) {
    level_free(&L);
    return rc;
  }
  params6[0] = L.alpha;
  params6[1] = L.beta;
  params6[2] = L.gamma;
  params6[3] = L.delta;
  params6[4] = L.lo_bits;
  params6[5] = L.hi_bits;
  *status = L.status;
  if (L.status == 0) {
    memcpy(sample_idx, L.sample_idx, L.alpha * sizeof(uint64_t));
    memcpy(b, L.b, (L.beta + 1) * sizeof(uint64_t));
    memcpy(T, L.T, (L.beta + 1) * sizeof(uint64_t));
    memcpy(counts, L.counts, (L.gamma + 1) * sizeof(uint64_t));
  }
  level_free(&L);
  return ORC_OK;
}

/* One model-based bucketing of keys[0..n) with alpha, beta, gamma given
 * (Sec. 4.2: alpha = floor(n^a) ... varied over a grid), the CDF model
 * (0 PCF, 1 spline) and the range (0 the array's, 1 the sample's, R14): the
 * bucket sizes counts[0..gamma] and *status (0 bucketed, 1 single value, 2
 * degenerate).
 * Keys are not modified. */
int orc_bucket_sizes(const uint64_t* keys, uint64_t n, int kt, uint64_t seed, uint64_t alpha,
                     uint64_t beta, uint64_t gamma, uint32_t model, uint32_t range_mode,
                     uint64_t* counts, int* status) {
  if (n < 2 || alpha < 1 || beta < 1 || gamma < 1 || has_nan(keys, n, kt)) return ORC_ERR_ARG;
  uint64_t* k = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* aux = (uint64_t*)malloc(n * sizeof(uint64_t));
  if (!k || !aux) {
    free(k);
    free(aux);
    return ORC_ERR_OOM;
  }
  memcpy(k, keys, n * sizeof(uint64_t));
  const uint64_t fixed3[3] = {alpha, beta, gamma};
  orc_level L;
  orc_policy rp;
  memset(&rp, 0, sizeof rp);
  rp.model = model;
  rp.range_mode = range_mode;
  int rc = bucketize_with(&rp, fixed3, model, k, NULL, n, kt, seed, 0, 0, &L, aux, NULL);
  free(k);
  free(aux);
  if (rc) {
    level_free(&L);
    return rc;
  }
  *status = L.status;
  if (L.status == 0) memcpy(counts, L.counts, (gamma + 1) * sizeof(uint64_t));
  else memset(counts, 0, (gamma + 1) * sizeof(uint64_t));
  level_free(&L);
  return ORC_OK;
}

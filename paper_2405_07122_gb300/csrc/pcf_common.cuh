// pcf_common.cuh -- shared host/device definitions of the PCF Learned Sort
// kernels (Sato & Matsui, "PCF Learned Sort", TMLR 2025).
//
// Everything here is compiled both for sm_103a and for the host (the host
// copies back the C ABI's self-test entry points); none of it is shared
// with the CPU oracle.
//
// Readings of the paper the kernels follow, cited by label in comments:
//   R1  floor(n^{p/q}) is the largest m with m^q <= n^p, in exact integers.
//   R2  the alpha samples are drawn uniformly with replacement, sample j
//       being floor(r_j n / 2^64) for output j of a SplitMix64 stream keyed
//       by (seed, depth, start, n).
//   R3  bin(x) = clamp(floor(RN(RN(x - lo) s)), 0, beta), s = RN(beta / RN(hi
//       - lo)), binary64 round-to-nearest without contraction.
//   R4  a (sub)array whose min and max are the same bits is already sorted.
//   R5  a range that is zero, not finite, or gives a non-normal s goes to
//       Standard-Sort.
//   R6  the bucket id floor(b gamma / alpha) is exact integer arithmetic.
//   R7  Standard-Sort may be any sort: the sorted output is unique.
//   R8  the fallback test is |c| >= delta, with the parent's delta.
//   R9  NaN keys are rejected.
//   R13 spline model (App. A.5): the position inside the bin and the linear
//       interpolation between b_{k-1} and b_k in binary64, in a fixed order.
//   R14 sample range: lo, hi are the min and max of the alpha samples; the
//       (sub)array's own range is used when they are equal or degenerate.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define PCF_HD __host__ __device__ __forceinline__
#else
#define PCF_HD inline
#endif

namespace pcf {

enum : uint32_t { KEY_F64 = 0, KEY_U64 = 1 };

// --------------------------------------------------------------------------
// IEEE-754 total order (keys are raw 64-bit patterns)
// --------------------------------------------------------------------------
// Maps a key to an unsigned integer whose order is the key order: binary64
// keys flip all bits when negative and only the sign bit otherwise, so that
// -inf < ... < -0 < +0 < ... < +inf; u64 keys are their own order.
PCF_HD uint64_t ord_of(uint64_t bits, uint32_t kt) {
  if (kt == KEY_U64) return bits;
  uint64_t m = (uint64_t)((int64_t)bits >> 63) | 0x8000000000000000ull;
  return bits ^ m;
}
PCF_HD uint64_t bits_of_ord(uint64_t ord, uint32_t kt) {
  if (kt == KEY_U64) return ord;
  return (ord >> 63) ? (ord ^ 0x8000000000000000ull) : ~ord;
}
PCF_HD bool is_nan_bits(uint64_t bits) {
  return (bits & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
}

// --------------------------------------------------------------------------
// Sampling (alpha draws with replacement, Sec. 3.3): SplitMix64 stream keyed
// by (seed, depth, start, n); draw j picks element floor(r_j * n / 2^64).
// --------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

PCF_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// SplitMix64 output function (Steele, Lea & Flood 2014).
PCF_HD uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
PCF_HD uint64_t sample_state(uint64_t seed, uint64_t depth, uint64_t start, uint64_t n) {
  uint64_t h = splitmix_mix(seed + kGolden * (depth + 1));
  h = splitmix_mix(h + start);
  return splitmix_mix(h + n);
}
PCF_HD uint64_t sample_index(uint64_t state, uint64_t j, uint64_t n) {
  return mulhi64(splitmix_mix(state + kGolden * (j + 1)), n);
}

// --------------------------------------------------------------------------
// Parameters: floor(n^{p/q}) exactly (largest m with m^q <= n^p).
// q <= 4 and p <= q, n < 2^32: every power fits in 128 bits.
// --------------------------------------------------------------------------
PCF_HD unsigned __int128 pow_u128(uint64_t b, uint32_t e) {
  unsigned __int128 r = 1;
  for (uint32_t i = 0; i < e; ++i) r *= b;
  return r;
}
PCF_HD uint64_t root_floor(uint64_t n, uint32_t p, uint32_t q) {
  if (p >= q || n < 2) return n;
#ifdef __CUDA_ARCH__
  uint64_t m = (uint64_t)powf((float)n, (float)p / (float)q);
#else
  uint64_t m = (uint64_t)__builtin_powf((float)n, (float)p / (float)q);
#endif
  const unsigned __int128 np = pow_u128(n, p);
  while (m > 0 && pow_u128(m, q) > np) --m;
  while (pow_u128(m + 1, q) <= np) ++m;
  return m;
}

// CDF model of a bucketing step: the PCF of Sec. 3.3, or the piecewise
// linear spline through the same counts (Spline Learned Sort, App. A.5).
enum : uint32_t { MODEL_PCF = 0, MODEL_SPLINE = 1 };

// Range the bins span: the (sub)array's min and max (Sec. 3.3), or the
// alpha samples' (reading R14: one pass fewer per level; keys outside take
// the end bins).
enum : uint32_t { RANGE_ARRAY = 0, RANGE_SAMPLE = 1 };

struct Policy {
  uint32_t a_num, b_num, c_num, d_num, den;
  uint32_t model;  // MODEL_*
  uint64_t tau;
  uint32_t range_mode;  // RANGE_*
  uint32_t pad;
};

struct Params {
  uint32_t alpha, beta, gamma, delta;
};

PCF_HD Params params_of(const Policy& P, uint64_t n) {
  Params r;
  uint64_t a = root_floor(n, P.a_num, P.den), b = root_floor(n, P.b_num, P.den);
  r.alpha = (uint32_t)(a < 1 ? 1 : a);
  r.beta = (uint32_t)(b < 1 ? 1 : b);
  r.gamma = (uint32_t)root_floor(n, P.c_num, P.den);
  r.delta = (uint32_t)root_floor(n, P.d_num, P.den);
  return r;
}

// --------------------------------------------------------------------------
// The bin function of Sec. 3.3, i(x) - 1 = floor((x - x_min) beta / range),
// read in binary64 as   bin(x) = clamp(floor(RN(RN(x - lo) * s)), 0, beta),
// s = RN(beta / RN(hi - lo)),  no fused multiply-add;  u64 keys use
// RN((double)(x - lo)) with an exact unsigned subtraction.
//
// GB300 runs binary64 at ~2 operations/clock/SM, so the kernels evaluate it
// with a certified integer fast path and fall back to the exact binary64
// sequence only when the fast value cannot decide the floor:
//   X(y)  = trunc(y / 2^H), a fixed point of the key on a grid 2^H fine
//           enough that X(hi) - X(lo) lies in [2^61, 2^62); X is computed
//           modulo 2^64 with one shift of the significand, and since trunc
//           is monotone, Dn = X(x) - X(lo) is the exact integer difference
//           in [0, 2^62 + 2) for every key of the range
//   V     = hi64(Dn * Sig)   Sig = 53-bit significand of s shifted left 11
//   V / 2^F approximates v = (x - lo) s.
// Truncation moves Dn by at most 2 (so V by at most 2), hi64 drops less
// than 1, and the two binary64 roundings move the exact result P by at most
// v 2^-52 (1 + 2^-50) <= (beta+1) 2^(F-52) units.  With Eu above all three,
// floor(P) = floor(V / 2^F) whenever [V - Eu, V + Eu] holds no multiple of
// 2^F; otherwise the exact sequence runs.
// --------------------------------------------------------------------------
struct BinModel {
  uint64_t lo_bits;  // raw bits of lo
  double lo_d;       // lo as binary64 (f64 keys)
  double s;          // beta / range
  uint64_t LOw;      // X(lo) modulo 2^64 (f64, mode 0) / lo's 52-bit fraction (modes 1, 2) / lo (u64)
  uint64_t sig;      // significand of s << 11, in [2^63, 2^64)
  uint64_t eu;       // error bound in V units
  int32_t C;         // f64: X(y) shifts the significand by max(e,1) - C
  int32_t w;         // u64: Dn = (x - lo) << w (w < 0: >> -w); f64 modes 1, 2: the shift
  int32_t F;         // fractional bits of V
  uint32_t beta;
  uint32_t kt;
  uint32_t mode;     // f64: 0 general; 1 / 2: lo and hi share sign and exponent (+ / -)
  uint32_t spline;   // 1: the spline model (bucket ids from spline_bucket)
  uint32_t gamma;    // spline: the bucket count - 1 ...
  double g;          // ... and RN(gamma / alpha)
  uint32_t clamp;    // 1: [lo, hi] is the samples' range, keys may lie outside (R14)
  uint32_t pad;
  uint64_t ord_lo, ord_hi;  // clamp: lo and hi in the total order
};

PCF_HD double as_f64(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}
PCF_HD uint64_t f64_bits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  __builtin_memcpy(&b, &d, 8);
  return b;
#endif
}
PCF_HD double dsub(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
PCF_HD double dadd(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
PCF_HD double dmul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
PCF_HD double ddiv(double a, double b) {
#ifdef __CUDA_ARCH__
  return __ddiv_rn(a, b);
#else
  return a / b;
#endif
}
PCF_HD double u64_to_f64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __ull2double_rn((unsigned long long)v);
#else
  return (double)v;
#endif
}
PCF_HD int floor_log2_u64(uint64_t v) {  // v > 0
#ifdef __CUDA_ARCH__
  return 63 - __clzll((long long)v);
#else
  return 63 - __builtin_clzll(v);
#endif
}
PCF_HD bool finite_f64(double d) {
  return (f64_bits(d) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

// X(y) = sign(y) trunc(|y| / 2^(C - 1075)) modulo 2^64.
PCF_HD uint64_t fixed_mod(uint64_t bits, int32_t C) {
  const uint32_t e = (uint32_t)(bits >> 52) & 0x7FFu;
  const uint64_t m = (bits & 0x000FFFFFFFFFFFFFull) | (e ? 0x0010000000000000ull : 0ull);
  const int32_t sh = (int32_t)(e ? e : 1u) - C;
  const uint64_t mag = sh >= 0 ? (sh < 64 ? (m << sh) : 0ull) : (sh > -64 ? (m >> (-sh)) : 0ull);
  return (bits >> 63) ? (0ull - mag) : mag;
}

// v >> F as 32 bits (the quotient never exceeds beta + 1 < 2^32)
PCF_HD uint32_t shr_F(uint64_t v, int32_t F) {
  return F >= 32 ? ((uint32_t)(v >> 32) >> (F - 32)) : (uint32_t)(v >> F);
}

// Builds the model of the range [lo, hi] with beta bins.  Returns 0, or 1
// when the range is degenerate (zero, not finite, or a non-normal scale):
// such (sub)arrays go to the standard sort.
PCF_HD int make_bin_model(uint32_t kt, uint64_t lo_bits, uint64_t hi_bits, uint32_t beta,
                          BinModel* M) {
  M->kt = kt;
  M->beta = beta;
  M->lo_bits = lo_bits;
  M->mode = 0;
  M->spline = 0;
  M->gamma = 0;
  M->g = 0.0;
  M->clamp = 0;
  M->pad = 0;
  M->ord_lo = ord_of(lo_bits, kt);
  M->ord_hi = ord_of(hi_bits, kt);
  double r;
  int32_t H;  // grid exponent: X(y) ~ y / 2^H
  if (kt == KEY_F64) {
    M->lo_d = as_f64(lo_bits);
    r = dsub(as_f64(hi_bits), M->lo_d);
    if (!(r > 0.0) || !finite_f64(r)) return 1;
    // coarse grid 2^G with |X| < 2^62, then refine so the range has 62 bits
    uint32_t elo = (uint32_t)(lo_bits >> 52) & 0x7FFu, ehi = (uint32_t)(hi_bits >> 52) & 0x7FFu;
    uint32_t em = elo > ehi ? elo : ehi;
    if (em < 1) em = 1;
    const int32_t G = (int32_t)em - 1075 - 9;
    const uint64_t coarse = fixed_mod(hi_bits, 1075 + G) - fixed_mod(lo_bits, 1075 + G);
    if (coarse == 0) return 1;  // cannot happen for distinct finite keys
    const int32_t w = 61 - floor_log2_u64(coarse);
    H = G - w;
    M->C = 1075 + H;
    M->w = 0;
    M->LOw = fixed_mod(lo_bits, M->C);
  } else {
    M->lo_d = 0.0;
    const uint64_t range = hi_bits - lo_bits;
    r = u64_to_f64(range);
    if (range == 0) return 1;
    M->w = 61 - floor_log2_u64(range);
    H = -M->w;
    M->C = 0;
    M->LOw = lo_bits;
  }
  M->s = ddiv((double)beta, r);
  if (!finite_f64(M->s) || !(M->s >= 2.2250738585072014e-308)) return 1;
  const uint64_t sb = f64_bits(M->s);
  const int32_t es = (int32_t)((sb >> 52) & 0x7FFu) - 1075;
  M->sig = ((sb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  // v = Dn 2^H s = Dn Sig 2^(H + es - 11), V = Dn Sig 2^-64  =>  F = -(H + es + 53)
  M->F = -(H + es + 53);
  if (M->F < 1 || M->F > 63) return 1;  // unreachable for beta < 2^32
  // (beta + 1) 2^(F-52) + slack, rounded up
  double e2 = (double)(beta + 1ull);
  const int32_t ex = M->F - 52;
  e2 = ex >= 0 ? e2 * (double)(1ull << ex) : e2 / (double)(1ull << (-ex));
  M->eu = (uint64_t)e2 + 8ull;
  // lo and hi with the same sign and exponent: so has every key between
  // them, X(y) is its 52-bit fraction shifted by one fixed amount, and Dn is
  // the difference of fractions shifted (the same integer as the general
  // formula, without a per-key exponent)
  if (kt == KEY_F64 && (lo_bits >> 52) == (hi_bits >> 52)) {
    const uint32_t e = (uint32_t)(lo_bits >> 52) & 0x7FFu;
    const int32_t sh = (int32_t)(e ? e : 1u) - M->C;
    if (sh >= 0 && sh < 64) {
      M->mode = (lo_bits >> 63) ? 2u : 1u;
      M->LOw = lo_bits & 0x000FFFFFFFFFFFFFull;
      M->w = sh;
    }
  }
  return 0;
}

// Dn of a key (see above)
PCF_HD uint64_t bin_dn(const BinModel& M, uint64_t xbits) {
  if (M.kt == KEY_F64) {
    if (M.mode == 0) return fixed_mod(xbits, M.C) - M.LOw;
    const uint64_t fx = xbits & 0x000FFFFFFFFFFFFFull;
    return (M.mode == 1 ? fx - M.LOw : M.LOw - fx) << M.w;
  }
  const uint64_t d = xbits - M.LOw;
  return M.w >= 0 ? (d << M.w) : (d >> (-M.w));
}

// Exact binary64 evaluation (the reading above, op by op).
PCF_HD uint32_t bin_exact_v(uint32_t kt, uint64_t lo_bits, double lo_d, double s, uint32_t beta,
                            uint64_t xbits) {
  double d = kt == KEY_F64 ? dsub(as_f64(xbits), lo_d) : u64_to_f64(xbits - lo_bits);
  double p = dmul(d, s);
  if (!(p < (double)beta)) return beta;
  if (!(p > 0.0)) return 0u;
#ifdef __CUDA_ARCH__
  return __double2uint_rd(p);
#else
  return (uint32_t)__builtin_floor(p);
#endif
}
PCF_HD uint32_t bin_exact(const BinModel& M, uint64_t xbits) {
  if (M.clamp && ord_of(xbits, M.kt) < M.ord_lo) return 0u;  // below a sample range
  return bin_exact_v(M.kt, M.lo_bits, M.lo_d, M.s, M.beta, xbits);
}

#ifdef __CUDA_ARCH__
// Out of line, so that the binary64 instructions run only in the lanes that
// need them (GB300 issues binary64 at 1/64 of the fp32 rate; a predicated
// inline copy would cost every key four of them).
__device__ __noinline__ uint32_t bin_exact_call(uint32_t kt, uint64_t lo_bits, double lo_d,
                                                double s, uint32_t beta, uint64_t xbits) {
  return bin_exact_v(kt, lo_bits, lo_d, s, beta, xbits);
}
#endif

// Keys outside a sample range (R14): below it bin 0; above it the exact
// sequence (the fixed-point form covers [lo, hi] only).  Returns 1 and sets
// *k when it decides, 2 when the exact sequence must, 0 otherwise.
PCF_HD int bin_outside(const BinModel& M, uint64_t xbits, uint32_t* k) {
  if (!M.clamp) return 0;
  const uint64_t o = ord_of(xbits, M.kt);
  if (o < M.ord_lo) {
    *k = 0u;
    return 1;
  }
  return o > M.ord_hi ? 2 : 0;
}

// Certified fast path, exact binary64 sequence when it cannot decide.
PCF_HD uint32_t bin_of(const BinModel& M, uint64_t xbits) {
  uint32_t ko = 0;
  const int out = bin_outside(M, xbits, &ko);
  if (out == 1) return ko;
  if (out == 2) {
#ifdef __CUDA_ARCH__
    return bin_exact_call(M.kt, M.lo_bits, M.lo_d, M.s, M.beta, xbits);
#else
    return bin_exact(M, xbits);
#endif
  }
  const uint64_t V = mulhi64(bin_dn(M, xbits), M.sig);
  const uint32_t klo = shr_F(V > M.eu ? V - M.eu : 0ull, M.F), khi = shr_F(V + M.eu, M.F);
  if (klo >= M.beta) return M.beta;
  if (klo == khi) return klo;
#ifdef __CUDA_ARCH__
  return bin_exact_call(M.kt, M.lo_bits, M.lo_d, M.s, M.beta, xbits);
#else
  return bin_exact(M, xbits);
#endif
}

// Fast path only: the bin when *amb stays false; callers that evaluate many
// keys collect the undecided ones and run bin_exact afterwards, keeping the
// out-of-line call out of their load/compute loops.
// (a model over the array's range: every key lies in [lo, hi])
PCF_HD uint32_t bin_fast(const BinModel& M, uint64_t xbits, bool& amb) {
  const uint64_t V = mulhi64(bin_dn(M, xbits), M.sig);
  const uint32_t klo = shr_F(V > M.eu ? V - M.eu : 0ull, M.F), khi = shr_F(V + M.eu, M.F);
  amb = klo < M.beta && klo != khi;
  return klo >= M.beta ? M.beta : klo;
}

// The same for a model that may be over the samples' range (R14): keys
// below it bin 0, keys above it undecided (the exact sequence decides).
PCF_HD uint32_t bin_fast_clamped(const BinModel& M, uint64_t xbits, bool& amb) {
  uint32_t ko = 0;
  const int out = bin_outside(M, xbits, &ko);
  if (out) {
    amb = out == 2;
    return ko;
  }
  return bin_fast(M, xbits, amb);
}

// Exact bin of a key (out of line on the device)
// (callers reach it only for keys that bin_fast or bin_fast_clamped left
// undecided, none of which lies below a sample range)
PCF_HD uint32_t bin_exact_of(const BinModel& M, uint64_t xbits) {
#ifdef __CUDA_ARCH__
  return bin_exact_call(M.kt, M.lo_bits, M.lo_d, M.s, M.beta, xbits);
#else
  return bin_exact(M, xbits);
#endif
}

// Whether the fast path decides this key (for tests and counters).
PCF_HD bool bin_fast_decides(const BinModel& M, uint64_t xbits) {
  uint32_t ko = 0;
  const int out = bin_outside(M, xbits, &ko);
  if (out) return out == 1;
  const uint64_t V = mulhi64(bin_dn(M, xbits), M.sig);
  const uint32_t klo = shr_F(V > M.eu ? V - M.eu : 0ull, M.F), khi = shr_F(V + M.eu, M.F);
  return klo >= M.beta || klo == khi;
}

// --------------------------------------------------------------------------
// Bucket id of bin k (Alg. 1: floor(F gamma) with F = b_k / alpha), exact.
// --------------------------------------------------------------------------
PCF_HD uint32_t bucket_of_count(uint32_t bk, uint32_t alpha, uint32_t gamma) {
  if (alpha == gamma) return bk;
  return (uint32_t)(((uint64_t)bk * gamma) / alpha);
}

// --------------------------------------------------------------------------
// Spline model (App. A.5).  For x in bin k at relative position f in
// [t_k, t_{k+1}), F(x) = (b_{k-1} + f (b_k - b_{k-1})) / alpha with
// b_{-1} = 0, and the bucket is floor(F gamma).  Binary64, round to nearest,
// no contraction, in this order:
//   p = RN(RN(x - lo) s)   (the bin's own value: k = clamp(floor(p), 0, beta))
//   f = p - k for 0 < p < beta (exact), else 0
//   y = RN(b_{k-1} + RN(f (b_k - b_{k-1})))
//   j = min(floor(RN(y g)), gamma),  g = RN(gamma / alpha)
// j does not decrease with x (each step is monotone, and y never passes b_k
// inside bin k), so buckets stay ordered (Sec. 3.2).
// --------------------------------------------------------------------------
PCF_HD void spline_set(BinModel* M, uint32_t alpha, uint32_t gamma) {
  M->spline = 1;
  M->gamma = gamma;
  M->g = ddiv((double)gamma, (double)alpha);
}

// bin of x and its position in it (the first two steps above)
PCF_HD uint32_t spline_bin(const BinModel& M, uint64_t xbits, double* f) {
  if (M.clamp && ord_of(xbits, M.kt) < M.ord_lo) {  // below a sample range
    *f = 0.0;
    return 0u;
  }
  const double d = M.kt == KEY_F64 ? dsub(as_f64(xbits), M.lo_d) : u64_to_f64(xbits - M.lo_bits);
  const double p = dmul(d, M.s);
  if (!(p < (double)M.beta)) {
    *f = 0.0;
    return M.beta;
  }
  if (!(p > 0.0)) {
    *f = 0.0;
    return 0u;
  }
#ifdef __CUDA_ARCH__
  const uint32_t k = __double2uint_rd(p);
#else
  const uint32_t k = (uint32_t)__builtin_floor(p);
#endif
  *f = dsub(p, (double)k);
  return k;
}

// bucket of x from its bin k, position f and the cumulative counts
// b_{k-1} (0 for k = 0) and b_k
PCF_HD uint32_t spline_bucket(const BinModel& M, double f, uint32_t bkm1, uint32_t bk) {
  const double y = dadd((double)bkm1, dmul(f, (double)(bk - bkm1)));
  const double z = dmul(y, M.g);
  if (!(z < (double)M.gamma)) return M.gamma;
#ifdef __CUDA_ARCH__
  return z > 0.0 ? __double2uint_rd(z) : 0u;
#else
  return z > 0.0 ? (uint32_t)__builtin_floor(z) : 0u;
#endif
}

}  // namespace pcf

// pcf_common.cuh -- shared host/device definitions of the PCF Learned Sort
// kernels (Sato & Matsui, "PCF Learned Sort", TMLR 2025).
//
// Everything here is compiled both for sm_103a and for the host (the host
// copies back the C ABI's self-test entry points); none of it is shared
// with the CPU oracle.
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

struct Policy {
  uint32_t a_num, b_num, c_num, d_num, den;
  uint32_t pad;
  uint64_t tau;
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
//   X(x)  = trunc(x / 2^G)        64-bit fixed point, G chosen so |X| < 2^62
//   D     = X(x) - X(lo)          in [0, X(hi) - X(lo)]  (trunc is monotone)
//   V     = hi64((D << w) * Sig)  Sig = 53-bit significand of s, << 11
//   V / 2^F approximates v = (x - lo) s.
// Truncation of X moves V by at most 8 units (it only happens when the range
// spans zero, and then w <= 2), hi64 by 1 unit, and the two binary64 roundings
// move the exact result P by at most v 2^-52 (1 + 2^-50) <= (beta+1) 2^(F-52)
// units.  With Eu bounding all three, floor(P) = floor(V / 2^F) whenever
// [V - Eu, V + Eu] holds no multiple of 2^F.
// --------------------------------------------------------------------------
struct BinModel {
  uint64_t lo_bits;  // raw bits of lo
  double lo_d;       // lo as binary64 (f64 keys)
  double s;          // beta / range
  int64_t LO;        // X(lo) (f64 keys)
  uint64_t sig;      // significand of s << 11, in [2^63, 2^64)
  uint64_t eu;       // error bound in V units
  int32_t C;         // f64: X(x) uses shift max(e,1) - C
  int32_t w;         // left shift of D (-1: right shift by one, u64 only)
  int32_t F;         // fractional bits of V
  uint32_t beta;
  uint32_t kt;
  uint32_t pad;
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

// Fixed point trunc(x / 2^G) with G = C - 1075, as a signed integer.
PCF_HD int64_t fixed_of(uint64_t bits, int32_t C) {
  uint32_t e = (uint32_t)(bits >> 52) & 0x7FFu;
  uint64_t m = (bits & 0x000FFFFFFFFFFFFFull) | (e ? 0x0010000000000000ull : 0ull);
  int32_t sh = (int32_t)(e ? e : 1u) - C;
  uint64_t mag = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
  return (bits >> 63) ? -(int64_t)mag : (int64_t)mag;
}

// Builds the model of the range [lo, hi] with beta bins.  Returns 0, or 1
// when the range is degenerate (zero, not finite, or a non-normal scale):
// such (sub)arrays go to the standard sort.
PCF_HD int make_bin_model(uint32_t kt, uint64_t lo_bits, uint64_t hi_bits, uint32_t beta,
                          BinModel* M) {
  M->kt = kt;
  M->beta = beta;
  M->lo_bits = lo_bits;
  M->pad = 0;
  double r;
  uint64_t range;
  int32_t G;
  if (kt == KEY_F64) {
    M->lo_d = as_f64(lo_bits);
    r = dsub(as_f64(hi_bits), M->lo_d);
    if (!(r > 0.0) || !finite_f64(r)) return 1;
    uint32_t elo = (uint32_t)(lo_bits >> 52) & 0x7FFu, ehi = (uint32_t)(hi_bits >> 52) & 0x7FFu;
    uint32_t em = elo > ehi ? elo : ehi;
    if (em < 1) em = 1;
    G = (int32_t)em - 1075 - 9;
    M->C = 1075 + G;
    M->LO = fixed_of(lo_bits, M->C);
    range = (uint64_t)(fixed_of(hi_bits, M->C) - M->LO);
  } else {
    M->lo_d = 0.0;
    range = hi_bits - lo_bits;
    r = u64_to_f64(range);
    G = 0;
    M->C = 0;
    M->LO = (int64_t)lo_bits;
  }
  M->s = ddiv((double)beta, r);
  if (!finite_f64(M->s) || !(M->s >= 2.2250738585072014e-308)) return 1;
  if (range == 0) return 1;  // cannot happen for distinct finite keys
  M->w = 62 - floor_log2_u64(range);
  uint64_t sb = f64_bits(M->s);
  int32_t es = (int32_t)((sb >> 52) & 0x7FFu) - 1075;
  M->sig = ((sb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
  M->F = M->w - G - es - 53;
  if (M->F < 1 || M->F > 63) return 1;  // unreachable for beta < 2^32
  // (beta + 1) 2^(F-52) + slack, rounded up
  double e2 = (double)(beta + 1ull);
  int32_t ex = M->F - 52;
  e2 = ex >= 0 ? e2 * (double)(1ull << ex) : e2 / (double)(1ull << (-ex));
  M->eu = (uint64_t)e2 + 17ull;
  return 0;
}

// Exact binary64 evaluation (the reading above, op by op).
PCF_HD uint32_t bin_exact(const BinModel& M, uint64_t xbits) {
  double d = M.kt == KEY_F64 ? dsub(as_f64(xbits), M.lo_d) : u64_to_f64(xbits - M.lo_bits);
  double p = dmul(d, M.s);
  if (!(p < (double)M.beta)) return M.beta;
  if (!(p > 0.0)) return 0u;
#ifdef __CUDA_ARCH__
  return __double2uint_rd(p);
#else
  return (uint32_t)__builtin_floor(p);
#endif
}

// Certified fast path; *amb is set when the exact path was needed.
PCF_HD uint32_t bin_of(const BinModel& M, uint64_t xbits) {
  uint64_t D = M.kt == KEY_F64 ? (uint64_t)(fixed_of(xbits, M.C) - M.LO) : (xbits - M.lo_bits);
  uint64_t Dn = M.w >= 0 ? (D << M.w) : (D >> 1);
  uint64_t V = mulhi64(Dn, M.sig);
  uint64_t vlo = V > M.eu ? V - M.eu : 0ull;
  uint64_t klo = vlo >> M.F, khi = (V + M.eu) >> M.F;
  if (klo >= M.beta) return M.beta;
  if (klo == khi) return (uint32_t)klo;
  return bin_exact(M, xbits);
}

// Whether the fast path decides this key (for tests and counters).
PCF_HD bool bin_fast_decides(const BinModel& M, uint64_t xbits) {
  uint64_t D = M.kt == KEY_F64 ? (uint64_t)(fixed_of(xbits, M.C) - M.LO) : (xbits - M.lo_bits);
  uint64_t Dn = M.w >= 0 ? (D << M.w) : (D >> 1);
  uint64_t V = mulhi64(Dn, M.sig);
  uint64_t vlo = V > M.eu ? V - M.eu : 0ull;
  uint64_t klo = vlo >> M.F, khi = (V + M.eu) >> M.F;
  return klo >= M.beta || klo == khi;
}

// --------------------------------------------------------------------------
// Bucket id of bin k (Alg. 1: floor(F gamma) with F = b_k / alpha), exact.
// --------------------------------------------------------------------------
PCF_HD uint32_t bucket_of_count(uint32_t bk, uint32_t alpha, uint32_t gamma) {
  if (alpha == gamma) return bk;
  return (uint32_t)(((uint64_t)bk * gamma) / alpha);
}

}  // namespace pcf

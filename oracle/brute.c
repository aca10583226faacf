/*
 * brute.c -- brute-force references used only to pin the oracle in tests.
 * TEST INFRASTRUCTURE ONLY (see pcf_oracle.c).  Deliberately naive and
 * independent of pcf_oracle.c's code paths.
 */
#include <stdint.h>

/* Total-order comparison of two keys given as raw bits.
 * f64 (kt = 0): IEEE-754 totalOrder restricted to non-NaN values, i.e.
 * -inf < ... < -0 < +0 < ... < +inf, decided here from sign and magnitude
 * rather than by the bit transform the oracle uses. */
static int brute_less(uint64_t a, uint64_t b, int kt) {
  if (kt == 1) return a < b;
  int sa = (int)(a >> 63), sb = (int)(b >> 63);
  uint64_t ma = a & 0x7FFFFFFFFFFFFFFFULL, mb = b & 0x7FFFFFFFFFFFFFFFULL;
  if (sa != sb) return sa > sb;   /* negative before non-negative */
  if (sa == 0) return ma < mb;    /* both non-negative: larger magnitude is larger */
  return ma > mb;                 /* both negative: larger magnitude is smaller */
}

/* Stable insertion sort (O(n^2)); vals may be NULL. */
void brute_insertion_sort(uint64_t* k, uint32_t* v, uint64_t n, int kt) {
  for (uint64_t i = 1; i < n; ++i) {
    uint64_t key = k[i];
    uint32_t val = v ? v[i] : 0;
    uint64_t j = i;
    while (j > 0 && brute_less(key, k[j - 1], kt)) {
      k[j] = k[j - 1];
      if (v) v[j] = v[j - 1];
      --j;
    }
    k[j] = key;
    if (v) v[j] = val;
  }
}

/* b_i = |{ j : bin(a_j) <= i }| for i = 0..beta, straight from the
 * definition: O(alpha * beta). */
void brute_cumulative_counts(const uint64_t* sample_bins, uint64_t alpha, uint64_t beta,
                             uint64_t* b) {
  for (uint64_t i = 0; i <= beta; ++i) {
    uint64_t c = 0;
    for (uint64_t j = 0; j < alpha; ++j)
      if (sample_bins[j] <= i) c += 1;
    b[i] = c;
  }
}

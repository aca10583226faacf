/*
 * pcfsort_debug.h -- self-test hooks of the PCF Learned Sort library.
 *
 * These entry points exist for the library's own tests: host copies of
 * the device arithmetic (checked on a machine without a GPU against the
 * CPU oracle), the level-0 intermediates of one array (compared with a
 * sequential run of Sec. 3.3's training), the decoupled look-back scan
 * with a tile that never publishes (the bounded wait's timeout path), and
 * an injected allocation failure.  They are not part of the sorting
 * interface (pcfsort.h) and may change without notice.
 */
#ifndef PCFSORT_DEBUG_H
#define PCFSORT_DEBUG_H

#include <stdint.h>

#include "pcfsort.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The k-th device workspace allocation from now on this host thread (0:
 * the next) fails as an exhausted device reports it (PCF_ERR_OOM from the
 * call); k < 0 clears the injection. */
void pcf_debug_fail_alloc_after(int64_t k);

/* Host copy of the kernels' bin function (Sec. 3.3, i(x) - 1 in binary64
 * as the library reads it) for the range [lo_bits, hi_bits] and beta bins:
 * out[i] = bin of xs[i] (m keys, HOST arrays), fast_decided[i] (may be
 * NULL) = 1 where the integer fast path decided it alone.  Returns 1, and
 * writes nothing, when the range is degenerate. */
int pcf_debug_bins_host(uint32_t kt, uint64_t lo_bits, uint64_t hi_bits, uint32_t beta,
                        const uint64_t* xs, uint64_t m, uint32_t* out, uint8_t* fast_decided);

/* Host copies of floor(n^(p/q)) (the policy's alpha..delta) and of sample
 * index j of the (sub)array keyed by (seed, depth, start, n). */
uint64_t pcf_debug_root_floor(uint64_t n, uint32_t p, uint32_t q);
uint64_t pcf_debug_sample_index(uint64_t seed, uint64_t depth, uint64_t start, uint64_t n,
                                uint64_t j);

/* The decoupled look-back exclusive scan on d_data[0..n) (DEVICE u32) in
 * place; withhold_tile: a tile that never publishes (UINT32_MAX: none), so
 * that its successor's bounded wait gives up after spin_limit polls (0: the
 * library's limit) and the call returns PCF_ERR_TIMEOUT. */
pcf_status pcf_debug_scan(pcf_ctx* ctx, uint32_t* d_data, uint64_t n, uint32_t withhold_tile,
                          uint64_t spin_limit, void* stream);

/* Level 0 of one array of n >= 2 DEVICE keys: h_params8 (HOST, 8 u64) =
 * alpha, beta, gamma, delta, lo bits, hi bits, status (0 bucketed, 1 one
 * value, 2 degenerate range), 0; h_T (HOST, T_cap >= beta + 1 entries, may
 * be NULL) = the bucket table floor(b_k gamma / alpha). */
pcf_status pcf_debug_level0(pcf_ctx* ctx, const void* d_keys, uint64_t n, pcf_key_type kt,
                            uint64_t seed, uint64_t* h_params8, uint32_t* h_T, uint64_t T_cap);

#ifdef __cplusplus
}
#endif

#endif /* PCFSORT_DEBUG_H */

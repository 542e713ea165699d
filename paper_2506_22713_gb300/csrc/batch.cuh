// Host interface of the persistent batched factorisation (batch.cu).
#pragma once

#include "common.cuh"

#include <cstdint>
#include <vector>

namespace eod {

constexpr int kPRcap = 128;       // basis columns one CTA keeps (the core's leaf width)
constexpr int kPKmax = 64;        // largest block size k of the persistent form
constexpr int kPTdCap = kPRcap + 2;
constexpr int kPFallback = -1;    // item status: left to the single-matrix path
constexpr int64_t kPMaxDim = 16384;   // largest m or n of an item of the persistent form
constexpr int kPPhases = 11;          // phases of the measurement hook
constexpr double kPF32Floor = 1e-5;   // eps below this x ||A||_F: EOD_EPRECISION (FP32 products cannot resolve it)

// Factors items of FP32 data in one persistent launch on `s`.  Items that
// finish there get their factors in out[i] and status in per_item[i];
// `fallback` receives the indices the single-matrix path must take (rank
// above kPRcap, core Gram needing the shifted CholQR, or sizes outside the
// form).  Returns EOD_OK unless the launch itself failed, in which case
// every item is in `fallback` (or, once the kernel ran, EOD_ECUDA with no
// item to retry).
eod_status factor_batched_persistent(const void *const *A, const int64_t *m, const int64_t *n, const int64_t *lda,
                                     int64_t count, double tol, uint64_t seed, const eod_opts &o, eod_factors **out,
                                     eod_status *per_item, std::vector<int64_t> &fallback);

// Releases a factor set's device memory when it lives in a persistent
// batch's shared pool (returns false, touching nothing, otherwise).
bool release_pooled_factors(eod_factors *f);

}  // namespace eod

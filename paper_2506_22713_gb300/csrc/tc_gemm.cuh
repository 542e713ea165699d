// Interface of the tensor-core (tcgen05) contractions of the mixed path.
#pragma once
#include "common.cuh"

namespace eod {

template <typename T>
struct MixedOps {
    eod_status prepare(const T *, int64_t, int64_t, int64_t, struct Arena &, cudaStream_t) { return EOD_EUNSUPPORTED; }
    eod_status sketch(int64_t, int64_t, uint64_t, uint64_t, T *, int64_t, cudaStream_t) { return EOD_EUNSUPPORTED; }
    eod_status project(const T *, int64_t, T *, cudaStream_t) { return EOD_EUNSUPPORTED; }
    eod_status recon_error(const T *, int64_t, const T *, const double *, double *, cudaStream_t) { return EOD_EUNSUPPORTED; }
};

}  // namespace eod

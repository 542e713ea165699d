// Launch counting and per-kind CUDA-event timing (see instrument.cu).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace eod {

// kernel kinds, as reported by eod_abe_debug_profile_read()
enum ProfKind {
    PROF_GEMM_SIMT = 0,   // SIMT GEMM in FP64 arithmetic (plain path contractions), incl. its split-K reduction
    PROF_CHOL = 1,        // one-CTA Cholesky / rank test
    PROF_OMEGA = 2,       // Gaussian test blocks
    PROF_STREAM = 3,      // norms, copies, scaling, splitting
    PROF_TC_GEMM = 4,     // tcgen05 tensor-core contractions (mixed path)
    PROF_OZ_GEMM = 5,     // FP64 contractions emulated on tcgen05 (plain FP64 path)
    PROF_OZ_SLICE = 6,    // FP64 operands cut into BF16 digit slices for those contractions
    PROF_GEMM_SIMT32 = 7, // SIMT GEMM and Gram in FP32 arithmetic (FP32-data paths)
    PROF_BATCH = 8,       // the persistent batched factorisation (one launch per batch)
    PROF_KINDS = 9
};

void count_launch(int n = 1);

class ProfScope {
  public:
    ProfScope(int kind, double flops, double bytes, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    cudaStream_t s_;
    int rec_;
};

// NVTX range for one phase of the method (visible to nsys / ncu --nvtx);
// names are "eod.<phase>".
class Phase {
  public:
    explicit Phase(const char *name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

}  // namespace eod

// Interface of the tensor-core (tcgen05) contractions and of the mixed
// (BF16 or TF32 split, FP32 accumulation) forms of the sketch, the
// projection and the reconstruction error.
#pragma once
#include "common.cuh"

#include <cuda_bf16.h>

namespace eod {

// A BF16 (or, in the TF32 form, FP32) matrix operand as TMA sees it:
// `inner` contiguous elements per row of the map, `outer` rows, `ld`
// elements between rows (ld times the element size must be a multiple of
// 16 bytes, the base 16-byte aligned).
struct TcOperand {
    const void *ptr = nullptr;
    int64_t inner = 0, outer = 0, ld = 0;
};

// D (M x N, FP32, column-major) = alpha * sum over pairs p of op(a[p]) *
// op(b[p]) + beta * D (D is read only when beta != 0).
// B operands are always K-major (K = inner).  A operands are K-major (inner =
// K, outer = M) unless a_mn_major, then inner = M and outer = K.
// EPI_ERR: instead of storing D, each CTA writes sum((ref - D)^2) over its
// tile to err_partials[cta] (tc_gemm_err_ctas() entries).
struct TcGemmDesc {
    int64_t M = 0, N = 0, K = 0;
    bool a_mn_major = false;
    bool tf32 = false;            // FP32-stored TF32 operands (kind::tf32, K-major only)
    int npairs = 1;
    TcOperand a[3], b[3];
    int epilogue = EPI_STORE;
    float *D = nullptr;
    int64_t ldd = 0;
    const float *ref = nullptr;
    int64_t ldref = 0;
    double *err_partials = nullptr;
    int *err_flag = nullptr;      // set to 1 by a CTA whose bounded wait ran out
    int bn = 0;                   // N tile (32, 64, 128, 256); 0 = by N
    float alpha = 1.f, beta = 0.f;
};

cudaError_t tc_gemm_run(const TcGemmDesc &g, Scratch *ws, cudaStream_t s);
int64_t tc_gemm_err_ctas(int64_t M, int64_t N, int bn);

// X (rows x cols, FP32) -> X_hi = bf16(X), X_lo = bf16(X - X_hi) and, when
// x3 is given, X_3 = bf16(X - X_hi - X_lo) (then X_hi + X_lo + X_3 == X),
// same layout with ld ldo; with partials != nullptr also the S0 sums of
// squares and non-finite flags per block (blocks entries each).
cudaError_t split_norm(const float *X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16 *hi,
                       __nv_bfloat16 *lo, int64_t ldo, double *partials, int *flags, int blocks, cudaStream_t s,
                       __nv_bfloat16 *x3 = nullptr);
// Xt_hi / Xt_lo (cols x rows, ld ldt) = split of X^T.
cudaError_t split_transpose(const float *X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16 *hi,
                            __nv_bfloat16 *lo, int64_t ldt, cudaStream_t s);
// TF32 form: X_hi = X with the 13 low significand bits cleared, X_lo = X - X_hi
// (FP32 storage), same layout (ld ldo) or transposed (cols x rows, ld ldt).
cudaError_t split_tf32(const float *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo, int64_t ldo,
                       cudaStream_t s);
cudaError_t split_transpose_tf32(const float *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo,
                                 int64_t ldt, cudaStream_t s);
// The same split of FP64 data rounded to FP32 first (same layout, ld ldo).
cudaError_t split_tf32_f64(const double *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo,
                           int64_t ldo, cudaStream_t s);

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// The mixed forms used by factor_impl<float> when precision is
// EOD_MIXED_BF16 or EOD_MIXED_TF32 (implemented in mixed.cu).  Other storage
// types never reach the tensor cores (FP64 input is narrowed to FP32 first).
template <typename T>
struct MixedOps {
    Scratch *ws = nullptr;
    eod_status prepare(const T *, int64_t, int64_t, int64_t, int64_t, Arena &, Scratch *, cudaStream_t, bool,
                       double * = nullptr, int * = nullptr) {
        return EOD_EUNSUPPORTED;
    }
    eod_status sketch(int64_t, int64_t, uint64_t, uint64_t, T *, int64_t, cudaStream_t) { return EOD_EUNSUPPORTED; }
    eod_status project(const T *, int64_t, T *, cudaStream_t) { return EOD_EUNSUPPORTED; }
    eod_status recon_error(const T *, int64_t, const T *, const double *, double *, cudaStream_t, cudaStream_t) {
        return EOD_EUNSUPPORTED;
    }
    eod_status check(cudaStream_t) { return EOD_OK; }
};

template <>
struct MixedOps<float> {
    Arena *ar = nullptr;
    Scratch *ws = nullptr;
    const float *A = nullptr;
    int64_t m = 0, n = 0, lda = 0, cap = 0, k = 0, ldm8 = 0, ldn8 = 0;
    bool tf32 = false;
    // BF16 form: A split into three terms, Omega in BF16
    __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr, *A3 = nullptr;
    __nv_bfloat16 *Om = nullptr;
    // TF32 form: A's two terms as stored (m x n) and transposed (n x m, for
    // the sketch's K-major operand), Omega in FP32
    float *Th = nullptr, *Tl = nullptr, *Tth = nullptr, *Ttl = nullptr, *Om32 = nullptr;
    // sketch window: Yw holds A Omega for global columns win_c0 .. win_c0 + win_w - 1
    float *Yw = nullptr;
    int64_t win_cap = 0, win_c0 = -1, win_w = 0, next_w = 0;
    int *err_flag = nullptr;

    // splits A; with d_norm (BF16 form only) the same pass also gives
    // ||A||_F into d_norm and ORs the non-finite flag into d_flag
    eod_status prepare(const float *A, int64_t m, int64_t n, int64_t lda, int64_t k, Arena &ar, Scratch *ws,
                       cudaStream_t s, bool tf32, double *d_norm = nullptr, int *d_flag = nullptr);
    eod_status sketch(int64_t col0, int64_t f, uint64_t seed, uint64_t batch, float *Y, int64_t ldy, cudaStream_t s);
    eod_status project(const float *Q, int64_t r, float *Ct, cudaStream_t s);
    // buffers from the arena on `s`; the kernels run on `run` (which may be
    // `s`), ordered after those allocations
    eod_status recon_error(const float *Q, int64_t r, const float *Ct, const double *d_norm, double *d_err,
                           cudaStream_t s, cudaStream_t run);
    eod_status check(cudaStream_t s);   // EOD_ETIMEOUT if a bounded device wait ran out
};

}  // namespace eod

// Small dense factorisations in FP64, one CTA each:
//  * Cholesky of a w x w Gram matrix (w <= 128) with the rank test of
//    Alg. 1 steps 6-11 folded into the pivot loop, plus the inverse of the
//    triangular factor (CholQR: P = Y R^{-1}) -- the leaf itself, and its
//    rank decisions, are in chol_leaf.cuh;
//  * the diagonal of T = R2 R1 (the T_j(l,l) the test reads, Rem. 3.6);
//  * trace(G) for the shift of shifted CholQR.
#include "common.cuh"
#include "chol_leaf.cuh"
#include "instrument.cuh"

#include <algorithm>

namespace eod {
namespace {

template <bool LA>
__global__ void __launch_bounds__(kLeafThreads) chol_small_kernel(const double *__restrict__ G, int64_t ldg, int w,
                                                                  int decide, double eps2, double delta_coef,
                                                                  double rho, double shift, double *__restrict__ R,
                                                                  int64_t ldr, double *__restrict__ Rinv,
                                                                  int64_t ldinv, int *info, double ni_tau2) {
    extern __shared__ double sh[];
    chol_leaf_cta<LA>(G, ldg, w, decide, eps2, delta_coef, rho, shift, R, ldr, Rinv, ldinv, info, ni_tau2, sh);
}

__global__ void recip_kernel(const double *d, double *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = recip_pos(d[i]);
}

__global__ void tdiag_kernel(const double *R1, const double *R2, int64_t ldr, const int *p_dev,
                             double *tdiag) {
    const int p = *p_dev;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
        tdiag[j] = fabs(R1[j + j * ldr] * R2[j + j * ldr]);
}

// ||G - I||_F^2 of a symmetric p x p matrix from its upper triangle.
// Partial sums of ||G - I||_F^2 (upper triangle read): CTA b takes the
// columns c = b, b + gridDim.x, ..., a warp per column, lanes down it; the
// partials are added in CTA order by offidentity_finish_kernel.
__global__ void offidentity_partial_kernel(const double *G, int64_t ldg, int64_t p, double *part) {
    __shared__ double red[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double acc = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * nw + warp; c < p; c += (int64_t)gridDim.x * nw) {
        const double *col = G + c * ldg;
        for (int64_t i = lane; i <= c; i += 32) {
            const double v = col[i] - (i == c ? 1.0 : 0.0);
            acc = fma(i == c ? v : 2.0 * v, v, acc);
        }
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void offidentity_finish_kernel(const double *part, int n, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) out[0] = tot;
}

// R = I + Phi(G - I) (p x p, upper, zeros below) and, for every diagonal
// panel J of width pb, R_JJ^{-1} = I - Phi(G_JJ - I) at RiD + J pb^2 (ld pb):
// the first-order Cholesky factor of a near-identity Gram and its inverse.
__global__ void near_identity_kernel(const double *G, int64_t ldg, int64_t p, double *R, int64_t ldr, double *RiD,
                                     int pb) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p * p; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % p, c = e / p;
        const double g = (i <= c) ? G[i + c * ldg] : 0.0;
        const double x = (i < c) ? g : (i == c ? 0.5 * (g - 1.0) : 0.0);
        R[i + c * ldr] = (i == c ? 1.0 : 0.0) + x;
        if (i / pb == c / pb) {
            const int64_t J = i / pb, ii = i - J * pb, cc = c - J * pb;
            RiD[J * (int64_t)pb * pb + ii + cc * pb] = (i == c ? 1.0 : 0.0) - x;
        }
    }
}

__global__ void trace_kernel(const double *G, int64_t ldg, int64_t p, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < p; j += blockDim.x) acc += G[j + j * ldg];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) out[0] = tot;
}

}  // namespace

cudaError_t chol_small(const double *G, int64_t ldg, int w, int decide, double eps2, double delta_coef,
                       double rho, double shift, double *R, int64_t ldr, double *Rinv, int64_t ldinv, int *info,
                       cudaStream_t s, double ni_tau2, bool classic) {
    if (w < 1 || w > 128) return cudaErrorInvalidValue;
    if (decide || shift != 0.0) ni_tau2 = 0.0;
    EOD_CUDA_TRY(set_smem_once(chol_small_kernel<true>, (int)leaf_smem_bytes(128)));
    EOD_CUDA_TRY(set_smem_once(chol_small_kernel<false>, (int)leaf_smem_bytes(128)));
    ProfScope prof(PROF_CHOL, (double)w * w * w * (Rinv ? 2.0 : 1.0) / 3.0, sizeof(double) * 3.0 * w * w, s);
    count_launch();
    if (classic)
        chol_small_kernel<false><<<1, kLeafThreads, leaf_smem_bytes(w), s>>>(G, ldg, w, decide, eps2, delta_coef, rho,
                                                                            shift, R, ldr, Rinv, ldinv, info, ni_tau2);
    else
        chol_small_kernel<true><<<1, kLeafThreads, leaf_smem_bytes(w), s>>>(G, ldg, w, decide, eps2, delta_coef, rho,
                                                                           shift, R, ldr, Rinv, ldinv, info, ni_tau2);
    return cudaGetLastError();
}

cudaError_t offidentity_sumsq(const double *G, int64_t ldg, int64_t p, double *part, double *out, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>((p + 7) / 8, kOffIdMaxBlocks);
    count_launch(2);
    offidentity_partial_kernel<<<blocks, 256, 0, s>>>(G, ldg, p, part);
    offidentity_finish_kernel<<<1, 256, 0, s>>>(part, blocks, out);
    return cudaGetLastError();
}

cudaError_t near_identity_factor(const double *G, int64_t ldg, int64_t p, double *R, int64_t ldr, double *RiD,
                                 int pb, cudaStream_t s) {
    count_launch();
    const int64_t tot = p * p;
    near_identity_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(G, ldg, p, R, ldr, RiD,
                                                                                                pb);
    return cudaGetLastError();
}

cudaError_t tdiag_product(const double *R1, const double *R2, int64_t ldr, const int *p_dev, double *tdiag,
                          cudaStream_t s) {
    count_launch();
    tdiag_kernel<<<1, 128, 0, s>>>(R1, R2, ldr, p_dev, tdiag);
    return cudaGetLastError();
}

cudaError_t trace_sum(const double *G, int64_t ldg, int64_t p, double *out, cudaStream_t s) {
    count_launch();
    trace_kernel<<<1, 1024, 0, s>>>(G, ldg, p, out);
    return cudaGetLastError();
}

}  // namespace eod

// ---------------------------------------------------------------------------
// Test hook: the leaf factorisation's reciprocal on n positive doubles.
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_recip(const double *d, double *out, int64_t n, void *stream) {
    using namespace eod;
    if (!d || !out || n < 1) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    count_launch();
    recip_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(d, out, n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EOD_ECUDA;
    }
    return EOD_OK;
}

// ---------------------------------------------------------------------------
// Test hook: one leaf factorisation (see the header).
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_chol(const double *G, int64_t ldg, int32_t w, int32_t decide, double eps2,
                                         double delta_coef, double rho, double shift, double *R, double *Rinv,
                                         int64_t ldr, int32_t *info, void *stream) {
    using namespace eod;
    if (!G || !R || !info || w < 1 || w > 128 || ldg < w || ldr < w) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const bool classic = (decide & 256) != 0;
    cudaError_t e = chol_small(G, ldg, w, (decide & 255) ? 1 : 0, eps2, delta_coef, rho, shift, R, ldr, Rinv, ldr, info,
                               s, 0.0, classic);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EOD_ECUDA;
    }
    return EOD_OK;
}

// Small dense factorisations in FP64, one CTA each:
//  * Cholesky of a w x w Gram matrix (w <= 128) with the rank test of
//    Alg. 1 steps 6-11 folded into the pivot loop, plus the inverse of the
//    triangular factor (CholQR: P = Y R^{-1});
//  * the diagonal of T = R2 R1 (the T_j(l,l) the test reads, Rem. 3.6);
//  * trace(G) for the shift of shifted CholQR.
//
// Rank decision per pivot (G = Y^T Y, pivot d_l = T(l,l)^2 computed from
// the Gram):  the rounding error of d_l is bounded by delta_l = c u G(l,l)
// (Gram accumulation plus Cholesky), so
//   d_l < eps^2 - delta_l              -> |T(l,l)| <= eps for certain: stop;
//   d_l > eps^2 + delta_l and d_l > rho G(l,l)
//                                      -> |T(l,l)| > eps for certain: keep;
//   otherwise                          -> undecided at this precision: stop
//                                         the factorisation here and let the
//                                         caller settle column l with an
//                                         explicit FP64 residual norm.
// The rho guard (1e-10) also keeps every accepted panel well enough
// conditioned for CholQR2 to reach orthogonality at the unit roundoff.
#include "common.cuh"
#include "instrument.cuh"

namespace eod {
namespace {

__global__ void __launch_bounds__(256) chol_small_kernel(const double *__restrict__ G, int64_t ldg, int w,
                                                         int decide, double eps2, double delta_coef, double rho,
                                                         double shift, double *__restrict__ R, int64_t ldr,
                                                         int *info) {
    // L = R^T (lower triangle, column-major): column j of L is row j of R and
    // is contiguous, so the rank-1 trailing update reads it without conflicts.
    extern __shared__ double sh[];
    double *S = sh;              // w x w, lower triangle
    double *g0 = sh + w * w;     // original diagonal
    __shared__ int p_sh, code_sh, go_sh;
    __shared__ double rinv_sh;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // S(i, c) = G(c, i) for i >= c (G's upper triangle, transposed)
    for (int c = ty; c < w; c += 16)
        for (int i = tx; i < w; i += 16)
            S[i + c * w] = (i >= c) ? G[c + (int64_t)i * ldg] + (i == c ? shift : 0.0) : 0.0;
    for (int j = tid; j < w; j += blockDim.x) g0[j] = G[j + (int64_t)j * ldg] + shift;
    if (tid == 0) { p_sh = w; code_sh = CHOL_ALL; }
    __syncthreads();

    double rinv_prev = 0.0;
    for (int j = 0; j < w; ++j) {
        // phase 1: thread 0 decides pivot j while every thread finishes
        // column j-1 of L (scaled by the previous pivot's 1/L(j-1,j-1))
        if (tid == 0) {
            const double d = S[j + j * w];
            int keep;
            if (decide) {
                const double delta = delta_coef * g0[j];
                if (d < eps2 - delta) { keep = 0; code_sh = CHOL_BELOW; }
                else if (d > eps2 + delta && d > rho * g0[j] && isfinite(d)) keep = 1;
                else { keep = 0; code_sh = CHOL_UNCERTAIN; }
            } else {
                keep = (d > 0.0 && isfinite(d)) ? 1 : 0;
                if (!keep) code_sh = CHOL_FAIL;
            }
            if (keep) {
                const double ri = rsqrt(d);
                S[j + j * w] = d * ri;
                rinv_sh = ri;
            } else {
                p_sh = j;
            }
            go_sh = keep;
        }
        if (j > 0)
            for (int i = j + tid; i < w; i += blockDim.x) S[i + (j - 1) * w] *= rinv_prev;
        __syncthreads();
        if (!go_sh) break;
        const double rinv = rinv_sh;
        // phase 2: trailing update S(ii, ll) -= L(ii, j) L(ll, j), j < ll <= ii,
        // from the still unscaled column j times 1/L(j,j)
        for (int ll = j + 1 + ty; ll < w; ll += 16) {
            const double lj = S[ll + j * w] * rinv;
            for (int ii = ll + tx; ii < w; ii += 16) S[ii + ll * w] = fma(-S[ii + j * w] * rinv, lj, S[ii + ll * w]);
        }
        __syncthreads();
        rinv_prev = rinv;
    }
    const int p = p_sh;
    for (int c = ty; c < p; c += 16)
        for (int i = tx; i < p; i += 16) R[i + (int64_t)c * ldr] = (i <= c) ? S[c + i * w] : 0.0;
    if (tid == 0) { info[0] = p; info[1] = code_sh; }
}

// X = R^{-1} for upper-triangular R (p x p, ld ldr), one warp per column:
// column c solves R x = e_c from the bottom, x_j = b_j / R(j,j), then
// b_i -= x_j R(i,j) for i < j, with b spread over the lanes.
__global__ void __launch_bounds__(128) tri_inverse_kernel(const double *__restrict__ R, int64_t ldr, int p,
                                                          const int *p_dev, double *__restrict__ X,
                                                          int64_t ldx) {
    __shared__ double rd[128];
    if (p_dev) p = *p_dev;
    for (int j = threadIdx.x; j < p; j += blockDim.x) rd[j] = 1.0 / R[j + (int64_t)j * ldr];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (c >= p) return;
    constexpr int PER = 4;                      // p <= 128: lane holds b_i for i = lane + 32 t
    const int tmax = c >> 5;
    double b[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) b[t] = (lane + 32 * t == c) ? 1.0 : 0.0;
    for (int j = c; j >= 0; --j) {
        const int owner = j & 31, slot = j >> 5;
        double bj = 0.0;
#pragma unroll
        for (int t = 0; t < PER; ++t)
            if (t == slot) bj = b[t];
        bj = __shfl_sync(0xffffffffu, bj, owner);
        const double xj = bj * rd[j];
        if (lane == owner) {
#pragma unroll
            for (int t = 0; t < PER; ++t)
                if (t == slot) b[t] = xj;
        }
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int i = lane + 32 * t;
            if (t <= tmax && i < j) b[t] = fma(-xj, R[i + (int64_t)j * ldr], b[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int i = lane + 32 * t;
        if (i < p) X[i + (int64_t)c * ldx] = (i <= c) ? b[t] : 0.0;
    }
}

__global__ void tdiag_kernel(const double *R1, const double *R2, int64_t ldr, const int *p_dev,
                             double *tdiag) {
    const int p = *p_dev;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p; j += gridDim.x * blockDim.x)
        tdiag[j] = fabs(R1[j + j * ldr] * R2[j + j * ldr]);
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
                       double rho, double shift, double *R, double *Rinv, int64_t ldr, int *info,
                       cudaStream_t s) {
    if (w < 1 || w > 128) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * ((size_t)w * w + (size_t)w);
    EOD_CUDA_TRY(set_smem_once(chol_small_kernel, (int)(sizeof(double) * (128 * 128 + 128))));
    {
        ProfScope prof(PROF_CHOL, (double)w * w * w / 3.0, sizeof(double) * 2.0 * w * w, s);
        count_launch();
        chol_small_kernel<<<1, 256, smem, s>>>(G, ldg, w, decide, eps2, delta_coef, rho, shift, R, ldr, info);
        EOD_CUDA_TRY(cudaGetLastError());
    }
    if (Rinv) {
        // the factored order p is read on the device (info[0])
        ProfScope prof(PROF_CHOL, (double)w * w * w / 3.0, sizeof(double) * 2.0 * w * w, s);
        count_launch();
        tri_inverse_kernel<<<(w + 3) / 4, 128, 0, s>>>(R, ldr, w, info, Rinv, ldr);
        EOD_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
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

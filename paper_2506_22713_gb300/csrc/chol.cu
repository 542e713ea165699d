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

__global__ void chol_small_kernel(const double *__restrict__ G, int64_t ldg, int w, int decide,
                                  double eps2, double delta_coef, double rho, double shift,
                                  double *__restrict__ R, double *__restrict__ Rinv, int64_t ldr,
                                  int *info) {
    extern __shared__ double sh[];
    double *S = sh;              // w x w: R in the upper triangle, X = R^{-1} transposed below it
    double *g0 = sh + w * w;     // original diagonal
    double *xd = g0 + w;         // diagonal of R^{-1}
    __shared__ int p_sh, code_sh, go_sh;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int e = tid; e < w * w; e += nt) {
        const int i = e % w, j = e / w;
        S[e] = (i <= j) ? G[i + (int64_t)j * ldg] + (i == j ? shift : 0.0) : 0.0;
    }
    for (int j = tid; j < w; j += nt) g0[j] = G[j + (int64_t)j * ldg] + shift;
    if (tid == 0) { p_sh = w; code_sh = CHOL_ALL; }
    __syncthreads();

    for (int j = 0; j < w; ++j) {
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
            if (keep) S[j + j * w] = sqrt(d);
            else p_sh = j;
            go_sh = keep;
        }
        __syncthreads();
        if (!go_sh) break;
        const double rjj = S[j + j * w];
        for (int l = j + 1 + tid; l < w; l += nt) S[j + l * w] /= rjj;
        __syncthreads();
        const int rem = w - j - 1;
        for (int e = tid; e < rem * rem; e += nt) {
            const int ii = j + 1 + e % rem, ll = j + 1 + e / rem;
            if (ii <= ll) S[ii + ll * w] = fma(-S[j + ii * w], S[j + ll * w], S[ii + ll * w]);
        }
        __syncthreads();
    }
    const int p = p_sh;

    // X = R^{-1}, row by row from the bottom: X(i,c) = -sum_{l=i+1..c} R(i,l) X(l,c) / R(i,i).
    // X(i,c), i < c, lives at S[c + i*w] (below the diagonal); X(i,i) in xd[i].
    for (int i = tid; i < p; i += nt) xd[i] = 1.0 / S[i + i * w];
    __syncthreads();
    for (int i = p - 2; i >= 0; --i) {
        const double rii = S[i + i * w];
        for (int c = i + 1 + tid; c < p; c += nt) {
            double acc = S[i + c * w] * xd[c];
            for (int l = i + 1; l < c; ++l) acc = fma(S[i + l * w], S[c + l * w], acc);
            S[c + i * w] = -acc / rii;
        }
        __syncthreads();
    }
    for (int e = tid; e < p * p; e += nt) {
        const int i = e % p, c = e / p;
        R[i + (int64_t)c * ldr] = (i <= c) ? S[i + c * w] : 0.0;
        Rinv[i + (int64_t)c * ldr] = (i < c) ? S[c + i * w] : (i == c ? xd[i] : 0.0);
    }
    if (tid == 0) { info[0] = p; info[1] = code_sh; }
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
    const size_t smem = sizeof(double) * ((size_t)w * w + 2 * (size_t)w);
    static bool attr_set = false;
    if (!attr_set) {
        EOD_CUDA_TRY(cudaFuncSetAttribute(chol_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(double) * (128 * 128 + 256))));
        attr_set = true;
    }
    ProfScope prof(PROF_CHOL, (double)w * w * w / 3.0, sizeof(double) * 2.0 * w * w, s);
    count_launch();
    chol_small_kernel<<<1, 256, smem, s>>>(G, ldg, w, decide, eps2, delta_coef, rho, shift, R, Rinv, ldr, info);
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

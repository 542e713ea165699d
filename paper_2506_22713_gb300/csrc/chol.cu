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

// Pivot decision for column j (one thread): the rank test when `decide`,
// else plain positivity.  Sets *go, and on acceptance S(j,j) = sqrt(d) and
// *rinv = 1/sqrt(d); on rejection *p_out = j and *code.
__device__ __forceinline__ void chol_pivot(double *S, int w, int j, const double *g0, int decide, double eps2,
                                           double delta_coef, double rho, int *go, double *rinv, int *p_out,
                                           int *code) {
    const double d = S[j + j * w];
    int keep;
    if (decide) {
        const double delta = delta_coef * g0[j];
        if (d < eps2 - delta) { keep = 0; *code = CHOL_BELOW; }
        else if (d > eps2 + delta && d > rho * g0[j] && isfinite(d)) keep = 1;
        else { keep = 0; *code = CHOL_UNCERTAIN; }
    } else {
        keep = (d > 0.0 && isfinite(d)) ? 1 : 0;
        if (!keep) *code = CHOL_FAIL;
    }
    if (keep) {
        const double ri = rsqrt(d);
        S[j + j * w] = d * ri;
        *rinv = ri;
    } else {
        *p_out = j;
    }
    *go = keep;
}

// One CTA of 256 threads.  L = R^T is built in shared memory (lower
// triangle, column-major: column j of L is row j of R).  Step j, after pivot
// j is accepted:
//   (A) every thread takes rows i > j: L(i,j) = S(i,j)/L(j,j) and the
//       update of column j+1, S(i,j+1) -= L(i,j) L(j+1,j);
//   (B) warp 0 decides pivot j+1 while warps 1-7 apply L(:,j) to the rest
//       of the trailing triangle (columns > j+1), whose entries are spread
//       evenly over the threads through a table of (row, column) pairs
//       ordered by column from the right, so the entries of columns > c form
//       a prefix of it.
// Every entry sees the same operations in the same order as the textbook
// right-looking loop, so the factor is identical to it.
__global__ void __launch_bounds__(256) chol_small_kernel(const double *__restrict__ G, int64_t ldg, int w,
                                                         int decide, double eps2, double delta_coef, double rho,
                                                         double shift, double *__restrict__ R, int64_t ldr,
                                                         int *info) {
    extern __shared__ double sh[];
    double *S = sh;                                    // w x w, lower triangle
    double *g0 = sh + w * w;                           // original diagonal
    uint16_t *pairs = (uint16_t *)(g0 + w);            // w (w - 1) / 2 entries: row | column << 8
    __shared__ int p_sh, code_sh, go_sh;
    __shared__ double rinv_sh;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // S(i, c) = G(c, i) for i >= c (G's upper triangle, transposed)
    for (int c = ty; c < w; c += 16)
        for (int i = tx; i < w; i += 16)
            S[i + c * w] = (i >= c) ? G[c + (int64_t)i * ldg] + (i == c ? shift : 0.0) : 0.0;
    for (int j = tid; j < w; j += blockDim.x) g0[j] = G[j + (int64_t)j * ldg] + shift;
    const int npairs = w * (w - 1) / 2;
    for (int e = tid; e < npairs; e += blockDim.x) {
        // column ll = w - 1 - c holds c + 1 entries; columns w-1 .. ll hold (c+1)(c+2)/2
        int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while ((c + 1) * (c + 2) / 2 <= e) ++c;
        while (c * (c + 1) / 2 > e) --c;
        const int ll = w - 1 - c, ii = ll + (e - c * (c + 1) / 2);
        pairs[e] = (uint16_t)(ii | (ll << 8));
    }
    if (tid == 0) {
        p_sh = w;
        code_sh = CHOL_ALL;
    }
    __syncthreads();
    if (tid == 0) chol_pivot(S, w, 0, g0, decide, eps2, delta_coef, rho, &go_sh, &rinv_sh, &p_sh, &code_sh);
    __syncthreads();

    for (int j = 0; j < w; ++j) {
        if (!go_sh) break;
        const double rinv = rinv_sh;
        const bool next = j + 1 < w;
        // (A) scale column j (rows > j; row j+1 is stored in (B), after every
        // thread has read it) and update column j+1
        const double lj1 = next ? S[(j + 1) + j * w] * rinv : 0.0;
        for (int i = j + 1 + tid; i < w; i += blockDim.x) {
            const double lij = S[i + j * w] * rinv;
            if (i > j + 1) S[i + j * w] = lij;
            S[i + (j + 1) * w] = fma(-lij, lj1, S[i + (j + 1) * w]);
        }
        __syncthreads();
        if (!next) break;
        // (B) pivot j+1 on warp 0; columns > j+1 on warps 1-7
        if (tid == 0) {
            chol_pivot(S, w, j + 1, g0, decide, eps2, delta_coef, rho, &go_sh, &rinv_sh, &p_sh, &code_sh);
        } else if (tid >= 32) {
            if (tid == 32) S[(j + 1) + j * w] = lj1;
            const int cnt = (w - 2 - j) * (w - 1 - j) / 2;
            for (int e = tid - 32; e < cnt; e += blockDim.x - 32) {
                const int pr = pairs[e];
                const int ii = pr & 0xff, ll = pr >> 8;
                S[ii + ll * w] = fma(-S[ii + j * w], S[ll + j * w], S[ii + ll * w]);
            }
        }
        __syncthreads();
    }
    const int p = p_sh;
    for (int c = ty; c < p; c += 16)
        for (int i = tx; i < p; i += 16) R[i + (int64_t)c * ldr] = (i <= c) ? S[c + i * w] : 0.0;
    if (tid == 0) { info[0] = p; info[1] = code_sh; }
}

// X = R^{-1} for upper-triangular R (p x p, ld ldr, p <= 32 PER), one warp
// per column: column c solves R x = e_c from the bottom, x_j = b_j / R(j,j),
// then b_i -= x_j R(i,j) for i < j, with b spread over the lanes.
template <int PER>
__global__ void __launch_bounds__(128) tri_inverse_kernel(const double *__restrict__ R, int64_t ldr, int p,
                                                          const int *p_dev, double *__restrict__ X,
                                                          int64_t ldx) {
    __shared__ double rd[32 * PER];
    if (p_dev) p = *p_dev;
    for (int j = threadIdx.x; j < p; j += blockDim.x) rd[j] = 1.0 / R[j + (int64_t)j * ldr];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (c >= p) return;
    // lane holds b_i for i = lane + 32 t
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
    const size_t smem = sizeof(double) * ((size_t)w * w + (size_t)w) + sizeof(uint16_t) * (size_t)(w * (w - 1) / 2);
    EOD_CUDA_TRY(set_smem_once(chol_small_kernel, (int)(sizeof(double) * (128 * 128 + 128) + sizeof(uint16_t) * 8128)));
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
        tri_inverse_kernel<4><<<(w + 3) / 4, 128, 0, s>>>(R, ldr, w, info, Rinv, ldr);
        EOD_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

cudaError_t tri_inverse(const double *R, int64_t ldr, int p, double *X, int64_t ldx, cudaStream_t s) {
    if (p < 1 || p > 256) return cudaErrorInvalidValue;
    ProfScope prof(PROF_CHOL, (double)p * p * p / 3.0, sizeof(double) * 2.0 * p * p, s);
    count_launch();
    if (p <= 128) tri_inverse_kernel<4><<<(p + 3) / 4, 128, 0, s>>>(R, ldr, p, nullptr, X, ldx);
    else tri_inverse_kernel<8><<<(p + 3) / 4, 128, 0, s>>>(R, ldr, p, nullptr, X, ldx);
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

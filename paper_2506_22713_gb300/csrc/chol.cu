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

// Monotone integer key of a finite double (x < y  <=>  key(x) < key(y)):
// the pivot decisions compare through these, on the integer units.
__device__ __forceinline__ long long dkey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : -(b & 0x7fffffffffffffffll);
}

// 1/d for finite d > 0: FP32 reciprocal of the mantissa as the seed (the
// exponent handled on the integer bits), then two Newton steps
// r <- r + r (1 - d r) in FP64, each doubling the 23 correct bits.  No FP64
// division anywhere (each FP64 instruction costs a warp 64 cycles here):
// a subnormal d gives +inf, a d near the top of the range 0.
__device__ __forceinline__ double recip_pos(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int E = (int)(b >> 52);                                  // biased exponent
    const unsigned int mf = 0x3f800000u | (unsigned int)((b >> 29) & 0x7fffffu);   // mantissa in [1, 2)
    const float rf = __frcp_rn(__uint_as_float(mf));               // (0.5, 1]
    const unsigned int rb = __float_as_uint(rf);
    const long long re = (long long)((rb >> 23) & 0xff) - 127 + 1023 - (E - 1023);
    const long long rbits = (re << 52) | ((long long)(rb & 0x7fffffu) << 29);
    double r = __longlong_as_double(rbits);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    return (E == 0 || re >= 2047) ? inf : (re <= 0 ? 0.0 : r);
}

// Pivot decision for column j (one thread) on the integer keys: the rank test
// when `decide` (thresholds precomputed per column), else positivity.  A
// non-finite pivot is undecided (rank test) or a failure.  On acceptance
// *rd = 1/d.
__device__ __forceinline__ void ldl_pivot(const double *S, int w, int j, const long long *klo, const long long *khi,
                                          const long long *krg, int decide, double *dv, int *go, double *rd,
                                          int *p_out, int *code, bool writer) {
    const double d = S[j + j * w];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const bool finite = ((bits >> 52) & 0x7ff) != 0x7ff;
    const long long kd = dkey(d);
    int keep, c = CHOL_ALL;
    if (!finite) {
        keep = 0;
        c = decide ? CHOL_UNCERTAIN : CHOL_FAIL;
    } else if (decide) {
        if (kd < klo[j]) { keep = 0; c = CHOL_BELOW; }
        else if (kd > khi[j] && kd > krg[j]) keep = 1;
        else { keep = 0; c = CHOL_UNCERTAIN; }
    } else {
        keep = kd > 0 ? 1 : 0;
        if (!keep) c = CHOL_FAIL;
    }
    const double r = recip_pos(d);
    if (writer) {
        if (keep) {
            dv[j] = d;
            *rd = r;
        } else {
            *p_out = j;
            *code = c;
        }
        *go = keep;
    }
}

// One CTA of 256 threads: G + shift I = L D L^T (unit lower L, no square
// roots on the critical path), R = D^{1/2} L^T, and optionally
// R^{-1} = L^{-T} D^{-1/2}.  Step j, once pivot j is accepted:
//   (A) every thread takes rows i > j: keeps u_i = S(i,j), stores
//       L(i,j) = u_i / d_j, and updates column j+1: S(i,j+1) -= L(i,j) u_{j+1};
//   (B) warp 0 decides pivot j+1 (integer compares, reciprocal by Newton)
//       while warps 1-7 apply S(ii,ll) -= L(ii,j) u_ll to the rest of the
//       trailing triangle, spread evenly over the threads through a table of
//       (row, column) pairs ordered by column from the right (the entries of
//       columns > c form a prefix of it).
// The rank test reads the pivots d_j = T(j,j)^2 exactly as the Cholesky form
// would; R differs from a square-root Cholesky only by rounding.
__global__ void __launch_bounds__(256) chol_small_kernel(const double *__restrict__ G, int64_t ldg, int w,
                                                         int decide, double eps2, double delta_coef, double rho,
                                                         double shift, double *__restrict__ R,
                                                         double *__restrict__ Rinv, int64_t ldr, int *info) {
    extern __shared__ double sh[];
    double *S = sh;                                    // w x w, lower triangle
    double *u = S + w * w;                             // unscaled column of the step
    double *dv = u + w;                                // pivots d_j
    double *sq = dv + w;                               // sqrt(d_j), then 1/sqrt(d_j)
    long long *klo = (long long *)(sq + w);            // keys of eps^2 - delta_j, eps^2 + delta_j, rho G(j,j)
    long long *khi = klo + w;
    long long *krg = khi + w;
    uint16_t *pairs = (uint16_t *)(krg + w);           // w (w - 1) / 2 entries: row | column << 8
    __shared__ int p_sh, code_sh, go_sh;
    __shared__ double rd_sh;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    // S(i, c) = G(c, i) for i >= c (G's upper triangle, transposed)
    for (int c = ty; c < w; c += 16)
        for (int i = tx; i < w; i += 16)
            S[i + c * w] = (i >= c) ? G[c + (int64_t)i * ldg] + (i == c ? shift : 0.0) : 0.0;
    if (decide) {
        for (int j = tid; j < w; j += blockDim.x) {
            const double g0 = G[j + (int64_t)j * ldg];
            const double delta = delta_coef * g0;
            klo[j] = dkey(eps2 - delta);
            khi[j] = dkey(eps2 + delta);
            krg[j] = dkey(rho * g0);
        }
    }
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
    if (tid < 32) ldl_pivot(S, w, 0, klo, khi, krg, decide, dv, &go_sh, &rd_sh, &p_sh, &code_sh, tid == 0);
    __syncthreads();

    for (int j = 0; j < w; ++j) {
        if (!go_sh) break;
        const double rd = rd_sh;
        const bool next = j + 1 < w;
        const double u1 = next ? S[(j + 1) + j * w] : 0.0;   // row j+1 is scaled in (B)
        for (int i = j + 1 + tid; i < w; i += blockDim.x) {
            const double ui = S[i + j * w];
            const double lij = ui * rd;
            u[i] = ui;
            if (i > j + 1) S[i + j * w] = lij;
            S[i + (j + 1) * w] = fma(-lij, u1, S[i + (j + 1) * w]);
        }
        __syncthreads();
        if (!next) break;
        if (tid < 32) {
            // the whole warp computes the pivot (no divergence on the
            // critical path; FP64 costs a warp the same for 1 or 32 lanes),
            // lane 0 publishes it
            ldl_pivot(S, w, j + 1, klo, khi, krg, decide, dv, &go_sh, &rd_sh, &p_sh, &code_sh, tid == 0);
        } else if (tid >= 32 && (tid >> 5) != 4) {
            // warps 1-3 and 5-7: warp 4 shares warp 0's sub-partition, whose
            // FP64 pipe (64 cycles per warp instruction) stays free for the pivot
            if (tid == 32) S[(j + 1) + j * w] = u1 * rd;
            const int cnt = (w - 2 - j) * (w - 1 - j) / 2;
            const int me = tid - 32 - ((tid >> 5) > 4 ? 32 : 0);
            for (int e = me; e < cnt; e += blockDim.x - 64) {
                const int pr = pairs[e];
                const int ii = pr & 0xff, ll = pr >> 8;
                S[ii + ll * w] = fma(-S[ii + j * w], u[ll], S[ii + ll * w]);
            }
        }
        __syncthreads();
    }
    const int p = p_sh;
    for (int j = tid; j < p; j += blockDim.x) sq[j] = sqrt(dv[j]);
    __syncthreads();
    // R(i, c) = sqrt(d_i) L(c, i) for i < c, sqrt(d_i) on the diagonal
    for (int c = ty; c < p; c += 16)
        for (int i = tx; i < p; i += 16)
            R[i + (int64_t)c * ldr] = (i < c) ? sq[i] * S[c + i * w] : (i == c ? sq[i] : 0.0);
    if (tid == 0) { info[0] = p; info[1] = code_sh; }
    if (!Rinv) return;
    __syncthreads();
    for (int j = tid; j < p; j += blockDim.x) sq[j] = 1.0 / sq[j];
    // Z = L^{-1} in place of L (strictly lower part).  With M = -L stored
    // first, step k takes Z(i,c) += M(i,k) Z(k,c) for i > k, c < k; column k
    // still holds M(i,k) = Z(i,k)'s first term when step k reads it, so one
    // barrier per step suffices.
    for (int c = ty; c < p; c += 16)
        for (int i = tx; i < p; i += 16)
            if (i > c) S[i + c * w] = -S[i + c * w];
    __syncthreads();
    for (int k = 1; k < p - 1; ++k) {
        const int rows = p - 1 - k, cnt = rows * k;
        // entry e = c * rows + (i - k - 1), i fastest (conflict-free column
        // accesses); advanced by the block size without a division per entry
        const int dc = (int)blockDim.x / rows, di = (int)blockDim.x - dc * rows;
        int c = tid / rows, io = tid - c * rows;
        for (int e = tid; e < cnt; e += blockDim.x) {
            const int i = k + 1 + io;
            S[i + c * w] = fma(S[i + k * w], S[k + c * w], S[i + c * w]);
            c += dc;
            io += di;
            if (io >= rows) { io -= rows; ++c; }
        }
        __syncthreads();
    }
    // R^{-1}(i, c) = Z(c, i) / sqrt(d_c) for i < c, 1/sqrt(d_c) on the diagonal
    for (int c = ty; c < p; c += 16)
        for (int i = tx; i < p; i += 16)
            Rinv[i + (int64_t)c * ldr] = (i < c) ? S[c + i * w] * sq[c] : (i == c ? sq[c] : 0.0);
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
    auto bytes = [](int n) {
        return sizeof(double) * ((size_t)n * n + 4 * (size_t)n) + sizeof(long long) * 3 * (size_t)n +
               sizeof(uint16_t) * (size_t)(n * (n - 1) / 2);
    };
    EOD_CUDA_TRY(set_smem_once(chol_small_kernel, (int)bytes(128)));
    ProfScope prof(PROF_CHOL, (double)w * w * w * (Rinv ? 2.0 : 1.0) / 3.0, sizeof(double) * 3.0 * w * w, s);
    count_launch();
    chol_small_kernel<<<1, 256, bytes(w), s>>>(G, ldg, w, decide, eps2, delta_coef, rho, shift, R, Rinv, ldr, info);
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
// Test hook: one leaf factorisation (see the header).
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_chol(const double *G, int64_t ldg, int32_t w, int32_t decide, double eps2,
                                         double delta_coef, double rho, double shift, double *R, double *Rinv,
                                         int64_t ldr, int32_t *info, void *stream) {
    using namespace eod;
    if (!G || !R || !info || w < 1 || w > 128 || ldg < w || ldr < w) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = chol_small(G, ldg, w, decide ? 1 : 0, eps2, delta_coef, rho, shift, R, Rinv, ldr, info, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EOD_ECUDA;
    }
    return EOD_OK;
}

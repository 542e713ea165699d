// The one-CTA FP64 factorisation of a small Gram matrix (w <= 128) with the
// rank test of Alg. 1 steps 6-11 folded into its pivot loop, as a device
// function: the leaf kernel of chol.cu runs it alone, the batched one-CTA
// factorisation inside its item loop.
//
// Rank decision per pivot (G = Y^T Y, pivot d_l = T(l,l)^2 computed from
// the Gram): the rounding error of d_l is bounded by delta_l = c u G(l,l)
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
#pragma once

#include "common.cuh"

#include <cstdint>

namespace eod {
namespace {

// Monotone integer key of a finite double (x < y  <=>  key(x) < key(y)):
// the pivot decisions compare through these, on the integer units.
__device__ __forceinline__ long long dkey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : -(b & 0x7fffffffffffffffll);
}

// 1/d for finite d > 0: FP32 reciprocal of the mantissa as the seed (the
// exponent handled on the integer bits, relative error e below 2^-22), then
// one third-order step r <- r (1 + e + e^2), e = 1 - d r: since
// 1/d = r / (1 - e), this is the geometric series of 1/(1 - e) truncated
// after e^2, in three dependent FP64 FMAs (the error left is e^3, far below
// 2^-53, plus the roundings of the last FMAs: within 2 ulp of 1/d, tested
// against CUDA's division over the exponent range).  No FP64 division
// anywhere (each FP64 instruction costs a warp 64 cycles here).  Deliberate
// edge returns: a subnormal d gives +inf, and a d whose reciprocal would be
// subnormal (d above about 2^1022) gives 0; the callers only pass pivots of
// Gram matrices, far inside that range.
__device__ __forceinline__ double recip_pos(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int E = (int)(b >> 52);                                  // biased exponent
    const unsigned int mf = 0x3f800000u | (unsigned int)((b >> 29) & 0x7fffffu);   // mantissa in [1, 2)
    const float rf = __frcp_rn(__uint_as_float(mf));               // (0.5, 1]
    const unsigned int rb = __float_as_uint(rf);
    const long long re = (long long)((rb >> 23) & 0xff) - 127 + 1023 - (E - 1023);
    const long long rbits = (re << 52) | ((long long)(rb & 0x7fffffu) << 29);
    const double r0 = __longlong_as_double(rbits);
    const double e = fma(-d, r0, 1.0);
    const double r = fma(r0, fma(e, e, e), r0);
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    return (E == 0 || re >= 2047) ? inf : (re <= 0 ? 0.0 : r);
}

// Pivot decision for column j (one warp, lane 0 publishes): the rank test
// when `decide` (thresholds precomputed per column), else positivity.  A
// non-finite pivot is undecided (rank test) or a failure.  On acceptance
// *rd = 1/d_j and *mt = -L(j+1, j), the multiplier the next column update
// needs.
__device__ __forceinline__ void ldl_pivot(const double *S, int ld, int w, int j, const long long *klo,
                                          const long long *khi, const long long *krg, int decide, double *dv,
                                          int *go, double *rd, double *mt, int *p_out, int *code, bool writer) {
    const double d = S[j + j * ld];
    const double below = (j + 1 < w) ? S[(j + 1) + j * ld] : 0.0;
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
    const double t = below * r;
    if (writer) {
        if (keep) {
            dv[j] = d;
            *rd = r;
            *mt = -t;
        } else {
            *p_out = j;
            *code = c;
        }
        *go = keep;
    }
}

constexpr int kLeafThreads = 512;

inline size_t leaf_smem_bytes(int w) {
    // S, M, pivots, sqrt and 1/sqrt, three key arrays, the entry table, then
    // (8-byte aligned) the lookahead's second M buffer
    return sizeof(double) * ((size_t)w * (w + 1) + 4 * (size_t)w) + sizeof(long long) * 3 * (size_t)w +
           sizeof(uint16_t) * (size_t)((w - 1) * (w - 2) / 2 + 1) + 8 + sizeof(double) * (size_t)w;
}

// One CTA: G + shift I = L D L^T (unit lower L, no square roots on the
// critical path), R = D^{1/2} L^T and, in the same steps, Z = L^{-1} (so
// R^{-1} = L^{-T} D^{-1/2}) by Gauss-Jordan: once L(:,j) is known, every row
// r > j takes S(r, c) += M(r) S(j, c) with M = -L(:, j), for the trailing
// columns j+2 <= c <= r (the Schur update) and for c < j (the rows of Z).
// Storage, one w x (w+1) array (odd stride: rows and columns are both read
// without bank conflicts): the trailing lower triangle; Z in the strict lower
// part of the finished columns; row j of the upper part holds u = column j
// before scaling (R's row j up to 1/sqrt(d_j)).  Step j, pivot j accepted:
//   (A) column j+1 takes its update (threads 0-127), the u row and M are
//       staged (the last 128 threads, rows 0-63 on the last two warps, on
//       other sub-partitions than the first two);
//   (B) warp 0 decides pivot j+1 (integer compares, reciprocal by a
//       third-order step) and computes -L(j+2, j+1); warp 4 stores M as
//       Z's column j; the warps off sub-partition 0 apply the updates,
//       spread evenly through a table of (row, k) pairs ordered by row from
//       the bottom (row r holds r-1 entries, so the rows > j form a prefix).
// The SM's FP64 unit is shared by its sub-partitions (a dependent DFMA
// chain takes 68 cycles per op alone, 135 beside six streaming warps on the
// other sub-partitions, 362 with one more on its own: probe), so sub-partition
// 0 carries no FP64 work besides the pivot chain; 16 warps rather than 8
// hide more of the update loop's latency (61 vs 70 us at w = 64).
// The rank test reads the pivots d_j = T(j,j)^2 exactly as the Cholesky form
// would; R differs from a square-root Cholesky only by rounding.
// The leaf as a device function of a whole CTA of kLeafThreads threads; sh
// is its dynamic shared memory (leaf_smem_bytes(w) bytes, 16-byte aligned)
// and info may point to shared or global memory.  Every thread of the CTA
// must call it; it ends without a trailing barrier.
template <bool LA>
__device__ void chol_leaf_cta(const double *__restrict__ G, int64_t ldg, int w, int decide, double eps2,
                              double delta_coef, double rho, double shift, double *__restrict__ R, int64_t ldr,
                              double *__restrict__ Rinv, int64_t ldinv, int *info, double ni_tau2, double *sh) {
    constexpr int NT = kLeafThreads;
    // Near-identity Gram (the second pass of CholQR2, G = P^T P = I + E with
    // P already orthonormal to first order): when ||E||_F^2 <= ni_tau2,
    // R = I + Phi(E) and R^{-1} = I - Phi(E) (Phi = the strict upper part
    // and half the diagonal), exact up to O(||E||^2): (I + Phi(E))^T
    // (I + Phi(E)) = I + E + Phi(E)^T Phi(E).
    if (ni_tau2 > 0.0) {
        __shared__ double red[32];
        const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
        double acc = 0.0;
        for (int c = wp; c < w; c += NT / 32)          // a warp per column, lanes down it
            for (int i = ln; i <= c; i += 32) {
                const double v = G[i + (int64_t)c * ldg] - (i == c ? 1.0 : 0.0);
                acc = fma(i == c ? v : 2.0 * v, v, acc);
            }
        const double tot = block_sum(acc, red);
        if (tot <= ni_tau2) {
            for (int c = wp; c < w; c += NT / 32)
                for (int i = ln; i < w; i += 32) {
                    const double g = (i <= c) ? G[i + (int64_t)c * ldg] : 0.0;
                    const double x = (i < c) ? g : (i == c ? 0.5 * (g - 1.0) : 0.0);
                    R[i + (int64_t)c * ldr] = (i == c ? 1.0 : 0.0) + x;
                    if (Rinv) Rinv[i + (int64_t)c * ldinv] = (i == c ? 1.0 : 0.0) - x;
                }
            if (threadIdx.x == 0) {
                info[0] = w;
                info[1] = CHOL_ALL;
            }
            return;
        }
    }
    const int ld = w + 1;
    double *S = sh;                                    // w x ld
    double *mcol = S + w * ld;                         // M = -L(:, j) of the current step
    double *dv = mcol + w;                             // pivots d_j
    double *sq = dv + w;                               // sqrt(d_j)
    double *rs = sq + w;                               // 1 / sqrt(d_j)
    long long *klo = (long long *)(rs + w);            // keys of eps^2 - delta_j, eps^2 + delta_j, rho G(j,j)
    long long *khi = klo + w;
    long long *krg = khi + w;
    uint16_t *ent = (uint16_t *)(krg + w);             // (w-1)(w-2)/2 entries: row | k << 8
    double *mcol2 = (double *)(((uintptr_t)(ent + (w - 1) * (w - 2) / 2 + 1) + 7) & ~(uintptr_t)7);   // LA: M of odd steps
    __shared__ int p_sh, code_sh, go_sh;
    __shared__ double rd_sh, mt_sh;
    __shared__ int go2_sh[2];
    __shared__ double rd2_sh[2], mt2_sh[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // S(i, c) = G(c, i) for i >= c: G's upper triangle read along its columns
    // (coalesced), eight loads in flight per thread
    {
        const int tot = w * w, di = NT / w, dc = NT - di * w;
        int i = tid / w, c = tid - i * w;
        for (int e0 = tid; e0 < tot; e0 += 8 * NT) {
            double v[8];
            int ii[8], cc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ii[q] = i;
                cc[q] = c;
                v[q] = (e0 + q * NT < tot && c <= i) ? G[c + (int64_t)i * ldg] : 0.0;
                c += dc;
                i += di;
                if (c >= w) { c -= w; ++i; }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (e0 + q * NT < tot && cc[q] <= ii[q])
                    S[ii[q] + cc[q] * ld] = v[q] + (ii[q] == cc[q] ? shift : 0.0);
        }
    }
    if (decide) {
        for (int j = tid; j < w; j += NT) {
            const double g0 = G[j + (int64_t)j * ldg];
            const double delta = delta_coef * g0;
            klo[j] = dkey(eps2 - delta);
            khi[j] = dkey(eps2 + delta);
            krg[j] = dkey(rho * g0);
        }
    }
    // row r (2 <= r < w) holds k = 0 .. r-2 (column k, or k+2 once k >= j);
    // rows r+1 .. w-1 come before it: sum of (x - 1) for x > r
    for (int r = w - 1 - warp; r >= 2; r -= NT / 32) {
        const int off = ((w - 2) * (w - 1) - (r - 1) * r) / 2;
        for (int k = lane; k < r - 1; k += 32) ent[off + k] = (uint16_t)(r | (k << 8));
    }
    if (tid == 0) {
        p_sh = w;
        code_sh = CHOL_ALL;
    }
    __syncthreads();
    constexpr int NW = (NT / 32 - NT / 128) * 32;          // update threads: warps not on sub-partition 0
    const bool worker = (warp & 3) != 0;
    const int me = (warp - (warp >> 2) - 1) * 32 + lane;
    if (LA) {
        // Lookahead: one barrier per step.  In phase j the workers apply step
        // j (multipliers M_j, row u_j) to the columns >= j + 2 and to the rows
        // of Z, warp 4 stores M_j as Z's column j, and warp 0 meanwhile gives
        // column j + 1 its step-j update, decides pivot j + 1 and stages u_{j+1}
        // and M_{j+1} (the other buffer) for phase j + 1.  Column j + 1 holds
        // the updates of steps < j from the workers of phase j - 1.
        double *mb[2] = {mcol, mcol2};
        if (warp == 0) {
            ldl_pivot(S, ld, w, 0, klo, khi, krg, decide, dv, &go2_sh[0], &rd2_sh[0], &mt2_sh[0], &p_sh, &code_sh,
                      lane == 0);
            __syncwarp();
            if (go2_sh[0]) {
                const double r0 = rd2_sh[0];
                for (int i = 1 + lane; i < w; i += 32) {
                    const double ui = S[i];
                    S[i * ld] = ui;
                    mcol[i] = -(ui * r0);
                }
            }
        }
        __syncthreads();
        for (int j = 0; j < w; ++j) {
            const int b = j & 1;
            if (!go2_sh[b] || j + 1 >= w) break;
            const double *M = mb[b];
            if (warp == 0) {
                const double uj1 = S[j + (j + 1) * ld];             // u_j(j + 1)
                for (int i = j + 1 + lane; i < w; i += 32) S[i + (j + 1) * ld] = fma(M[i], uj1, S[i + (j + 1) * ld]);
                __syncwarp();
                ldl_pivot(S, ld, w, j + 1, klo, khi, krg, decide, dv, &go2_sh[b ^ 1], &rd2_sh[b ^ 1], &mt2_sh[b ^ 1],
                          &p_sh, &code_sh, lane == 0);
                __syncwarp();
                if (go2_sh[b ^ 1]) {
                    const double r1 = rd2_sh[b ^ 1];
                    double *M1 = mb[b ^ 1];
                    for (int i = j + 2 + lane; i < w; i += 32) {
                        const double ui = S[i + (j + 1) * ld];
                        S[(j + 1) + i * ld] = ui;
                        M1[i] = -(ui * r1);
                    }
                }
            } else if (warp == 4) {
                for (int i = j + 1 + lane; i < w; i += 32) S[i + j * ld] = M[i];
            } else if (worker) {
                const int cnt = ((w - 2) * (w - 1) - j * (j - 1)) / 2;
                int e = me;
                for (; e + NW < cnt; e += 2 * NW) {   // two entries in flight
                    const int pa = ent[e], pb = ent[e + NW];
                    const int ra = pa & 0xff, ka = pa >> 8, rb = pb & 0xff, kb = pb >> 8;
                    const int ca = ka < j ? ka : ka + 2, cb = kb < j ? kb : kb + 2;
                    const double ma = M[ra], mbv = M[rb];
                    const double xa = S[j + ca * ld], xb = S[j + cb * ld];
                    const double sa = S[ra + ca * ld], sb = S[rb + cb * ld];
                    S[ra + ca * ld] = fma(ma, xa, sa);
                    S[rb + cb * ld] = fma(mbv, xb, sb);
                }
                if (e < cnt) {
                    const int pa = ent[e];
                    const int ra = pa & 0xff, ka = pa >> 8;
                    const int ca = ka < j ? ka : ka + 2;
                    S[ra + ca * ld] = fma(M[ra], S[j + ca * ld], S[ra + ca * ld]);
                }
            }
            __syncthreads();
        }
        go_sh = 0;   // the classic loop below is skipped
    } else {
        if (warp == 0)
            ldl_pivot(S, ld, w, 0, klo, khi, krg, decide, dv, &go_sh, &rd_sh, &mt_sh, &p_sh, &code_sh, tid == 0);
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (!go_sh) break;
        const double rd = rd_sh, mt = mt_sh;
        // (A)
        if (tid < 128) {
            const int i = j + 1 + tid;
            if (i < w) S[i + (j + 1) * ld] = fma(S[i + j * ld], mt, S[i + (j + 1) * ld]);
        } else if (tid >= NT - 128) {
            const int i = j + 1 + ((tid - (NT - 128) + 64) & 127);
            if (i < w) {
                const double ui = S[i + j * ld];
                S[j + i * ld] = ui;
                mcol[i] = -(ui * rd);
            }
        }
        __syncthreads();
        if (j + 1 >= w) break;
        // (B)
        if (warp == 0) {
            ldl_pivot(S, ld, w, j + 1, klo, khi, krg, decide, dv, &go_sh, &rd_sh, &mt_sh, &p_sh, &code_sh, tid == 0);
        } else if (warp == 4) {
            for (int i = j + 1 + lane; i < w; i += 32) S[i + j * ld] = mcol[i];
        } else if (worker) {
            const int cnt = ((w - 2) * (w - 1) - j * (j - 1)) / 2;
            int e = me;
            for (; e + NW < cnt; e += 2 * NW) {   // two entries in flight
                const int pa = ent[e], pb = ent[e + NW];
                const int ra = pa & 0xff, ka = pa >> 8, rb = pb & 0xff, kb = pb >> 8;
                const int ca = ka < j ? ka : ka + 2, cb = kb < j ? kb : kb + 2;
                const double ma = mcol[ra], mb = mcol[rb];
                const double xa = S[j + ca * ld], xb = S[j + cb * ld];
                const double sa = S[ra + ca * ld], sb = S[rb + cb * ld];
                S[ra + ca * ld] = fma(ma, xa, sa);
                S[rb + cb * ld] = fma(mb, xb, sb);
            }
            if (e < cnt) {
                const int pa = ent[e];
                const int ra = pa & 0xff, ka = pa >> 8;
                const int ca = ka < j ? ka : ka + 2;
                S[ra + ca * ld] = fma(mcol[ra], S[j + ca * ld], S[ra + ca * ld]);
            }
        }
        __syncthreads();
    }
    const int p = p_sh;
    for (int j = tid; j < p; j += NT) {
        const double s = sqrt(dv[j]);
        sq[j] = s;
        rs[j] = 1.0 / s;
    }
    __syncthreads();
    // R(i, c) = u_i(c) / sqrt(d_i) for i < c, sqrt(d_i) on the diagonal;
    // R^{-1}(i, c) = Z(c, i) / sqrt(d_c) for i < c, 1/sqrt(d_c) on the diagonal
    if (p > 0) {
        const int tot = p * p, dc = NT / p, di = NT - dc * p;
        int c = tid / p, i = tid - c * p;
        for (int e = tid; e < tot; e += NT) {
            R[i + (int64_t)c * ldr] = (i < c) ? S[i + c * ld] * rs[i] : (i == c ? sq[i] : 0.0);
            if (Rinv) Rinv[i + (int64_t)c * ldinv] = (i < c) ? S[c + i * ld] * rs[c] : (i == c ? rs[c] : 0.0);
            c += dc;
            i += di;
            if (i >= p) { i -= p; ++c; }
        }
    }
    if (tid == 0) {
        info[0] = p;
        info[1] = code_sh;
    }
}

}  // namespace
}  // namespace eod

// FP64 GEMM emulated on tcgen05 BF16 tensor cores (exact slicing in the
// manner of Ozaki, Ogita and Oishi's error-free splitting), used by the plain
// FP64 path for its large contractions.
//
// Each row i of op(A) (and each column j of op(B)) is scaled by a power of
// two 2^-e so that its entries lie in (-1, 1), then cut into S = 8 integer
// slices (exact BF16 values): q_0 in [-64, 64] (6 bits + rounding), q_1..q_7
// in [-64, 64] (7 bits each):
//     a = 2^e * sum_s q_s 2^(-6 - 7s),   truncation below 2^(e-56).
// Products of slices are integers of magnitude <= 2^12.  Pairs (s, t) with
// s + t <= 7 are grouped by g = s + t (weight 2^(-12 - 7g)); group g holds
// g + 1 <= 8 pairs, so over a K chunk of 448 every group sum stays below
// 8 * 448 * 2^12 < 2^24 and the tensor core's FP32 accumulation is exact.
// After each chunk the epilogue warps read the eight group sums from TMEM as
// integers, merge groups 0-3 and 4-7 exactly in int64 (each below 2^46), and
// add the two merged values, scaled, into FP64 registers.  The dropped pairs
// (s + t > 7) weigh at most 2^-68 of the row / column scales.  The result
// equals an FP64 GEMM to within the slicing truncation (about 2^-56 of the
// row / column maxima per term), accumulated in FP64.
//
// CTA tile 128 x 64; a K block of 64 stages all eight B slices (64 KB) and
// streams the eight A slices through a 4-deep ring; TMEM holds 8 x 64 FP32
// group accumulators (all 512 columns).  Warp 0: TMA producer, warp 1: MMA
// issuer, warps 2-9: drain and epilogue (two per TMEM lane quarter, 32
// columns each).  All waits are bounded (EOD_ETIMEOUT
// on expiry).
#include "common.cuh"
#include "instrument.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstring>

namespace eod {
namespace oz {

using namespace eod::tc;

constexpr int NS = kOzSlices;         // slices per operand (8)
constexpr int NG = 8;                 // weight groups g = s + t, pairs with s + t <= 7
constexpr int BM = 128, BN = 64, BK = 64;
constexpr int KCH = 7;                // K blocks per exact chunk (448)
constexpr int kOzMaxChunks = 16;      // chunks one CTA accumulates in int64
static_assert(kOzMaxChunks * KCH * BK == kOzErrMaxK, "fused-error K limit");
constexpr int UMMA_K = 16;            // K per tcgen05.mma kind::f16
#ifndef OZ_ASTAGES
#define OZ_ASTAGES 2
#endif
#ifndef OZ_BSTAGES
#define OZ_BSTAGES 2
#endif
constexpr int ASTAGES = OZ_ASTAGES, BSTAGES = OZ_BSTAGES;
constexpr int A_TILE = BM * BK * 2;   // 16 KB: one slice
constexpr int APS = 2;                // A slices per pipeline stage (one wait and one commit each)
constexpr int A_STAGE = APS * A_TILE;
static_assert(kOzSlices % APS == 0, "slices per stage");
constexpr int B_TILE = BN * BK * 2;   // 8 KB
constexpr int B_SET = NS * B_TILE;    // 64 KB
constexpr int SMEM = BSTAGES * B_SET + ASTAGES * A_STAGE + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;   // 8 x 64 used
constexpr int NTHREADS = 320;        // producer, MMA issuer, 8 drain warps
constexpr int ECOLS = BN / 2;         // columns per drain warp

struct Maps {
    CUtensorMap a[NS];
    CUtensorMap b[NS];
};

struct Params {
    int64_t M, N;
    int64_t kblocks, kb_per_split;
    const int *ea, *eb;       // row exponents of op(A), column exponents of op(B) (or null:
    int ea_fixed, eb_fixed;   // then every row / column uses the fixed exponent)
    double alpha, beta;
    double *C;                // output (or split partials when split_stride > 0)
    float *Cf;                // FP32 output instead of C (EPI_STORE without split partials)
    int64_t ldc, split_stride;
    const double *R;          // EPI_ERR reference
    int64_t ldr;
    double *errp;
    int *err_flag;
    int upper_only;           // store only entries with row <= col
    int a_tri, b_tri;         // op(A) / op(B) upper triangular: skip their zero K blocks
};

// v 2^e: one multiply by a power of two built from its bits (exact unless
// the result leaves the normal range, where ldexp takes over)
__device__ __forceinline__ double pow2_scale(double v, int e) {
    if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(v, e);
}

template <int EPI>
__global__ void __launch_bounds__(NTHREADS, 1) oz_gemm_kernel(const __grid_constant__ Maps maps, Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bbuf = smem;                                 // BSTAGES x 7 B slices
    uint8_t *abuf = smem + BSTAGES * B_SET;                // ASTAGES stages of APS A slices
    uint64_t *fullB = (uint64_t *)(abuf + ASTAGES * A_STAGE);
    uint64_t *emptyB = fullB + BSTAGES;
    uint64_t *fullA = emptyB + BSTAGES;
    uint64_t *emptyA = fullA + ASTAGES;
    uint64_t *tmem_full = emptyA + ASTAGES;
    uint64_t *tmem_empty = tmem_full + 1;
    uint32_t *tmem_slot = (uint32_t *)(tmem_empty + 1);
    int *abort_sh = (int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    if (p.upper_only && m0 >= n0 + BN) return;   // every entry of the tile is below the diagonal
    int64_t kb0 = (int64_t)blockIdx.z * p.kb_per_split;
    int64_t kb1 = kb0 + p.kb_per_split;
    if (kb1 > p.kblocks) kb1 = p.kblocks;
    if (p.a_tri && kb0 < m0 / BK) kb0 = m0 / BK;              // op(A)(i, k) = 0 for k < i
    if (p.b_tri && kb1 > (n0 + BN + BK - 1) / BK) kb1 = (n0 + BN + BK - 1) / BK;   // op(B)(k, j) = 0 for k > j
    const int64_t nkb = kb1 > kb0 ? kb1 - kb0 : 0;
    const int64_t nchunks = (nkb + KCH - 1) / KCH;

    if (threadIdx.x == 0) {
        for (int i = 0; i < BSTAGES; ++i) { mbar_init(&fullB[i], 1); mbar_init(&emptyB[i], 1); }
        for (int i = 0; i < ASTAGES; ++i) { mbar_init(&fullA[i], 1); mbar_init(&emptyA[i], 1); }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, 256);
        *abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        // The whole warp runs the loop (waits and control flow stay
        // warp-uniform); one elected lane issues the copies.
        const bool leader = elect_one();
        int64_t ib = 0, ia = 0;
        bool ok = true;
        for (int64_t kb = kb0; kb < kb1 && ok; ++kb) {
            const int sb = (int)(ib % BSTAGES);
            if (ib >= BSTAGES) ok = warp_wait(&emptyB[sb], (uint32_t)((ib / BSTAGES - 1) & 1));
            if (ok && __any_sync(0xffffffffu, *(volatile int *)abort_sh != 0)) ok = false;
            if (!ok) break;
            if (leader) {
                mbar_expect_tx(&fullB[sb], B_SET);
                for (int t = 0; t < NS; ++t)
                    tma_load_2d(bbuf + sb * B_SET + t * B_TILE, &maps.b[t], &fullB[sb], (int)(kb * BK), (int)n0);
            }
            ++ib;
            for (int s0 = 0; s0 < NS && ok; s0 += APS) {
                const int sa = (int)(ia % ASTAGES);
                if (ia >= ASTAGES) ok = warp_wait(&emptyA[sa], (uint32_t)((ia / ASTAGES - 1) & 1));
                if (!ok) break;
                if (leader) {
                    mbar_expect_tx(&fullA[sa], A_STAGE);
                    for (int u = 0; u < APS; ++u)
                        tma_load_2d(abuf + sa * A_STAGE + u * A_TILE, &maps.a[s0 + u], &fullA[sa], (int)(kb * BK),
                                    (int)m0);
                }
                ++ia;
            }
            __syncwarp();
        }
        if (!ok && leader) { atomicExch(p.err_flag, 1); *abort_sh = 1; }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        // Warp-uniform loop, one elected lane issues: single-thread divergent
        // control flow around tcgen05 instructions slows their issue.
        // Fully unrolled over the 36 slice pairs and the 4 K steps of a
        // block: descriptors are a base plus constant offsets (the 16-byte
        // unit field advances by 2 per 32-byte K step and by 512 per 8 KB B
        // slice).
        const bool leader = elect_one();
        constexpr uint32_t idesc = idesc_bf16(BM, BN, false, false);
        int64_t ib = 0, ia = 0;
        bool ok = true;
        for (int64_t q = 0; q < nkb && ok; ++q) {
            const bool first = (q % KCH) == 0;
            if (first) {
                const int64_t chunk = q / KCH;
                if (chunk > 0) ok = warp_wait(tmem_empty, (uint32_t)((chunk - 1) & 1));
                if (!ok) break;
                tc_fence_after();
            }
            const int sb = (int)(ib % BSTAGES);
            ok = warp_wait(&fullB[sb], (uint32_t)((ib / BSTAGES) & 1));
            if (!ok) break;
            tc_fence_after();
            const uint64_t bd0 = sdesc(smem_u32(bbuf + sb * B_SET), 16, 1024);
            if (__any_sync(0xffffffffu, *(volatile int *)abort_sh != 0)) ok = false;
#pragma unroll
            for (int s0 = 0; s0 < NS; s0 += APS) {
                const int sa = (int)(ia % ASTAGES);
                if (ok) ok = warp_wait(&fullA[sa], (uint32_t)((ia / ASTAGES) & 1));
                if (ok) {
                    tc_fence_after();
                    if (leader) {
                        const uint64_t as0 = sdesc(smem_u32(abuf + sa * A_STAGE), 16, 1024);
#pragma unroll
                        for (int u = 0; u < APS; ++u) {
                            const int s = s0 + u;
                            const uint64_t ad0 = as0 + (uint64_t)(u * (A_TILE >> 4));
#pragma unroll
                            for (int t = 0; t < NG; ++t) {
                                if (s + t < NG) {
#pragma unroll
                                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                                        // the first MMA of a group in a chunk overwrites it
                                        const uint32_t accum = (first && s == 0 && kk == 0) ? 0u : 1u;
                                        umma_bf16(tmem + (uint32_t)((s + t) * BN), ad0 + (uint64_t)(2 * kk),
                                                  bd0 + (uint64_t)(512 * t + 2 * kk), idesc, accum);
                                    }
                                }
                            }
                        }
                        umma_commit(&emptyA[sa]);
                    }
                    __syncwarp();
                }
                ++ia;
            }
            if (!ok) break;
            if (leader) {
                umma_commit(&emptyB[sb]);
                if (q % KCH == KCH - 1 || q == nkb - 1) umma_commit(tmem_full);
            }
            __syncwarp();
            ++ib;
        }
        if (!ok && leader) {
            atomicExch(p.err_flag, 1);
            *abort_sh = 1;
            umma_commit(tmem_full);   // release the epilogue once the MMAs already issued finish
        }
    } else if (warp >= 2) {
        // ---------------- drain + epilogue ----------------
        const int qtr = warp & 3;                 // TMEM lane quarter this warp may read
        const int c0 = ((warp - 2) >> 2) * ECOLS; // its half of the 64 columns
        const int64_t row = m0 + 32 * qtr + lane;
        // Per chunk the eight FP32 group sums (exact integers) merge into one
        // int64 in units of 2^-50 of the row x column scale:
        //   hi = groups 0-3 in base 128 (unit 2^-33), lo = groups 4-7 (unit 2^-61),
        //   c  = hi 2^17 + round(lo 2^-11);
        // |hi| < 2^41.9 (|v_g| <= (g+1) 2^12 448), so |c| < 2^58.9 and up to
        // kOzMaxChunks = 16 chunks (the host splits K to respect that)
        // accumulate without overflow, rounding 2^-51 of the scale per chunk,
        // with no FP64 instruction in the drain.
        long long acc[ECOLS];
#pragma unroll
        for (int j = 0; j < ECOLS; ++j) acc[j] = 0;
        bool ok = true;
        for (int64_t c = 0; c < nchunks; ++c) {
            ok = __all_sync(0xffffffffu, mbar_wait(tmem_full, (uint32_t)(c & 1)) ? 1 : 0) != 0;
            if (!ok || *(volatile int *)abort_sh) { ok = false; break; }
            tc_fence_after();
            // 4 columns at a time: the 8 groups' loads are in flight together
#pragma unroll
            for (int cc = 0; cc < ECOLS; cc += 4) {
                uint32_t r[NG][4];
#pragma unroll
                for (int g = 0; g < NG; ++g)
                    tmem_ld4_nowait(tmem + ((uint32_t)(32 * qtr) << 16) + (uint32_t)(g * BN + c0 + cc), r[g]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    long long hi = 0, lo = 0;
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        const long long iv = (long long)__float2int_rn(__uint_as_float(r[g][j]));   // exact: |v| <= 2^24
                        if (g < 4) hi = hi * 128 + iv;
                        else lo = lo * 128 + iv;
                    }
                    acc[cc + j] += hi * 131072 + ((lo + (1ll << 10)) >> 11);
                }
            }
            tc_fence_before();
            mbar_arrive(tmem_empty);
        }
        if (!ok) atomicExch(p.err_flag, 1);
        double local = 0.0;
        if (row < p.M) {
            const int ei = p.ea ? max(p.ea[row], -1100) : p.ea_fixed;
            const bool unit_alpha = p.alpha == 1.0;
#pragma unroll
            for (int j = 0; j < ECOLS; ++j) {
                const int64_t col = n0 + c0 + j;
                if (col < p.N && !(p.upper_only && row > col)) {
                    const double val =
                        pow2_scale((double)acc[j], ei + (p.eb ? max(p.eb[col], -1100) : p.eb_fixed) - 50);
                    if (EPI == EPI_STORE) {
                        if (p.split_stride > 0) {
                            p.C[(int64_t)blockIdx.z * p.split_stride + row + col * p.M] = val;
                        } else if (p.Cf) {
                            double out = unit_alpha ? val : p.alpha * val;
                            if (p.beta != 0.0) out = fma(p.beta, (double)p.Cf[row + col * p.ldc], out);
                            p.Cf[row + col * p.ldc] = (float)out;
                        } else {
                            double out = unit_alpha ? val : p.alpha * val;
                            if (p.beta != 0.0) out = fma(p.beta, p.C[row + col * p.ldc], out);
                            p.C[row + col * p.ldc] = out;
                        }
                    } else {
                        const double d = fma(-p.alpha, val, p.R[row + col * p.ldr]);
                        local = fma(d, d, local);
                    }
                }
            }
        }
        if (EPI == EPI_ERR) {
            local = warp_sum(local);
            __shared__ double red[8];
            if (lane == 0) red[warp - 2] = local;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (warp == 2 && lane == 0) {
                double t = 0.0;
                for (int i = 0; i < 8; ++i) t += red[i];
                p.errp[blockIdx.x + (int64_t)blockIdx.y * gridDim.x] = t;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Triangular operands (the SIMT kernel's a_upper / b_upper): with tri == 1
// op(A) is upper triangular, X(r, k) = op(A)(r, k) is zero for r > k; with
// tri == 2 op(B) is, and X(r, k) = op(B)(k, r) is zero for k > r.  Those
// entries are never read.
__device__ __forceinline__ bool tri_zero(int tri, int64_t r, int64_t k) {
    return (tri == 1 && r > k) || (tri == 2 && k > r);
}

// |x| as its bit pattern (orders like the value for non-negative doubles);
// non-finite entries count as zero (the contraction expects finite data).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return (a >> 52) == 0x7ff ? 0ull : a;
}

// frexp exponent of the double with bit pattern a > 0 (a < 2^e)
__device__ __forceinline__ int exp_of_bits(unsigned long long a) {
    const int E = (int)(a >> 52);
    if (E > 0) return E - 1022;
    int ex;
    frexp(__longlong_as_double((long long)a), &ex);   // subnormal
    return ex;
}

constexpr int kExpZero = -2000000000;   // exponent of an all-zero row (< -1100)
constexpr int kMaxExpSplit = 16;        // K ranges of the row-exponent pass

// ep[z][r] = exponent of max |X(r, k)| over the z-th K range (frexp
// convention: max < 2^e), kExpZero if that range of the row is zero; blocks
// cover 32 rows x one K range, so every entry is written once (no atomics,
// no initialisation pass).  Integer compares of the bit patterns: no FP64
// arithmetic.
template <typename TX>
__global__ void rowexp_kernel(const TX *__restrict__ X, int64_t R, int64_t K, int64_t sr, int64_t sk,
                              int64_t kper, int tri, int *ep) {
    int *e = ep + (int64_t)blockIdx.y * R;
    __shared__ unsigned long long red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int64_t kb = (int64_t)blockIdx.y * kper;
    int64_t ke = kb + kper;
    if (ke > K) ke = K;
    if (sk == 1) {
        // K contiguous: lanes along k, warps over rows
        for (int rr = ty; rr < 32; rr += 8) {
            const int64_t r = r0 + rr;
            unsigned long long m = 0ull;
            if (r < R)
                for (int64_t k = kb + tx; k < ke; k += 32)
                    if (!tri_zero(tri, r, k)) m = max(m, abs_bits((double)X[r * sr + k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (tx == 0 && r < R) e[r] = m > 0ull ? exp_of_bits(m) : kExpZero;
        }
        return;
    }
    // rows contiguous: lanes along rows, warps split the K range
    const int64_t r = r0 + tx;
    unsigned long long mx = 0ull;
    if (r < R)
        for (int64_t k = kb + ty; k < ke; k += 8)
            if (!tri_zero(tri, r, k)) mx = max(mx, abs_bits((double)X[r + k * sk]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && r < R) {
        unsigned long long m = red[0][tx];
#pragma unroll
        for (int i = 1; i < 8; ++i) m = max(m, red[i][tx]);
        e[r] = m > 0ull ? exp_of_bits(m) : kExpZero;
    }
}

// The eight BF16 digits of x 2^-er into o[s * slice_stride] (see below).
__device__ __forceinline__ void write_slices(double x, int er, __nv_bfloat16 *o, int64_t slice_stride) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const bool neg = (bits >> 63) != 0;
    int E = (int)((bits >> 52) & 0x7ff);
    unsigned long long M = bits & 0xfffffffffffffull;
    if (E == 0x7ff) M = 0;               // non-finite: not representable, taken as zero
    else if (E == 0) E = 1;              // subnormal: M 2^(1 - 1075)
    else M |= 1ull << 52;                // |x| = M 2^(E - 1075)
    long long v = 0;
    const int sh = E - 1020 - er;        // v = M 2^sh; sh <= 2 since |x| < 2^er
    if (er >= -1100 && M != 0) {
        if (sh >= 0) v = (long long)(M << sh);
        else if (sh > -63) v = (long long)((M >> (-sh)) + ((M >> (-sh - 1)) & 1ull));
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int w = 49 - 7 * s;
        long long q;
        if (w > 0) q = (v + (1ll << (w - 1))) >> w;   // balanced digit: |q| <= 64
        else q = v;
        v -= q << w;
        const float qf = (float)(neg ? -q : q);
        o[s * slice_stride] = __float2bfloat16_rn(qf);
    }
}

// out[s][r * ldk + k] = slice s of X(r, k) 2^-e[r]; 32 x 32 tiles through
// shared memory so reads follow X's contiguous axis and writes follow k.
// Integer arithmetic on the bit pattern: v = round(|x| 2^(55 - e)) < 2^55 + 1
// is split into 8 balanced base-128 digits q_s in [-64, 64] (digit s has
// weight 2^(49 - 7 s)), so x = sign 2^(e - 55) sum_s q_s 2^(49 - 7 s) up to
// 2^(e - 56); every q_s is exact in BF16.
// The row exponents come from the nsplit partial ones of rowexp_kernel (the
// blocks of the first K column also store them in e_out for the product), or
// every row takes fixed_e when ep is null.
template <typename TX>
__global__ void slice_kernel(const TX *__restrict__ X, int64_t R, int64_t K, int64_t sr, int64_t sk,
                             int tri, const int *__restrict__ ep, int nsplit, int *__restrict__ e_out, int fixed_e,
                             __nv_bfloat16 *__restrict__ out, int64_t ldk, int64_t slice_stride) {
    __shared__ double tile[32][33];
    __shared__ int erow[32];
    const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    if (ty == 0) {
        const int64_t r = r0 + tx;
        int er = fixed_e;
        if (ep && r < R) {
            er = kExpZero;
            for (int z = 0; z < nsplit; ++z) er = max(er, ep[(int64_t)z * R + r]);
            if (blockIdx.x == 0 && e_out) e_out[r] = er;
        }
        erow[tx] = er;
    }
    for (int i = ty; i < 32; i += 8) {
        int64_t r, k;
        if (sk == 1) { r = r0 + i; k = k0 + tx; } else { r = r0 + tx; k = k0 + i; }
        const double v = (r < R && k < K && !tri_zero(tri, r, k)) ? (double)X[r * sr + k * sk] : 0.0;
        if (sk == 1) tile[i][tx] = v; else tile[tx][i] = v;   // tile[r - r0][k - k0]
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i, k = k0 + tx;
        if (r >= R || k >= K) continue;
        write_slices(tile[i][tx], erow[i], out + r * ldk + k, slice_stride);
    }
}

// Rows with K contiguous (sk == 1) and their own exponents, one CTA per row:
// the row maximum (as in rowexp_kernel) and then the slices (as in
// slice_kernel), in one launch; the second read of the row hits L1 / L2.
template <typename TX>
__global__ void __launch_bounds__(256) slice_rows_kernel(const TX *__restrict__ X, int64_t K, int64_t sr,
                                                         int tri, int *__restrict__ e_out,
                                                         __nv_bfloat16 *__restrict__ out, int64_t ldk,
                                                         int64_t slice_stride) {
    __shared__ unsigned long long red[8];
    __shared__ int er_sh;
    const int64_t r = blockIdx.x;
    const TX *x = X + r * sr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long m = 0ull;
    for (int64_t k = tid; k < K; k += 256)
        if (!tri_zero(tri, r, k)) m = max(m, abs_bits((double)x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (tid == 0) {
        unsigned long long t = red[0];
#pragma unroll
        for (int i = 1; i < 8; ++i) t = max(t, red[i]);
        const int er = t > 0ull ? exp_of_bits(t) : kExpZero;
        er_sh = er;
        e_out[r] = er;
    }
    __syncthreads();
    const int er = er_sh;
    __nv_bfloat16 *o = out + r * ldk;
    for (int64_t k = tid; k < K; k += 256)
        write_slices(tri_zero(tri, r, k) ? 0.0 : (double)x[k], er, o + k, slice_stride);
}

template <typename TC>
__global__ void split_sum_kernel(const double *__restrict__ part, int S, int64_t M, int64_t N, double alpha,
                                 double beta, TC *C, int64_t ldc, int upper_only) {
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % M, j = e / M;
        if (upper_only && i > j) continue;
        double sum = 0.0;
        for (int z = 0; z < S; ++z) sum += part[(int64_t)z * total + e];
        double out = alpha * sum;
        if (beta != 0.0) out = fma(beta, (double)C[i + j * ldc], out);
        C[i + j * ldc] = (TC)out;
    }
}

struct Slices {
    __nv_bfloat16 *q = nullptr;
    int *e = nullptr;
    int64_t R = 0, ldk = 0;
};

template <typename TX>
cudaError_t slice_into(const TX *X, int64_t R, int64_t K, int64_t sr, int64_t sk, __nv_bfloat16 *q, int *e,
                       int fixed_e, int64_t ldk, int64_t slice_stride, cudaStream_t s, int tri = 0) {
    if (R <= 0 || K <= 0) return cudaSuccess;
    ProfScope prof(PROF_OZ_SLICE, 0.0, (double)sizeof(TX) * R * K + 2.0 * NS * (double)R * K, s);
    if (e && sk == 1 && (R >= kNumSMs || K <= 8192)) {
        count_launch();
        slice_rows_kernel<<<(unsigned)R, 256, 0, s>>>(X, K, sr, tri, e, q, ldk, slice_stride);
        return cudaGetLastError();
    }
    int *ep = nullptr;
    int64_t ksplit = 1;
    if (e) {
        const int64_t rblocks = (R + 31) / 32;
        ksplit = (4 * kNumSMs + rblocks - 1) / rblocks;
        const int64_t kmax = (K + 255) / 256;
        if (ksplit > kmax) ksplit = kmax;
        if (ksplit > kMaxExpSplit) ksplit = kMaxExpSplit;
        if (ksplit < 1) ksplit = 1;
        const int64_t kper = (K + ksplit - 1) / ksplit;
        ksplit = (K + kper - 1) / kper;
        ep = e;   // one range: the partial exponents are the exponents
        if (ksplit > 1) EOD_CUDA_TRY(lib_malloc_async((void **)&ep, sizeof(int) * (size_t)ksplit * R, s));
        count_launch();
        rowexp_kernel<<<dim3((unsigned)rblocks, (unsigned)ksplit), 256, 0, s>>>(X, R, K, sr, sk, kper, tri, ep);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            if (ep != e) cudaFreeAsync(ep, s);
            return le;
        }
    }
    count_launch();
    dim3 grid((unsigned)((K + 31) / 32), (unsigned)((R + 31) / 32));
    slice_kernel<<<grid, dim3(32, 8), 0, s>>>(X, R, K, sr, sk, tri, ep, (int)ksplit, (ep && ep != e) ? e : nullptr,
                                               fixed_e, q, ldk, slice_stride);
    cudaError_t le = cudaGetLastError();
    if (ep && ep != e) cudaFreeAsync(ep, s);
    return le;
}

template <typename TX>
cudaError_t make_slices(const TX *X, int64_t R, int64_t K, int64_t sr, int64_t sk, Slices &sl, cudaStream_t s,
                        int tri = 0) {
    sl.R = R;
    sl.ldk = round_up(K, 8);
    EOD_CUDA_TRY(lib_malloc_async((void **)&sl.q, sizeof(__nv_bfloat16) * (size_t)NS * R * sl.ldk, s));
    EOD_CUDA_TRY(lib_malloc_async((void **)&sl.e, sizeof(int) * (size_t)R, s));
    return slice_into(X, R, K, sr, sk, sl.q, sl.e, 0, sl.ldk, R * sl.ldk, s, tri);
}

void free_slices(Slices &sl, cudaStream_t s) {
    if (sl.q) cudaFreeAsync(sl.q, s);
    if (sl.e) cudaFreeAsync(sl.e, s);
    sl.q = nullptr;
    sl.e = nullptr;
}

}  // namespace oz

// Slices of op(X) as `rows` x K with K contiguous (see oz_gemm.cu header).
cudaError_t oz_slice(const double *X, int64_t rows, int64_t K, int64_t sr, int64_t sk, void *q, int *e,
                     int fixed_e, int64_t ldk, int64_t slice_stride, cudaStream_t s) {
    return oz::slice_into(X, rows, K, sr, sk, (__nv_bfloat16 *)q, e, fixed_e, ldk, slice_stride, s);
}

cudaError_t oz_gemm_ops(const OzOperand &A, const OzOperand &B, int64_t M, int64_t N, int64_t K, double alpha,
                        double beta, double *C, int64_t ldc, const GemmExtra &x, int *err_flag, cudaStream_t s,
                        float *Cf) {
    using namespace oz;
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (Cf && x.epilogue != EPI_STORE) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    Maps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int i = 0; i < NS; ++i) {
        const __nv_bfloat16 *qa = (const __nv_bfloat16 *)A.q, *qb = (const __nv_bfloat16 *)B.q;
        if (!make_map(&maps.a[i], qa + (size_t)i * A.slice_stride, K, M, A.ldk, BK, BM) ||
            !make_map(&maps.b[i], qb + (size_t)i * B.slice_stride, K, N, B.ldk, BK, BN))
            return cudaErrorInvalidValue;
    }
    // exponents: a fixed exponent is passed as a one-entry array by the caller
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.M = M;
    p.N = N;
    p.kblocks = (K + BK - 1) / BK;
    p.ea = A.e;
    p.eb = B.e;
    p.alpha = alpha;
    p.beta = beta;
    p.err_flag = err_flag;
    p.R = (const double *)x.ref;
    p.ldr = x.ldref;
    p.errp = x.err_partials;
    p.ea_fixed = A.e_fixed;
    p.eb_fixed = B.e_fixed;
    p.upper_only = x.upper_only ? 1 : 0;
    p.a_tri = x.a_upper ? 1 : 0;
    p.b_tri = x.b_upper ? 1 : 0;
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    // K split until the grid covers the SMs, at least two K blocks per split
    // (a split's exact chunks start at its own first block)
    int64_t splits = 1;
    if (x.epilogue == EPI_STORE && tiles < kNumSMs) {
        splits = (kNumSMs + tiles - 1) / tiles;
        const int64_t smax = p.kblocks / 2;
        if (splits > smax) splits = smax;
        if (splits < 1) splits = 1;
    }
    // the drain's int64 accumulators hold at most kOzMaxChunks chunks of KCH blocks
    const int64_t smin = (p.kblocks + kOzMaxChunks * KCH - 1) / (kOzMaxChunks * KCH);
    if (smin > 1 && x.epilogue != EPI_STORE) return cudaErrorInvalidValue;   // K > kOzErrMaxK with a fused error
    if (splits < smin) splits = smin;
    p.kb_per_split = (p.kblocks + splits - 1) / splits;
    if (p.kb_per_split < 1) p.kb_per_split = 1;
    splits = (p.kblocks + p.kb_per_split - 1) / p.kb_per_split;
    if (splits < 1) splits = 1;
    double *part = nullptr;
    e = set_smem_once(oz_gemm_kernel<EPI_STORE>, SMEM);
    if (e == cudaSuccess) e = set_smem_once(oz_gemm_kernel<EPI_ERR>, SMEM);
    if (e == cudaSuccess && splits > 1) {
        e = lib_malloc_async((void **)&part, sizeof(double) * (size_t)splits * M * N, s);
        p.C = part;
        p.ldc = M;
        p.split_stride = M * N;
    } else {
        p.C = C;
        p.Cf = Cf;
        p.ldc = ldc;
        p.split_stride = 0;
    }
    // the method's flops: an upper-only output or a triangular operand halves
    // the multiply-adds (both triangular: a sixth), as the kernel skips them
    double frac = 1.0;
    if (x.upper_only) frac *= 0.5;
    if (x.a_upper && x.b_upper) frac /= 6.0;
    else if (x.a_upper || x.b_upper) frac *= 0.5;
    ProfScope prof(PROF_OZ_GEMM, 2.0 * M * N * K * frac,
                   2.0 * NS * ((double)M * K + (double)K * N) + 8.0 * 2 * M * N, s);
    if (e == cudaSuccess) {
        dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
        count_launch();
        if (x.epilogue == EPI_ERR) oz_gemm_kernel<EPI_ERR><<<grid, NTHREADS, SMEM, s>>>(maps, p);
        else oz_gemm_kernel<EPI_STORE><<<grid, NTHREADS, SMEM, s>>>(maps, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && splits > 1) {
        count_launch();
        const int blocks = (int)std::min<int64_t>((M * N + 255) / 256, 4LL * kNumSMs * 8);
        if (Cf) split_sum_kernel<float><<<blocks, 256, 0, s>>>(part, (int)splits, M, N, alpha, beta, Cf, ldc,
                                                                 p.upper_only);
        else split_sum_kernel<double><<<blocks, 256, 0, s>>>(part, (int)splits, M, N, alpha, beta, C, ldc,
                                                              p.upper_only);
        e = cudaGetLastError();
    }
    if (part) cudaFreeAsync(part, s);
    return e;
}

namespace oz {
template <typename T>
cudaError_t gemm_any(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const T *A, int64_t lda,
                     const T *B, int64_t ldb, double beta, double *C, float *Cf, int64_t ldc, const GemmExtra &x,
                     int *err_flag, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    Slices sa, sb;
    // op(A)(i, k): rows i, reduction k; op(B)(k, j) seen as rows j
    // a_upper / b_upper: op(A) / op(B) is upper triangular and its zero part
    // is not read, as in the SIMT kernel
    cudaError_t e = make_slices(A, M, K, ta ? lda : 1, ta ? 1 : lda, sa, s, x.a_upper ? 1 : 0);
    const bool same = (A == B) && (ta != tb) && (lda == ldb) && (M == N) && !x.a_upper && !x.b_upper;
    if (e == cudaSuccess && !same) e = make_slices(B, N, K, tb ? 1 : ldb, tb ? ldb : 1, sb, s, x.b_upper ? 2 : 0);
    const Slices &SB = same ? sa : sb;
    if (e == cudaSuccess) {
        OzOperand oa{sa.q, sa.e, 0, sa.ldk, (int64_t)M * sa.ldk};
        OzOperand ob{SB.q, SB.e, 0, SB.ldk, (int64_t)N * SB.ldk};
        e = oz_gemm_ops(oa, ob, M, N, K, alpha, beta, C, ldc, x, err_flag, s, Cf);
    }
    free_slices(sa, s);
    if (!same) free_slices(sb, s);
    return e;
}
}  // namespace oz

// C = alpha op(A) op(B) + beta C (EPI_STORE) or the squared error against
// x.ref (EPI_ERR), FP64, through the sliced tensor-core product.
cudaError_t oz_gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double beta, double *C, int64_t ldc, const GemmExtra &x,
                    int *err_flag, cudaStream_t s) {
    return oz::gemm_any<double>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, nullptr, ldc, x, err_flag, s);
}

// The same product of FP32 data (exact in FP64, so sliced the same way) with
// an FP32 result: C = alpha op(A) op(B) + beta C rounded once to FP32.
cudaError_t oz_gemm_f32(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const float *A, int64_t lda,
                        const float *B, int64_t ldb, double beta, float *C, int64_t ldc, const GemmExtra &x,
                        int *err_flag, cudaStream_t s) {
    if (x.epilogue != EPI_STORE) return cudaErrorInvalidValue;
    return oz::gemm_any<float>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, nullptr, C, ldc, x, err_flag, s);
}

int64_t oz_gemm_err_ctas(int64_t M, int64_t N) { return ((M + oz::BM - 1) / oz::BM) * ((N + oz::BN - 1) / oz::BN); }

}  // namespace eod

// The batched form in one persistent launch: many matrices of uneven sizes
// and ranks (the per-image use of Sec. 4.1) factored by a kernel whose CTAs
// take matrices from an atomic work queue, largest first, and run the whole
// method on each one without returning to the host: ||A||_F (the RelErr
// denominator, and eps in relative mode; summed from the tiles of the first
// sketch, which read every element once), Alg. 1 with its block loop and its
// stop decision on the device (Omega_j, Y = A Omega_j, Y <- (I - Q Q^T) Y
// twice, CholQR2 with the rank test folded into the first Cholesky, the
// explicit residual for undecided pivots), Alg. 2 steps 8-11 (C^T = A^T Q,
// C^T = V R, R^T = Qh D, U = Q Qh) and ||A - Q C||_F.
//
// One CTA (512 threads, one per SM) owns an item from start to end: a CTA
// never waits for another, so there is no inter-CTA wait of any kind.  The
// arithmetic is that of the FP32 forms of the single-matrix path: FP32
// products with FP32 accumulation, Grams formed from exact FP32 products
// summed by TwoSum into FP64 values, FP64 Cholesky (the same leaf
// factorisation, chol_leaf.cuh) and FP64 products of triangular factors.
//
// Capacity: an item keeps at most kPRcap = 128 basis columns (the core's
// Cholesky is one leaf of width r).  An item whose rank would exceed it, or
// whose core Gram is too ill-conditioned for unshifted CholQR, stops with
// kPFallback and the host factors it with the single-matrix path.
#include "common.cuh"
#include "chol_leaf.cuh"
#include "omega.cuh"
#include "instrument.cuh"
#include "batch.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <type_traits>
#include <vector>

namespace eod {
namespace {

constexpr int PT = kLeafThreads;   // threads per CTA (the leaf's CTA size)
static_assert(PT == 512, "the tile shapes below assume 512 threads");

// ------------------------------------------------------------ FP32 GEMM ----
// C = alpha op(A) op(B) + beta C on one CTA, FP32 accumulation.
//   op(A) M x K: TA = false: A(i, k) at A[i + k lda]; TA = true: A[k + i lda]
//   op(B) K x N: TB = false: B(k, j) at B[k + j ldb]; TB = true: B[j + k ldb]
// Tiles of BM x BN (BN = 64: 128 x 64; BN = 32: 256 x 32), K steps of 16
// through a three-stage ring of shared buffers filled by 4-byte cp.async
// copies (two steps in flight while one is multiplied; one barrier per
// step); each thread owns a 4 x 4 block of the tile.  ERR: no store; the thread adds
// (ref(i, j) - alpha acc(i, j))^2 to *ss instead (the reconstruction error,
// each square exact, summed by TwoSum; the ref tile is copied to shared
// memory, coalesced, while the K loop runs).  COMP: every four K steps the
// 64-term partial sum is added to a TwoSum pair (hi, lo) instead of running
// on in one FP32 accumulator, so a long dot product (K = m or n) carries the
// rounding of 64-term sums rather than of K-term ones: those errors, in the
// sketch and in the projections against Q, are what the singular-value
// decay amplifies into the basis (about u sqrt(K) s_1 / s_r).
constexpr int GK = 16;

// Exact FP32 products summed by TwoSum: s + c carries the sum of the exact
// products to about 2^-46 relative, at FP32 ALU rates.
struct TwoSumAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        const float t = s + p;
        const float z = t - s;
        const float err = (s - (t - z)) + (p - z);
        s = t;
        c += err + e;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};


constexpr int GS = 3;   // pipeline stages

constexpr int GFOLD = 4;   // K steps per compensated fold (64-term partial sums)

template <int BN, int TM, bool ERR>
__host__ __device__ constexpr int gemm_smem_floats() {
    // the stage ring, then (ERR) the reference tile, BN columns of BM + 4
    return GS * GK * ((PT / (BN / 4)) * TM + 4) + GS * GK * (BN + 4) + (ERR ? BN * ((PT / (BN / 4)) * TM + 4) : 0);
}

// one 4-byte asynchronous copy global -> shared, zero-filled when !valid
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int BN, bool TA, bool TB, bool ERR, bool COMP, int TM>
__device__ __noinline__ void cta_gemm(int M, int N, int K, float alpha, const float *__restrict__ A, int64_t lda,
                                      const float *__restrict__ B, int64_t ldb, float beta, float *C, int64_t ldc,
                                      const float *__restrict__ ref, int64_t ldref, TwoSumAcc *ss, float *sm,
                                      TwoSumAcc *nrm, int *nonfinite) {
    constexpr int TX = BN / 4, TY = PT / TX, BM = TY * TM;
    constexpr bool LO = COMP && TM == 4;   // a TwoSum pair per output; TM = 8 keeps one running FP32 sum
    constexpr int LAS = BM + 4, LBS = BN + 4;
    constexpr int AL = BM * GK / PT, BL = BN * GK / PT;
    float *As = sm;                     // [GS][GK][LAS]
    float *Bs = sm + GS * GK * LAS;     // [GS][GK][LBS]
    float *Rs = Bs + GS * GK * LBS;     // ERR: [BN][LAS], the tile of ref
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int nk = (K + GK - 1) / GK;
    TwoSumAcc nacc;                    // the norm's share of this thread, in registers
    int nbad = 0;
    for (int m0 = 0; m0 < M; m0 += BM) {
        for (int n0 = 0; n0 < N; n0 += BN) {
            float acc[TM][4], hi[COMP ? TM : 1][4], lo[LO ? TM : 1][4];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b] = 0.f;
                    if (COMP) hi[a][b] = 0.f;
                    if (LO) lo[a][b] = 0.f;
                }
            // stage t of the K loop into buffer t % GS: each thread copies
            // AL elements of the A tile and BL of the B tile, element (i, k)
            // of op(A) to As[k][i] and (k, j) of op(B) to Bs[k][j] (the
            // transposes happen in the addressing)
            // per-thread sources: element q of this thread's share of the A
            // tile sits at pa + q sa_q + t sa_k (B likewise)
            const int ia = TA ? tid / GK : tid % BM, ka = TA ? tid % GK : tid / BM;
            const int64_t sa_q = TA ? (int64_t)(PT / GK) * lda : (int64_t)(PT / BM) * lda;
            const int64_t sa_k = TA ? GK : (int64_t)GK * lda;
            const float *pa = TA ? A + ka + (int64_t)(m0 + ia) * lda : A + (m0 + ia) + (int64_t)ka * lda;
            const int jb = TB ? tid % BN : tid / GK, kb = TB ? tid / BN : tid % GK;
            const int64_t sb_q = TB ? (int64_t)(PT / BN) * ldb : (int64_t)(PT / GK) * ldb;
            const int64_t sb_k = TB ? (int64_t)GK * ldb : GK;
            const float *pb = TB ? B + (n0 + jb) + (int64_t)kb * ldb : B + kb + (int64_t)(n0 + jb) * ldb;
            auto issue = [&](int t) {
                const int k0 = t * GK, buf = t % GS;
                float *as = As + buf * GK * LAS, *bs = Bs + buf * GK * LBS;
                const float *a_t = pa + (int64_t)t * sa_k, *b_t = pb + (int64_t)t * sb_k;
#pragma unroll
                for (int q = 0; q < AL; ++q) {
                    const int i = TA ? ia + q * (PT / GK) : ia, kk = TA ? ka : ka + q * (PT / BM);
                    const bool v = m0 + i < M && k0 + kk < K;
                    cp_async4(as + kk * LAS + i, v ? a_t + q * sa_q : A, v);
                }
#pragma unroll
                for (int q = 0; q < BL; ++q) {
                    const int j = TB ? jb : jb + q * (PT / GK), kk = TB ? kb + q * (PT / BN) : kb;
                    const bool v = n0 + j < N && k0 + kk < K;
                    cp_async4(bs + kk * LBS + j, v ? b_t + q * sb_q : B, v);
                }
            };
            if (ERR) {
                // the reference tile, column by column (coalesced), in the
                // first stage's group: it lands while the K loop runs
                for (int e = tid; e < BM * BN; e += PT) {
                    const int i = e % BM, j = e / BM;
                    const bool v = m0 + i < M && n0 + j < N;
                    cp_async4(Rs + j * LAS + i, v ? ref + (m0 + i) + (int64_t)(n0 + j) * ldref : ref, v);
                }
            }
#pragma unroll
            for (int t = 0; t < GS - 1; ++t) {
                if (t < nk) issue(t);
                cp_async_commit();
            }
            for (int t = 0; t < nk; ++t) {
                cp_async_wait<GS - 2>();      // stage t has landed (this thread's copies)
                __syncthreads();              // ... everyone's; buffer (t - 1) % GS is free
                if (nrm) {
                    // the squares of the A elements this thread copied (zero
                    // outside A): with a single column tile every element of A
                    // passes through exactly once
                    const float *as = As + (t % GS) * GK * LAS;
#pragma unroll
                    for (int q = 0; q < AL; ++q) {
                        const int i = TA ? ia + q * (PT / GK) : ia, kk = TA ? ka : ka + q * (PT / BM);
                        const float v = as[kk * LAS + i];
                        nbad |= !isfinite(v);
                        nacc.add(v, v);
                    }
                }
                if (t + GS - 1 < nk) issue(t + GS - 1);
                cp_async_commit();
                const int buf = t % GS;
                const float *as = As + buf * GK * LAS + ty * TM, *bs = Bs + buf * GK * LBS + tx * 4;
#pragma unroll
                for (int kk = 0; kk < GK; ++kk) {
                    float av[TM];
#pragma unroll
                    for (int h = 0; h < TM / 4; ++h) {
                        const float4 a = *(const float4 *)(as + kk * LAS + 4 * h);
                        av[4 * h] = a.x;
                        av[4 * h + 1] = a.y;
                        av[4 * h + 2] = a.z;
                        av[4 * h + 3] = a.w;
                    }
                    const float4 b = *(const float4 *)(bs + kk * LBS);
                    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int x = 0; x < TM; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
                }
                if (COMP && ((t + 1) % GFOLD == 0 || t + 1 == nk)) {
#pragma unroll
                    for (int x = 0; x < TM; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            if (LO) {
                                const float a = hi[x][y], b = acc[x][y];
                                const float t2 = a + b, z = t2 - a;
                                lo[LO ? x : 0][y] += (a - (t2 - z)) + (b - z);
                                hi[x][y] = t2;
                            } else {
                                hi[x][y] += acc[x][y];
                            }
                            acc[x][y] = 0.f;
                        }
                }
            }
            cp_async_wait<0>();
            __syncthreads();                  // the buffers are reused by the next tile
#pragma unroll
            for (int x = 0; x < TM; ++x) {
                const int gi = m0 + ty * TM + x;
                if (gi >= M) continue;
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int gj = n0 + tx * 4 + y;
                    if (gj >= N) continue;
                    const float v = alpha * (COMP ? (LO ? hi[x][y] + lo[LO ? x : 0][y] : hi[x][y]) : acc[x][y]);
                    if (ERR) {
                        const float d = Rs[(tx * 4 + y) * LAS + ty * TM + x] - v;
                        ss->add(d, d);
                    } else {
                        float *c = C + gi + (int64_t)gj * ldc;
                        *c = (beta == 0.f) ? v : fmaf(beta, *c, v);
                    }
                }
            }
            if (ERR) __syncthreads();         // the next tile's reference copies overwrite Rs
        }
    }
    if (nrm) {
        // fold this call's share into the caller's accumulator
        const double v = nacc.value();
        const float h = (float)v;
        nrm->add(h, 1.f);
        nrm->add((float)(v - (double)h), 1.f);
        *nonfinite |= nbad;
    }
}

// op(A) op(B); COMP for the long dot products (K = m or n)
// With nrm (N <= 64: one column tile) the squares of every element of
// op(A) are also summed into *nrm and its finiteness ORed into *nonfinite.
template <bool TA, bool TB, bool COMP = false>
__device__ void cta_mm(int M, int N, int K, float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                       float beta, float *C, int64_t ldc, float *sm, TwoSumAcc *nrm = nullptr,
                       int *nonfinite = nullptr) {
    // whole 64-column tiles, then a remainder of at most 32 columns on the
    // narrow tile (N = 83 computes 96 columns, not 128)
    // 64-column tiles with 8-row register blocks (256 x 64 per CTA) when M
    // fills them, else 4-row ones (128 x 64); 32-column tiles keep 4-row
    // blocks (256 x 32: with 8 rows their 16 copies per thread and step spill)
    const int n64 = (N % 64 != 0 && N % 64 <= 32) ? N / 64 * 64 : N;
    if (n64 > 0) {
        if (M >= 192)
            cta_gemm<64, TA, TB, false, COMP, 8>(M, n64, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, 0, nullptr,
                                                 sm, nrm, nonfinite);
        else
            cta_gemm<64, TA, TB, false, COMP, 4>(M, n64, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, 0, nullptr,
                                                 sm, nrm, nonfinite);
    }
    if (n64 < N) {
        const float *Bn = TB ? B + n64 : B + (int64_t)n64 * ldb;
        cta_gemm<32, TA, TB, false, COMP, 4>(M, N - n64, K, alpha, A, lda, Bn, ldb, beta, C + (int64_t)n64 * ldc,
                                             ldc, nullptr, 0, nullptr, sm, nrm, nonfinite);
    }
    __syncthreads();
}

// S(0:M) = A^T z (A: K x M, ld lda): a warp per output, exact products
// summed by TwoSum per lane, then an FP64 warp sum
__device__ void cta_tmv(int M, int K, const float *__restrict__ A, int64_t lda, const float *__restrict__ z,
                        float *S) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < M; j += PT / 32) {
        TwoSumAcc a;
        const float *col = A + (int64_t)j * lda;
        for (int i = lane; i < K; i += 32) a.add(col[i], z[i]);
        const double v = warp_sum(a.value());
        if (lane == 0) S[j] = (float)v;
    }
    __syncthreads();
}

// z(0:m) -= A S (A: m x K, ld lda): a thread per row
__device__ void cta_mv_sub(int64_t m, int K, const float *__restrict__ A, int64_t lda, const float *__restrict__ S,
                           float *z) {
    for (int64_t i = threadIdx.x; i < m; i += PT) {
        float acc = 0.f;
        for (int l = 0; l < K; ++l) acc = fmaf(A[i + (int64_t)l * lda], S[l], acc);
        z[i] -= acc;
    }
    __syncthreads();
}

// ------------------------------------------------------------ FP64 Gram ----
// G = Y^T Y (w x w, w <= 128, upper triangle with the diagonal blocks whole,
// ld ldg) for FP32 Y (rows x w, ld ldy): every product formed exactly as
// p + e (e = fma(a, b, -p)), the p's summed with TwoSum, the e's and the
// TwoSum errors in FP32, converted to FP64 per thread; thread groups taking
// every groups-th row are combined in a fixed order.  Rows are staged in
// chunks of 32 (row-major, odd stride) in shared memory.
constexpr int GRC = 32;   // rows per staged chunk

__host__ __device__ constexpr size_t gram_smem_bytes() {
    return sizeof(float) * GRC * (kPRcap + 1) + sizeof(double) * PT * 16;
}

__device__ __forceinline__ void block_of(int b, int &bi, int &bj) {
    int j = (int)((sqrtf(8.f * b + 1.f) - 1.f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= b) ++j;
    while (j * (j + 1) / 2 > b) --j;
    bi = b - j * (j + 1) / 2;
    bj = j;
}

__device__ __noinline__ void cta_gram(const float *__restrict__ Y, int64_t rows, int w, int64_t ldy, double *G,
                                      int ldg, unsigned char *smraw) {
    float *sY = (float *)smraw;                                   // GRC x (w + 1)
    double *red = (double *)(smraw + sizeof(float) * GRC * (kPRcap + 1));
    const int ld = w + 1;
    const int nb4 = (w + 3) / 4, nblocks = nb4 * (nb4 + 1) / 2;   // <= 528
    const int tid = threadIdx.x;
    // sweeps of at most PT blocks, one block per thread (two sweeps only
    // above w = 124); a sweep of at most PT / 2 blocks splits the rows
    // among groups of threads instead
    for (int sb = 0; sb < nblocks; sb += PT) {
        const int nbs = nblocks - sb < PT ? nblocks - sb : PT;
        const int groups = nbs <= PT / 2 ? PT / nbs : 1;
        const int grp = tid / nbs;
        const bool active = grp < groups;
        int bi = 0, bj = 0;
        if (active) block_of(sb + tid % nbs, bi, bj);
        const int i0 = 4 * bi, j0 = 4 * bj;
        TwoSumAcc acc[4][4];
        for (int64_t c0 = 0; c0 < rows; c0 += GRC) {
            const int cnt = (int)((rows - c0) < GRC ? (rows - c0) : GRC);
            __syncthreads();
            for (int e = tid; e < GRC * w; e += PT) {
                const int r = e % GRC, c = e / GRC;
                sY[r * ld + c] = (r < cnt) ? Y[(c0 + r) + (int64_t)c * ldy] : 0.f;
            }
            __syncthreads();
            if (active) {
                for (int r = grp; r < cnt; r += groups) {
                    const float *row = sY + r * ld;
                    float a[4], b[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        a[t] = (i0 + t < w) ? row[i0 + t] : 0.f;
                        b[t] = (j0 + t < w) ? row[j0 + t] : 0.f;
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y].add(a[x], b[y]);
                }
            }
        }
        if (groups > 1) {
            // the row groups combined in a fixed order
            if (active) {
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) red[((size_t)grp * nbs + tid % nbs) * 16 + x * 4 + y] = acc[x][y].value();
            }
            __syncthreads();
            for (int e = tid; e < nbs * 16; e += PT) {
                const int blk = e / 16, x = (e % 16) / 4, y = e % 4;
                double sum = 0.0;
                for (int g = 0; g < groups; ++g) sum += red[((size_t)g * nbs + blk) * 16 + x * 4 + y];
                int ib, jb;
                block_of(sb + blk, ib, jb);
                if (4 * ib + x < w && 4 * jb + y < w) G[(4 * ib + x) + (int64_t)(4 * jb + y) * ldg] = sum;
            }
        } else if (tid < nbs) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y)
                    if (i0 + x < w && j0 + y < w) G[(i0 + x) + (int64_t)(j0 + y) * ldg] = acc[x][y].value();
        }
    }
    __syncthreads();
}

// --------------------------------------------------------- small helpers ----
// FP64 sum of squares of a vector of FP32 values
__device__ double cta_norm2(const float *z, int64_t m, double *red) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += PT) acc = fma((double)z[i], (double)z[i], acc);
    return block_sum(acc, red);
}

// Dst (p x p, FP32) = Src or Src^T (FP64), zeros kept
__device__ void cta_to_f32(const double *Src, int lds, int p, float *Dst, int ldd, bool transpose) {
    for (int e = threadIdx.x; e < p * p; e += PT) {
        const int i = e % p, j = e / p;
        Dst[i + j * ldd] = (float)(transpose ? Src[j + i * lds] : Src[i + j * lds]);
    }
    __syncthreads();
}

// C = A B for upper triangular p x p FP64 factors (C upper, zeros below)
__device__ void cta_triu_mul(const double *A, int lda, const double *B, int ldb, double *C, int ldc, int p) {
    for (int e = threadIdx.x; e < p * p; e += PT) {
        const int i = e % p, j = e / p;
        double s = 0.0;
        for (int l = i; l <= j; ++l) s = fma(A[i + l * lda], B[l + j * ldb], s);
        C[i + j * ldc] = s;
    }
    __syncthreads();
}

// Omega_j (n x f, ld n) in FP32: the same draws as the streaming fill
__device__ void cta_omega(int64_t n, int64_t col0, int f, uint64_t seed, uint32_t batch, float *Om) {
    const int64_t tot = n * f;
    for (int64_t e = threadIdx.x; e < tot; e += PT) {
        const int64_t c = e / n, i = e - c * n;
        Om[e] = omega_value_fast<float>(seed, (uint32_t)i, (uint32_t)(col0 + c), batch);
    }
    __syncthreads();
}

// ---------------------------------------------------------- the kernel ----
struct PItem {
    const float *A;
    int64_t m, n, lda;
    float *Q, *C, *U, *V;     // m x cap, n x cap, m x cap, n x cap (ld m, n, m, n)
    double *D;                // r x r, ld r
    int64_t cap;              // min(m, n, kPRcap)
    uint32_t batch;           // Omega's third counter word (the item's index)
};

struct PRes {
    int32_t status, rank, blocks, restarts, ntdiag, pad;
    double norm_a, eps, rel_err;
};

struct PParams {
    const PItem *items;
    const int32_t *order;     // queue order: largest first
    PRes *res;
    double *tdiag;            // count x kPTdCap
    unsigned char *scratch;   // one region per CTA
    int64_t stride, mmax, nmax;
    unsigned *next;           // the single CTAs' queue counter (items npair .. count-1)
    unsigned *pair_next;      // the pairs' queue counter (items 0 .. npair-1)
    unsigned *team_bar;       // per cluster: its team barrier counter
    int *team_slot;           // per cluster: the item its pair took
    int *err;                 // set when a team barrier ran out
    float *xf;                // per cluster: the team's exchange slots
    double *xd;
    unsigned long long *phase;   // null, or kPPhases cycle counters summed over items (measurement)
    int count, npair, k, tol_mode, compute_err;
    double tol;
    uint64_t seed;
};

// per-CTA scratch: FP64 k x k / r x r factors first, then the FP32 panels
struct PLayout {
    int64_t g, r1, r1i, r2, r2i, rc;            // doubles
    int64_t y, yw, t1, om, sp, w, rf, rtf, w2, qh;  // floats, after the doubles
    int64_t dbytes, bytes;
};

__host__ __device__ inline PLayout playout(int64_t mmax, int64_t nmax) {
    auto up = [](int64_t x) { return (x + 63) / 64 * 64; };
    PLayout L;
    const int64_t rr = (int64_t)kPRcap * kPRcap;
    L.g = 0;
    L.r1 = L.g + rr;
    L.r1i = L.r1 + rr;
    L.r2 = L.r1i + rr;
    L.r2i = L.r2 + rr;
    L.rc = L.r2i + rr;
    L.dbytes = (L.rc + rr) * (int64_t)sizeof(double);
    L.y = 0;
    L.yw = L.y + up(mmax * kPKmax);
    L.t1 = L.yw + up(mmax * kPKmax);
    L.om = L.t1 + up(mmax * kPKmax);
    L.sp = L.om + up(nmax * kPKmax);
    L.w = L.sp + up((int64_t)kPRcap * kPKmax);
    L.rf = L.w + up(nmax * kPRcap);
    L.rtf = L.rf + rr;
    L.w2 = L.rtf + rr;
    L.qh = L.w2 + rr;
    L.bytes = L.dbytes + (L.qh + rr) * (int64_t)sizeof(float);
    L.bytes = (L.bytes + 255) / 256 * 256;
    return L;
}

__device__ __noinline__ void leaf(const double *G, int w, int decide, double eps2, double delta_coef, double rho,
                                     double *R, double *Ri, int *info, double ni_tau2, unsigned char *sm) {
    chol_leaf_cta<true>(G, kPRcap, w, decide, eps2, delta_coef, rho, 0.0, R, kPRcap, Ri, kPRcap, info, ni_tau2,
                        (double *)sm);
    __syncthreads();
}
// Per-phase cycle accounting of the measurement hook: thread 0 adds the
// SM clock ticks since the previous mark to the phase's counter.
enum PPhase { PH_NORM, PH_OMEGA, PH_SKETCH, PH_DEFLATE, PH_GRAM_LEAF, PH_PANEL, PH_RESIDUAL, PH_PROJECT, PH_ERR,
              PH_CORE, PH_U };
struct PhaseClock {
    unsigned long long *ctr;
    long long t;
    __device__ __forceinline__ void start(unsigned long long *c) {
        ctr = c;
        t = c ? (long long)clock64() : 0;
    }
    __device__ __forceinline__ void mark(int ph) {
        if (!ctr) return;
        const long long now = (long long)clock64();
        if (threadIdx.x == 0) atomicAdd(ctr + ph, (unsigned long long)(now - t));
        t = now;
    }
};

// ----------------------------------------------------------------- teams ----
// A team of one CTA, or of the two CTAs of a cluster, runs one item: the two
// split the rows of m (Alg. 1, U, the error) and of n (C, the core's tall
// panels); what spans the rows (Q^T Y, the Grams, norms, the error sum) is
// summed over the ranks in rank order through a per-team exchange buffer, so
// both ranks hold bit-identical values, run the leaf on identical Grams and
// take every decision alike.  A team of one skips the exchange.
constexpr long long kTeamWait = 4000000000ll;   // cycles (~2 s) a team barrier waits at most
constexpr double kPairFrac = 0.5;                // items with m n >= this x the largest go to pairs
constexpr int kXF = kPRcap * kPKmax;             // floats per exchange slot
constexpr int kXD = kPRcap * kPRcap + 8;         // doubles per exchange slot

struct Team {
    int rank, size;
    unsigned *bar;        // the team's barrier counter (zeroed by the launch)
    unsigned epoch;       // barriers this CTA has passed
    unsigned xchg;        // exchanges done (the slot parity)
    float *xf;            // [2 parities][2 ranks][kXF]
    double *xd;           // [2 parities][2 ranks][kXD]
    int *err;             // set when a wait ran out
    __device__ int64_t lo(int64_t M) const { return M * rank / size; }
    __device__ int64_t hi(int64_t M) const { return M * (rank + 1) / size; }
};

// barrier of the team (every thread calls); false when the wait ran out
__device__ bool team_sync(Team &t) {
    __syncthreads();
    if (t.size == 1) return true;
    __shared__ int ok_sh;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned target = (unsigned)t.size * (t.epoch + 1);
        atomicAdd(t.bar, 1u);
        const long long t0 = clock64();
        int ok = 1;
        while (*(volatile unsigned *)t.bar < target) {
            if (clock64() - t0 > kTeamWait) {
                ok = 0;
                atomicExch(t.err, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    ++t.epoch;
    return ok_sh != 0;
}

// v[i * ldv + j] (i < rows, j < cols) becomes the sum over the ranks (rank
// order); false when the team barrier ran out
template <typename T>
__device__ bool team_sum(Team &t, T *v, int rows, int cols, int ldv) {
    if (t.size == 1) return true;
    __syncthreads();
    const unsigned par = t.xchg & 1u;
    ++t.xchg;
    const int slot = std::is_same<T, float>::value ? kXF : kXD;
    T *x = std::is_same<T, float>::value ? (T *)t.xf : (T *)t.xd;
    T *mine = x + ((size_t)par * 2 + t.rank) * slot;
    for (int e = threadIdx.x; e < rows * cols; e += PT) mine[e] = v[(e % rows) + (e / rows) * ldv];
    if (!team_sync(t)) return false;
    const T *x0 = x + (size_t)par * 2 * slot, *x1 = x0 + slot;
    for (int e = threadIdx.x; e < rows * cols; e += PT) v[(e % rows) + (e / rows) * ldv] = x0[e] + x1[e];
    __syncthreads();
    return true;
}

// One matrix, start to end, on a team of one or two CTAs (rows of m and n
// split between the ranks).  Returns false when a team barrier ran out (the
// item then reports EOD_ETIMEOUT and the CTA leaves the kernel).
__device__ __noinline__ bool batch_item(const PParams &P, int idx, Team &T, unsigned char *sm, int *info, double *red) {
    const PItem it = P.items[idx];
    PRes *res = P.res + idx;
    double *tdg = P.tdiag + (int64_t)idx * kPTdCap;
    const int tid = threadIdx.x;
    const bool lead = T.rank == 0;   // the rank that writes the item's shared results
    const int64_t m = it.m, n = it.n, lda = it.lda;
    const int64_t mlo = T.lo(m), ml = T.hi(m) - mlo;   // this rank's rows of m
    const int64_t nlo = T.lo(n), nl = T.hi(n) - nlo;   // and of n
    const PLayout L = playout(P.mmax, P.nmax);
    unsigned char *base = P.scratch + (int64_t)blockIdx.x * P.stride;
    double *G = (double *)base + L.g, *R1 = (double *)base + L.r1, *R1i = (double *)base + L.r1i;
    double *R2 = (double *)base + L.r2, *R2i = (double *)base + L.r2i, *Rc = (double *)base + L.rc;
    float *fb = (float *)(base + L.dbytes);
    float *Y = fb + L.y, *Yw = fb + L.yw, *T1 = fb + L.t1, *Om = fb + L.om, *S = fb + L.sp, *W = fb + L.w;
    float *Rf = fb + L.rf, *Rtf = fb + L.rtf, *W2 = fb + L.w2, *Qh = fb + L.qh;
    float *smf = (float *)sm;
    __shared__ double dsum[2];
    constexpr double kNearId = 4e-8;   // ||G - I||_F^2 below which R = I + Phi(G - I) (FP32 panels)

    int kept = 0, blocks = 0, restarts = 0, ntd = 0;
    double eps = 0.0, norm = 0.0;
    auto finish = [&](int status, double rel) {
        if (tid == 0 && lead) {
            res->status = status;
            res->rank = kept;
            res->blocks = blocks;
            res->restarts = restarts;
            res->ntdiag = ntd;
            res->norm_a = norm;
            res->eps = eps;
            res->rel_err = rel;
        }
    };
    // a value summed over the team's ranks (FP64, rank order)
    auto tsum1 = [&](double v, double *out) -> bool {
        if (tid == 0) dsum[0] = v;
        __syncthreads();
        if (!team_sum<double>(T, dsum, 1, 1, 1)) return false;
        *out = dsum[0];
        __syncthreads();
        return true;
    };
#define TEAM_OK(call)                              \
    do {                                           \
        if (!(call)) {                             \
            finish(EOD_ETIMEOUT, -1.0);            \
            return false;                          \
        }                                          \
    } while (0)

    PhaseClock pc;
    pc.start(P.phase);

    // ---- Alg. 1 ----
    const int64_t cap = m < n ? m : n;
    double eps2 = 0.0;
    const double delta_coef = 64.0 * ((double)P.k + sqrt((double)m)) * kU64;
    const double rho = 1e-6;
    bool stop = false;
    // sketch window: Yw holds (this rank's rows of) A Omega for global columns
    // win_c0 .. win_c0 + win_w - 1; a pass over A computes two blocks at once
    // when k <= 32 (the second is wasted only if the rank is revealed in the
    // first)
    int64_t win_c0 = -1;
    int win_w = 0;
    while (!stop && kept < cap) {
        const int f = (int)((int64_t)P.k < cap - kept ? (int64_t)P.k : cap - kept);
        ++blocks;
        if (win_c0 < 0 || kept < win_c0 || kept + f > win_c0 + win_w) {
            int64_t w = 2 * (int64_t)P.k <= kPKmax ? 2 * (int64_t)P.k : (int64_t)P.k;
            w = w < cap - kept ? w : cap - kept;
            win_c0 = kept;
            win_w = (int)w;
            cta_omega(n, kept, win_w, P.seed, it.batch, Om);                                // step 3
            pc.mark(PH_OMEGA);
            if (blocks == 1) {
                // the first sketch reads every element of A once: ||A||_F and
                // the finiteness check come from its shared-memory tiles
                TwoSumAcc nrm;
                int nf = 0;
                cta_mm<false, false, true>((int)ml, win_w, (int)n, 1.f, it.A + mlo, lda, Om, n, 0.f, Yw + mlo, m, smf,
                                           &nrm, &nf);
                const int bad_local = __syncthreads_or(nf);
                const double part = block_sum(nrm.value(), red);
                double tot = 0.0, badsum = 0.0;
                TEAM_OK(tsum1(part, &tot));
                TEAM_OK(tsum1((double)bad_local, &badsum));
                norm = sqrt(tot);
                pc.mark(PH_SKETCH);
                if (badsum != 0.0) { finish(EOD_ENONFINITE, -1.0); return true; }
                eps = P.tol_mode == EOD_TOL_REL_FRO ? P.tol * norm : P.tol;
                eps2 = eps * eps;
                // below this the FP32 rounding of the sketch reaches |T(l,l)|:
                // refused, as the single-matrix FP32 forms do
                if (norm > 0.0 && eps < kPF32Floor * norm) { finish(EOD_EPRECISION, -1.0); return true; }
                if (norm == 0.0) {
                    if (tid == 0 && lead) tdg[0] = 0.0;
                    ntd = 1;
                    blocks = 0;
                    finish(EOD_OK, P.compute_err ? 0.0 : -1.0);
                    return true;
                }
            } else {
                cta_mm<false, false, true>((int)ml, win_w, (int)n, 1.f, it.A + mlo, lda, Om, n, 0.f, Yw + mlo, m, smf);
                pc.mark(PH_SKETCH);
            }
        }
        {   // Y = the window's columns of this block (this rank's rows)
            const int64_t tot = (int64_t)f * ml;
            for (int64_t e = tid; e < tot; e += PT) {
                const int64_t c = e / ml, i = mlo + (e - c * ml);
                Y[i + c * m] = Yw[i + (kept - win_c0 + c) * m];
            }
            __syncthreads();
        }
        int cur = 0;
        while (!stop && cur < f) {
            float *Yc = Y + (int64_t)cur * m;
            const int wdt = f - cur;
            for (int pass = 0; pass < 2 && kept > 0; ++pass) {                             // step 4, twice
                cta_mm<true, false, true>(kept, wdt, (int)ml, 1.f, it.Q + mlo, m, Yc + mlo, m, 0.f, S, kPRcap, smf);
                TEAM_OK(team_sum<float>(T, S, kept, wdt, kPRcap));
                cta_mm<false, false>((int)ml, wdt, kept, -1.f, it.Q + mlo, m, S, kPRcap, 1.f, Yc + mlo, m, smf);
            }
            pc.mark(PH_DEFLATE);
            cta_gram(Yc + mlo, ml, wdt, m, G, kPRcap, sm);                                   // step 5, pass 1
            TEAM_OK(team_sum<double>(T, G, wdt, wdt, kPRcap));
            leaf(G, wdt, 1, eps2, delta_coef, rho, R1, R1i, info, 0.0, sm);                    // steps 6-11
            pc.mark(PH_GRAM_LEAF);
            const int p = info[0], code = info[1];
            __syncthreads();
            if (p > 0) {
                if (kept + p > it.cap) { finish(kPFallback, -1.0); return true; }
                cta_to_f32(R1i, kPRcap, p, Rf, kPRcap, false);
                cta_mm<false, false>((int)ml, p, p, 1.f, Yc + mlo, m, Rf, kPRcap, 0.f, T1 + mlo, m, smf);
                cta_gram(T1 + mlo, ml, p, m, G, kPRcap, sm);                                 // pass 2
                TEAM_OK(team_sum<double>(T, G, p, p, kPRcap));
                leaf(G, p, 0, 0.0, 0.0, 0.0, R2, R2i, info, kNearId, sm);
                const int p2 = info[0], c2 = info[1];
                __syncthreads();
                if (p2 != p || c2 != CHOL_ALL) { finish(kPFallback, -1.0); return true; }
                cta_to_f32(R2i, kPRcap, p, Rf, kPRcap, false);
                cta_mm<false, false>((int)ml, p, p, 1.f, T1 + mlo, m, Rf, kPRcap, 0.f, it.Q + (int64_t)kept * m + mlo, m,
                                     smf);
                if (lead)
                    for (int l = tid; l < p; l += PT) tdg[ntd + l] = fabs(R1[l + l * kPRcap] * R2[l + l * kPRcap]);
                ntd += p;
                kept += p;
                pc.mark(PH_PANEL);
            }
            if (code == CHOL_ALL) {
                cur = f;
            } else {
                // column p: its explicit residual after two more projections
                float *z = Yc + (int64_t)p * m;
                for (int pass = 0; pass < 2 && kept > 0; ++pass) {
                    cta_tmv(kept, (int)ml, it.Q + mlo, m, z + mlo, S);
                    TEAM_OK(team_sum<float>(T, S, kept, 1, kPRcap));
                    cta_mv_sub(ml, kept, it.Q + mlo, m, S, z + mlo);
                }
                double t2 = 0.0;
                TEAM_OK(tsum1(cta_norm2(z + mlo, ml, red), &t2));
                const double t = sqrt(t2);
                pc.mark(PH_RESIDUAL);
                if (tid == 0 && lead) tdg[ntd] = t;
                ++ntd;
                if (code == CHOL_BELOW) {
                    stop = true;
                } else {
                    ++restarts;
                    if (!(t > eps)) {
                        stop = true;
                    } else {
                        if (kept + 1 > it.cap) { finish(kPFallback, -1.0); return true; }
                        const double inv = 1.0 / t;
                        float *q = it.Q + (int64_t)kept * m;
                        for (int64_t i = mlo + tid; i < mlo + ml; i += PT) q[i] = (float)((double)z[i] * inv);
                        __syncthreads();
                        kept += 1;
                        cur += p + 1;
                    }
                }
            }
        }
    }
    const int r = kept;
    if (r == 0) { finish(EOD_OK, P.compute_err ? 1.0 : -1.0); return true; }

    // ---- Alg. 2 step 8: C (n x r) = A^T Q, this rank's rows of n (all of Q) ----
    TEAM_OK(team_sync(T));
    cta_mm<true, false, true>((int)nl, r, (int)m, 1.f, it.A + nlo * lda, lda, it.Q, m, 0.f, it.C + nlo, n, smf);
    pc.mark(PH_PROJECT);
    TEAM_OK(team_sync(T));   // every row of C before the error and the core read them
    double rel = -1.0;
    if (P.compute_err) {                                                   // ||A - Q C^T||_F / ||A||_F
        TwoSumAcc ssq;
        cta_gemm<64, false, true, true, false, 8>((int)ml, (int)n, r, 1.f, it.Q + mlo, m, it.C, n, 0.f, nullptr, 0,
                                                  it.A + mlo, lda, &ssq, smf, nullptr, nullptr);
        double e2 = 0.0;
        TEAM_OK(tsum1(block_sum(ssq.value(), red), &e2));
        rel = sqrt(e2) / norm;
    }
    pc.mark(PH_ERR);

    // ---- steps 9-10: C^T = V R (rows of n split), then R^T = Qh D (r x r, on every rank) ----
    cta_gram(it.C + nlo, nl, r, n, G, kPRcap, sm);
    TEAM_OK(team_sum<double>(T, G, r, r, kPRcap));
    leaf(G, r, 0, 0.0, 0.0, 0.0, R1, R1i, info, 0.0, sm);
    if (info[0] != r || info[1] != CHOL_ALL) { finish(kPFallback, -1.0); return true; }
    cta_to_f32(R1i, kPRcap, r, Rf, kPRcap, false);
    cta_mm<false, false>((int)nl, r, r, 1.f, it.C + nlo, n, Rf, kPRcap, 0.f, W + nlo, n, smf);
    cta_gram(W + nlo, nl, r, n, G, kPRcap, sm);
    TEAM_OK(team_sum<double>(T, G, r, r, kPRcap));
    leaf(G, r, 0, 0.0, 0.0, 0.0, R2, R2i, info, kNearId, sm);
    if (info[0] != r || info[1] != CHOL_ALL) { finish(kPFallback, -1.0); return true; }
    cta_to_f32(R2i, kPRcap, r, Rf, kPRcap, false);
    cta_mm<false, false>((int)nl, r, r, 1.f, W + nlo, n, Rf, kPRcap, 0.f, it.V + nlo, n, smf);
    cta_triu_mul(R2, kPRcap, R1, kPRcap, Rc, kPRcap, r);                  // R = R2 R1

    cta_to_f32(Rc, kPRcap, r, Rtf, kPRcap, true);                         // R^T
    cta_gram(Rtf, r, r, kPRcap, G, kPRcap, sm);
    leaf(G, r, 0, 0.0, 0.0, 0.0, R1, R1i, info, 0.0, sm);
    if (info[0] != r || info[1] != CHOL_ALL) { finish(kPFallback, -1.0); return true; }
    cta_to_f32(R1i, kPRcap, r, Rf, kPRcap, false);
    cta_mm<false, false>(r, r, r, 1.f, Rtf, kPRcap, Rf, kPRcap, 0.f, W2, kPRcap, smf);
    cta_gram(W2, r, r, kPRcap, G, kPRcap, sm);
    leaf(G, r, 0, 0.0, 0.0, 0.0, R2, R2i, info, kNearId, sm);
    if (info[0] != r || info[1] != CHOL_ALL) { finish(kPFallback, -1.0); return true; }
    cta_to_f32(R2i, kPRcap, r, Rf, kPRcap, false);
    cta_mm<false, false>(r, r, r, 1.f, W2, kPRcap, Rf, kPRcap, 0.f, Qh, kPRcap, smf);
    if (lead) cta_triu_mul(R2, kPRcap, R1, kPRcap, it.D, r, r);          // D = R2 R1 of this pair
    pc.mark(PH_CORE);

    // ---- step 11: U = Q Qh (this rank's rows of m) ----
    cta_mm<false, false>((int)ml, r, r, 1.f, it.Q + mlo, m, Qh, kPRcap, 0.f, it.U + mlo, m, smf);
    pc.mark(PH_U);
    finish(EOD_OK, rel);
    return true;
#undef TEAM_OK
}

// Pairs first: the two CTAs of each cluster take the P.npair largest items
// together from their own queue; then every CTA alone takes the rest.  A
// team barrier that ran out ends the CTA (its partner's next wait runs out
// too), with the error flag set for the host.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PT, 1) batch_kernel(PParams P) {
    extern __shared__ __align__(16) unsigned char psm[];
    __shared__ int item_sh;
    __shared__ int info_sh[2];
    __shared__ double red_sh[32];
    const int team_id = blockIdx.x >> 1;
    Team T;
    T.err = P.err;
    T.epoch = 0;
    T.xchg = 0;
    T.xf = P.xf + (size_t)team_id * 4 * kXF;
    T.xd = P.xd + (size_t)team_id * 4 * kXD;
    T.bar = P.team_bar + team_id;
    if (P.npair > 0) {
        T.rank = (int)(blockIdx.x & 1);
        T.size = 2;
        for (;;) {
            if (T.rank == 0 && threadIdx.x == 0) P.team_slot[team_id] = (int)atomicAdd(P.pair_next, 1u);
            if (!team_sync(T)) return;
            const int j = *(volatile int *)&P.team_slot[team_id];
            if (j >= P.npair) break;
            if (!batch_item(P, P.order[j], T, psm, info_sh, red_sh)) return;
        }
    }
    T.rank = 0;
    T.size = 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_sh = P.npair + (int)atomicAdd(P.next, 1u);
        __syncthreads();
        const int j = item_sh;
        if (j >= P.count) return;
        if (!batch_item(P, P.order[j], T, psm, info_sh, red_sh)) return;
    }
}

size_t batch_smem_bytes() {
    size_t b = leaf_smem_bytes(kPRcap);
    b = std::max(b, gram_smem_bytes());
    b = std::max(b, sizeof(float) * (size_t)gemm_smem_floats<32, 4, false>());
    b = std::max(b, sizeof(float) * (size_t)gemm_smem_floats<64, 8, false>());
    b = std::max(b, sizeof(float) * (size_t)gemm_smem_floats<64, 8, true>());
    return (b + 15) / 16 * 16;
}

// ------------------------------------------------------- pooled factors ----
// The factors of one persistent batch share one allocation; each factor set
// holds a reference, the last release frees it.
struct Pool {
    void *base = nullptr;
    int refs = 0;
};
std::mutex g_pool_mu;
std::unordered_map<const void *, Pool *> g_pool_of;   // keyed by each factor set's Q

std::atomic<int> g_phase_on{0};
std::mutex g_phase_mu;
unsigned long long g_phase_last[kPPhases] = {};

}  // namespace

bool release_pooled_factors(eod_factors *f) {
    if (!f || !f->Q) return false;
    Pool *pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto itp = g_pool_of.find(f->Q);
        if (itp == g_pool_of.end()) return false;
        pool = itp->second;
        g_pool_of.erase(itp);
        if (--pool->refs > 0) pool = nullptr;
    }
    if (pool) {
        cudaFree(pool->base);
        delete pool;
    }
    f->U = f->V = f->Q = f->C = nullptr;
    f->D = nullptr;
    return true;
}

eod_status factor_batched_persistent(const void *const *A, const int64_t *m, const int64_t *n, const int64_t *lda,
                                     int64_t count, double tol, uint64_t seed, const eod_opts &o, eod_factors **out,
                                     eod_status *per_item, std::vector<int64_t> &fallback) {
    fallback.clear();
    const int k = o.block_k > 0 ? o.block_k : 32;
    const bool form_ok = o.a_dtype == EOD_F32 && o.power_iters == 0 && k <= kPKmax && tol > 0.0 &&
                         std::isfinite(tol) && (o.tol_mode == EOD_TOL_ABS || o.tol_mode == EOD_TOL_REL_FRO) &&
                         (o.precision == EOD_PLAIN || o.precision == EOD_MIXED_BF16 ||
                          o.precision == EOD_MIXED_TF32) && count <= 0x7FFFFFFF;
    std::vector<int64_t> items;
    for (int64_t i = 0; i < count; ++i) {
        const bool ok = form_ok && A[i] && m[i] >= 1 && n[i] >= 1 && lda[i] >= m[i] && m[i] <= kPMaxDim &&
                        n[i] <= kPMaxDim;
        (ok ? items : fallback).push_back(i);
    }
    if (items.empty()) return EOD_OK;
    auto all_back = [&]() {
        fallback.clear();
        for (int64_t i = 0; i < count; ++i) fallback.push_back(i);
    };
    // largest m n first (an item's work here is about m n (r + k) with
    // r <= 128); items within a factor kPairFrac of the largest m n are taken
    // by pairs of CTAs (EOD_BATCH_PAIR sets the factor: 0 pairs every item,
    // above 1 none)
    std::stable_sort(items.begin(), items.end(),
                     [&](int64_t a, int64_t b) { return (double)m[a] * n[a] > (double)m[b] * n[b]; });
    const int64_t ne = (int64_t)items.size();
    double pair_frac = kPairFrac;
    if (const char *env = std::getenv("EOD_BATCH_PAIR")) pair_frac = std::atof(env);
    int npair = 0;
    {
        const double top = (double)m[items[0]] * n[items[0]];
        while (npair < ne && (double)m[items[npair]] * n[items[npair]] >= pair_frac * top) ++npair;
    }
    int64_t mmax = 1, nmax = 1;
    for (int64_t i : items) {
        mmax = std::max(mmax, m[i]);
        nmax = std::max(nmax, n[i]);
    }
    // the factors: one allocation, 256-byte aligned sections per item
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    std::vector<int64_t> off(ne);
    int64_t pool_bytes = 0;
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t i = items[e], c = std::min<int64_t>(std::min(m[i], n[i]), kPRcap);
        off[e] = pool_bytes;
        pool_bytes += 2 * up(4 * m[i] * c) + 2 * up(4 * n[i] * c) + up(8 * c * c);
    }
    cudaStream_t caller = (cudaStream_t)o.stream;
    void *pool = nullptr;   // stream-ordered, from the library's pool (eod_abe_free's cudaFree releases it)
    if (lib_malloc_async(&pool, (size_t)pool_bytes, caller) != cudaSuccess) {
        cudaGetLastError();
        all_back();
        return EOD_OK;
    }
    std::vector<PItem> hitems(ne);
    std::vector<int32_t> horder(ne);
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t i = items[e], c = std::min<int64_t>(std::min(m[i], n[i]), kPRcap);
        unsigned char *b = (unsigned char *)pool + off[e];
        PItem &it = hitems[e];
        it.A = (const float *)A[i];
        it.m = m[i];
        it.n = n[i];
        it.lda = lda[i];
        it.Q = (float *)b;
        it.U = (float *)(b + up(4 * m[i] * c));
        it.C = (float *)(b + 2 * up(4 * m[i] * c));
        it.V = (float *)(b + 2 * up(4 * m[i] * c) + up(4 * n[i] * c));
        it.D = (double *)(b + 2 * up(4 * m[i] * c) + 2 * up(4 * n[i] * c));
        it.cap = c;
        it.batch = (uint32_t)i;
        horder[e] = (int32_t)e;
    }

    int dev = 0, sms = kNumSMs;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(pool, caller);
        all_back();
        return EOD_OK;
    }
    const int grid = (int)std::min<int64_t>((ne + 1) / 2 * 2, sms / 2 * 2);   // clusters of two
    const int nteams = grid / 2;
    const PLayout L = playout(mmax, nmax);
    std::vector<PRes> hres(ne);
    for (PRes &rs : hres) rs.status = EOD_ETIMEOUT;   // what an item the launch did not finish reports
    std::vector<double> htd((size_t)ne * kPTdCap);
    cudaStream_t ps = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ready = nullptr;
    bool launched = false;
    {
        Arena ar(caller);
        PItem *ditems;
        int32_t *dorder;
        PRes *dres;
        double *dtd;
        unsigned char *scratch;
        unsigned *ctl;       // next, pair_next, err, team barriers, team slots
        float *xf;
        double *xd;
        unsigned long long *dphase = nullptr;
        const bool phases = g_phase_on.load() != 0;
        eod_status st = ar.get(&ditems, (size_t)ne);
        if (st == EOD_OK && phases) st = ar.get(&dphase, (size_t)kPPhases);
        if (st == EOD_OK) st = ar.get(&dorder, (size_t)ne);
        if (st == EOD_OK) st = ar.get(&dres, (size_t)ne);
        if (st == EOD_OK) st = ar.get(&dtd, (size_t)ne * kPTdCap);
        if (st == EOD_OK) st = ar.get(&scratch, (size_t)(L.bytes * grid));
        const size_t nctl = 4 + 2 * (size_t)nteams;
        if (st == EOD_OK) st = ar.get(&ctl, nctl);
        if (st == EOD_OK) st = ar.get(&xf, (size_t)nteams * 4 * kXF);
        if (st == EOD_OK) st = ar.get(&xd, (size_t)nteams * 4 * kXD);
        cudaError_t e = st == EOD_OK ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemcpyAsync(ditems, hitems.data(), sizeof(PItem) * ne, cudaMemcpyHostToDevice, caller);
        if (e == cudaSuccess && dphase) e = cudaMemsetAsync(dphase, 0, sizeof(unsigned long long) * kPPhases, caller);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dorder, horder.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, caller);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dres, hres.data(), sizeof(PRes) * ne, cudaMemcpyHostToDevice, caller);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, caller);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, ready, 0);
        const size_t smem = batch_smem_bytes();
        if (e == cudaSuccess) e = set_smem_once(batch_kernel, (int)smem);
        PParams P;
        P.items = ditems;
        P.order = dorder;
        P.res = dres;
        P.tdiag = dtd;
        P.scratch = scratch;
        P.stride = L.bytes;
        P.mmax = mmax;
        P.nmax = nmax;
        P.next = ctl;
        P.pair_next = ctl + 1;
        P.err = (int *)(ctl + 2);
        P.team_bar = ctl + 4;
        P.team_slot = (int *)(ctl + 4 + nteams);
        P.xf = xf;
        P.xd = xd;
        P.phase = dphase;
        P.count = (int)ne;
        P.npair = npair;
        P.k = k;
        P.tol_mode = o.tol_mode;
        P.compute_err = o.compute_err;
        P.tol = tol;
        P.seed = seed;
        // the queue reset and the persistent kernel, captured as one graph
        if (e == cudaSuccess) e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(ctl, 0, sizeof(unsigned) * nctl, ps);
            if (e1 == cudaSuccess) {
                batch_kernel<<<grid, PT, smem, ps>>>(P);
                e1 = cudaGetLastError();
            }
            e = cudaStreamEndCapture(ps, &graph);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) {
            double flops = 0.0, bytes = 0.0;
            for (int64_t i : items) {
                const double c = (double)std::min<int64_t>(std::min(m[i], n[i]), kPRcap);
                flops += 2.0 * m[i] * n[i] * (3.0 * c + k);
                bytes += 4.0 * m[i] * n[i] * 4.0;
            }
            count_launch(1);
            ProfScope prof(PROF_BATCH, flops, bytes, ps);
            e = cudaGraphLaunch(exec, ps);
            launched = e == cudaSuccess;
        }
        if (launched) e = cudaStreamSynchronize(ps);
        if (e == cudaSuccess) e = cudaMemcpy(hres.data(), dres, sizeof(PRes) * ne, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(htd.data(), dtd, sizeof(double) * ne * kPTdCap, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && dphase) {
            std::lock_guard<std::mutex> lk(g_phase_mu);
            e = cudaMemcpy(g_phase_last, dphase, sizeof(g_phase_last), cudaMemcpyDeviceToHost);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ready) cudaEventDestroy(ready);
        if (ps) {
            cudaStreamSynchronize(ps);
            cudaStreamDestroy(ps);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(pool, caller);
            cudaStreamSynchronize(caller);
            if (launched) return EOD_ECUDA;   // the launch itself failed: no item is retried
            all_back();
            return EOD_OK;
        }
    }

    // factor sets of the items that finished here
    Pool *pl = new Pool;
    pl->base = pool;
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t i = items[e];
        const PRes &rs = hres[e];
        if (rs.status == kPFallback) {
            fallback.push_back(i);
            continue;
        }
        if (rs.status != EOD_OK) {
            per_item[i] = (eod_status)rs.status;
            continue;
        }
        eod_factors *F = (eod_factors *)std::calloc(1, sizeof(eod_factors));
        const int nt = std::max(1, rs.ntdiag);
        double *td = F ? (double *)std::malloc(sizeof(double) * nt) : nullptr;
        if (!F || !td) {
            std::free(F);
            std::free(td);
            per_item[i] = EOD_ENOMEM;
            continue;
        }
        F->m = m[i];
        F->n = n[i];
        F->rank = rs.rank;
        F->f_dtype = EOD_F32;
        F->precision = EOD_PLAIN;
        F->norm_a = rs.norm_a;
        F->eps = rs.eps;
        F->rel_err = rs.rel_err;
        F->blocks = rs.blocks;
        F->restarts = rs.restarts;
        F->block_k = k;
        F->ntdiag = rs.ntdiag;
        std::memcpy(td, htd.data() + (size_t)e * kPTdCap, sizeof(double) * std::max(0, rs.ntdiag));
        F->tdiag = td;
        double margin = INFINITY;
        for (int j = 0; j < rs.ntdiag; ++j)
            if (td[j] > 0.0 && rs.eps > 0.0) margin = std::min(margin, std::fabs(std::log10(td[j] / rs.eps)));
        F->t_margin = margin;
        if (rs.rank > 0) {
            const PItem &it = hitems[e];
            F->Q = it.Q;
            F->U = it.U;
            F->C = it.C;
            F->V = it.V;
            F->D = it.D;
            std::lock_guard<std::mutex> lk(g_pool_mu);
            g_pool_of[it.Q] = pl;
            ++pl->refs;
        }
        out[i] = F;
        per_item[i] = EOD_OK;
    }
    if (pl->refs == 0) {
        cudaFreeAsync(pool, caller);
        delete pl;
    }
    std::sort(fallback.begin(), fallback.end());
    return EOD_OK;
}

}  // namespace eod

// Measurement hook of the persistent batched launch: with enable != 0 every
// later launch sums, per phase of an item, the SM clock ticks its CTAs spent
// there (kPPhases counters: unused (the norm is summed in the first
// sketch), Omega, sketch, projection against Q, Gram
// and rank-test leaf, the panel's CholQR2 products, explicit residuals,
// projection C = A^T Q, reconstruction error, core QRs, U = Q Qh); out
// receives the last launch's counters (n >= kPPhases).  Timing only.
extern "C" eod_status eod_abe_debug_batch_phases(int32_t enable, double *out, int64_t n) {
    using namespace eod;
    g_phase_on.store(enable ? 1 : 0);
    if (!out) return EOD_OK;
    if (n < kPPhases) return EOD_EINVAL;
    std::lock_guard<std::mutex> lk(g_phase_mu);
    for (int i = 0; i < kPPhases; ++i) out[i] = (double)g_phase_last[i];
    return EOD_OK;
}

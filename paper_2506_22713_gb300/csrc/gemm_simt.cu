// SIMT GEMM of the plain (FP64 / FP32) path: the dense contractions of
// Alg. 1 and Alg. 2 that do not go to the tensor cores.  With FP32 data that
// is all of them but the core's large Gram matrices (widened to FP64 and
// emulated in oz_gemm.cu): the sketch A*Omega of Alg. 1 step 4, the two block
// Gram-Schmidt projections Q^T Y and Y - Q S of step 4, the CholQR Grams of
// step 5, the projection C^T = A^T Q of Alg. 2 step 8, the triangular solves
// and products of steps 9-11 and the reconstruction Q C with its fused
// Frobenius error of Sec. 4.1.  With FP64 data only the products below 2^25
// multiply-adds (and the CGS2 residual's matrix-vector products) run here:
// the larger ones are the FP64 emulation on tcgen05 in oz_gemm.cu.
//
// Tile TS x TS x 16 (TS = 64, 32 or 16: the smaller tiles spread products too
// small to fill the 152 SMs with 64-tiles), 256 threads, (TS/16)^2 outputs
// per thread with the row index fastest across lanes so that column-major
// stores coalesce.  The K range may be split as well, the partial tiles then
// summed by a second kernel in a fixed order.  FP64 runs at
// a few DFMA per clock per SM here, so small FP64 products are only fast when
// they are spread over every SM.
#include "common.cuh"
#include "instrument.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>

namespace eod {
namespace {

constexpr int BK = 16, NT = 256;
constexpr int BM = 64, BN = 64;   // the large tile (gemm_err_ctas)
constexpr int F_UPPER_ONLY = 1, F_A_UPPER = 2, F_B_UPPER = 4;

template <typename TA, typename TB, typename TC, typename Acc, bool TRA, bool TRB, int EPI, bool SPLIT, int TS>
__global__ void __launch_bounds__(NT)
gemm_simt_kernel(int64_t M, int64_t N, int64_t K, Acc alpha, const TA *__restrict__ A, int64_t lda,
                 const TB *__restrict__ B, int64_t ldb, Acc beta, TC *C, int64_t ldc, int64_t kchunk,
                 Acc *__restrict__ part, int flags, const TC *__restrict__ ref, int64_t ldref,
                 double *__restrict__ errp, unsigned *__restrict__ tile_count)
{
    constexpr int BM = TS, BN = TS, TPT = TS / 16;   // outputs per thread along each axis
    // FP32 tiles of 64 and 128: each thread owns runs of four consecutive
    // rows (and columns), read from shared memory as float4 (one 128-bit
    // load per four FMAs-rows instead of four 32-bit ones); the rows are
    // padded by 4 to keep those loads 16-byte aligned.  Otherwise a thread's
    // outputs are 16 apart.
    constexpr bool VEC = std::is_same<Acc, float>::value && TS >= 64;
    constexpr int PAD = VEC ? 4 : 1;
    __shared__ __align__(16) Acc As[BK][BM + PAD];
    __shared__ __align__(16) Acc Bs[BK][BN + PAD];
    __shared__ double red[32];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    // tile-local row of the thread's i-th output (column: same with ty)
    auto lo = [&](int t, int i) -> int { return VEC ? ((i >> 2) * 64 + t * 4 + (i & 3)) : (t + 16 * i); };

    if ((flags & F_UPPER_ONLY) && m0 > n0 + BN - 1) {
        if (EPI == EPI_ERR && tid == 0) errp[blockIdx.x + (int64_t)blockIdx.y * gridDim.x] = 0.0;
        return;
    }
    int64_t kb = (int64_t)blockIdx.z * kchunk;
    int64_t ke = kb + kchunk < K ? kb + kchunk : K;
    if (flags & F_A_UPPER) kb = kb > m0 ? kb : m0;                // op(A)(i,l) = 0 for l < i
    if (flags & F_B_UPPER) ke = ke < n0 + BN ? ke : n0 + BN;      // op(B)(l,j) = 0 for l > j

    Acc acc[TPT][TPT];
#pragma unroll
    for (int i = 0; i < TPT; ++i)
#pragma unroll
        for (int j = 0; j < TPT; ++j) acc[i][j] = Acc(0);

    // The next K tile's operands are loaded into registers while the
    // current one is multiplied out of shared memory, so the global loads'
    // latency overlaps the FMAs.
    constexpr int QA = (BM * BK) / NT, QB = (BN * BK) / NT;
    Acc ra[QA], rb[QB];
    auto load_tile = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < QA; ++q) {
            const int e = tid + q * NT;
            int i, kk;
            if (!TRA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
            const int64_t gi = m0 + i, gk = k0 + kk;
            ra[q] = (gi < M && gk < ke) ? (Acc)(TRA ? A[gk + gi * lda] : A[gi + gk * lda]) : Acc(0);
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const int e = tid + q * NT;
            int j, kk;
            if (!TRB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
            const int64_t gj = n0 + j, gk = k0 + kk;
            rb[q] = (gj < N && gk < ke) ? (Acc)(TRB ? B[gj + gk * ldb] : B[gk + gj * ldb]) : Acc(0);
        }
    };
    if (kb < ke) load_tile(kb);
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int q = 0; q < QA; ++q) {
            const int e = tid + q * NT;
            int i, kk;
            if (!TRA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
            As[kk][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            const int e = tid + q * NT;
            int j, kk;
            if (!TRB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
            Bs[kk][j] = rb[q];
        }
        __syncthreads();
        if (k0 + BK < ke) load_tile(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Acc a[TPT], b[TPT];
#pragma unroll
            if constexpr (VEC) {
#pragma unroll
                for (int h = 0; h < TPT / 4; ++h) {
                    const float4 av = *reinterpret_cast<const float4 *>(&As[kk][h * 64 + tx * 4]);
                    const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][h * 64 + ty * 4]);
                    a[4 * h] = av.x; a[4 * h + 1] = av.y; a[4 * h + 2] = av.z; a[4 * h + 3] = av.w;
                    b[4 * h] = bv.x; b[4 * h + 1] = bv.y; b[4 * h + 2] = bv.z; b[4 * h + 3] = bv.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < TPT; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < TPT; ++j) b[j] = Bs[kk][ty + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < TPT; ++i)
#pragma unroll
                for (int j = 0; j < TPT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (SPLIT) {
        Acc *dst = part + (int64_t)blockIdx.z * M * N;
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int64_t col = n0 + lo(ty, j);
            if (col >= N) continue;
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                const int64_t row = m0 + lo(tx, i);
                if (row < M) dst[row + col * M] = acc[i][j];
            }
        }
        if (!tile_count) return;
        // The last of the tile's S CTAs to finish sums the partials in split
        // order (the same order as the separate reduction) and stores C; it
        // also resets the tile's counter for the next product on the stream.
        __shared__ int last_sh;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const int64_t t = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
            const unsigned prev = atomicAdd(&tile_count[t], 1u);
            last_sh = (prev + 1 == gridDim.z);
            if (last_sh) tile_count[t] = 0u;
        }
        __syncthreads();
        if (!last_sh) return;
        __threadfence();
        // splits outer, the thread's outputs inner (their loads in flight
        // together); each sum still runs in split order
        Acc sum[TPT][TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j)
#pragma unroll
            for (int i = 0; i < TPT; ++i) sum[i][j] = Acc(0);
        for (unsigned z = 0; z < gridDim.z; ++z) {
            const Acc *src = part + (int64_t)z * M * N;
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const int64_t col = n0 + lo(ty, j);
#pragma unroll
                for (int i = 0; i < TPT; ++i) {
                    const int64_t row = m0 + lo(tx, i);
                    if (row < M && col < N) sum[i][j] += __ldcg(src + row + col * M);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int64_t col = n0 + lo(ty, j);
            if (col >= N) continue;
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                const int64_t row = m0 + lo(tx, i);
                if (row >= M) continue;
                Acc v = alpha * sum[i][j];
                if (beta != Acc(0)) v = fma(beta, (Acc)C[row + col * ldc], v);
                C[row + col * ldc] = (TC)v;
            }
        }
        return;
    }
    double local = 0.0;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        const int64_t col = n0 + lo(ty, j);
        if (col >= N) continue;
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
            const int64_t row = m0 + lo(tx, i);
            if (row >= M) continue;
            Acc v = alpha * acc[i][j];
            if (EPI == EPI_STORE) {
                if (beta != Acc(0)) v = fma(beta, (Acc)C[row + col * ldc], v);
                C[row + col * ldc] = (TC)v;
            } else {
                const TC vh = (TC)v;
                if (C != nullptr) C[row + col * ldc] = vh;
                const double d = (double)ref[row + col * ldref] - (double)vh;
                local = fma(d, d, local);
            }
        }
    }
    if (EPI == EPI_ERR) {
        const double tot = block_sum(local, red);
        if (tid == 0) errp[blockIdx.x + (int64_t)blockIdx.y * gridDim.x] = tot;
    }
}

template <typename TC, typename Acc>
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int S, const Acc *__restrict__ part,
                                     Acc alpha, Acc beta, TC *C, int64_t ldc, int upper_only, int ts)
{
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e % M, col = e / M;
        if (upper_only && (row / ts) * ts > (col / ts) * ts + ts - 1) continue;
        Acc s = Acc(0);
        for (int z = 0; z < S; ++z) s += part[(int64_t)z * total + e];
        Acc v = alpha * s;
        if (beta != Acc(0)) v = fma(beta, (Acc)C[row + col * ldc], v);
        C[row + col * ldc] = (TC)v;
    }
}

// Matrix-vector products (N = 1: the explicit CGS2 residual of an undecided
// pivot, Alg. 1 steps 6-11): HBM-bound, so one pass over A with full lanes
// instead of a GEMM tile that is 1/32 used.
//   y = alpha A x + beta y   (A M x K): a thread per row, K loop, coalesced;
//   y = alpha A^T x + beta y (A K x M): a CTA per (column, K range), a fixed
//   order block reduction, partial sums reduced in order by a second kernel.
template <typename TA, typename TB, typename TC, typename Acc>
__global__ void gemv_n_kernel(int64_t M, int64_t K, Acc alpha, const TA *__restrict__ A, int64_t lda,
                              const TB *__restrict__ x, Acc beta, TC *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        Acc acc = Acc(0);
        for (int64_t k = 0; k < K; ++k) acc = fma((Acc)A[i + k * lda], (Acc)x[k], acc);
        Acc v = alpha * acc;
        if (beta != Acc(0)) v = fma(beta, (Acc)y[i], v);
        y[i] = (TC)v;
    }
}

// y partials over K ranges (A M x K): a thread per row and range,
// coalesced along the rows; gemv_t_reduce_kernel sums the ranges in order.
template <typename TA, typename TB, typename Acc>
__global__ void __launch_bounds__(256) gemv_n_partial_kernel(int64_t M, int64_t K, int64_t chunk,
                                                             const TA *__restrict__ A, int64_t lda,
                                                             const TB *__restrict__ x, Acc *__restrict__ part) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t k0 = (int64_t)blockIdx.y * chunk;
    const int64_t k1 = k0 + chunk < K ? k0 + chunk : K;
    Acc acc = Acc(0);
    for (int64_t k = k0; k < k1; ++k) acc = fma((Acc)A[i + k * lda], (Acc)x[k], acc);
    part[(int64_t)blockIdx.y * M + i] = acc;
}

template <typename TA, typename TB, typename Acc>
__global__ void __launch_bounds__(256) gemv_t_partial_kernel(int64_t M, int64_t K, int64_t chunk,
                                                             const TA *__restrict__ A, int64_t lda,
                                                             const TB *__restrict__ x, Acc *__restrict__ part) {
    __shared__ Acc red[256];
    const int64_t i = blockIdx.x, k0 = (int64_t)blockIdx.y * chunk;
    int64_t k1 = k0 + chunk;
    if (k1 > K) k1 = K;
    Acc acc = Acc(0);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc = fma((Acc)A[k + i * lda], (Acc)x[k], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * M + i] = red[0];
}

template <typename TC, typename Acc>
__global__ void gemv_t_reduce_kernel(int64_t M, int S, const Acc *__restrict__ part, Acc alpha, Acc beta, TC *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        Acc s = Acc(0);
        for (int z = 0; z < S; ++z) s += part[(int64_t)z * M + i];
        Acc v = alpha * s;
        if (beta != Acc(0)) v = fma(beta, (Acc)y[i], v);
        y[i] = (TC)v;
    }
}

template <typename TA, typename TB, typename TC, typename Acc>
cudaError_t launch_gemv(bool ta, int64_t M, int64_t K, double alpha, const TA *A, int64_t lda, const TB *x,
                        double beta, TC *y, Scratch *ws, cudaStream_t s) {
    ProfScope prof(std::is_same<Acc, float>::value ? PROF_GEMM_SIMT32 : PROF_GEMM_SIMT, 2.0 * (double)M * K,
                   (double)sizeof(TA) * M * K, s);
    if (!ta) {
        // K split so that about four CTAs per SM work (a row's FMAs form one
        // dependent chain per range), ranges of at least 16
        const int64_t rblocks = (M + 255) / 256;
        int64_t S = (4 * kNumSMs + rblocks - 1) / rblocks;
        const int64_t smax = (K + 15) / 16;
        if (S > smax) S = smax;
        if (S > 65535) S = 65535;
        Acc *part = nullptr;
        size_t mark = ws ? ws->mark() : 0;
        if (S > 1) part = ws ? (Acc *)ws->take(sizeof(Acc) * (size_t)S * (size_t)M) : nullptr;
        if (S <= 1 || !part || rblocks > 2147483647LL) {
            count_launch();
            const int64_t blocks = std::min<int64_t>(rblocks, 8LL * kNumSMs);
            gemv_n_kernel<TA, TB, TC, Acc><<<(unsigned)blocks, 256, 0, s>>>(M, K, (Acc)alpha, A, lda, x, (Acc)beta,
                                                                             y);
            return cudaGetLastError();
        }
        const int64_t chunk = (K + S - 1) / S;
        S = (K + chunk - 1) / chunk;
        count_launch(2);
        gemv_n_partial_kernel<TA, TB, Acc><<<dim3((unsigned)rblocks, (unsigned)S), 256, 0, s>>>(M, K, chunk, A, lda,
                                                                                                  x, part);
        EOD_CUDA_TRY(cudaGetLastError());
        const int64_t blocks = std::min<int64_t>(rblocks, 8LL * kNumSMs);
        gemv_t_reduce_kernel<TC, Acc><<<(unsigned)blocks, 256, 0, s>>>(M, (int)S, part, (Acc)alpha, (Acc)beta, y);
        EOD_CUDA_TRY(cudaGetLastError());
        ws->release(mark);
        return cudaSuccess;
    }
    // K split so that about four CTAs per SM work, chunks of at least 2048
    int64_t S = (4 * kNumSMs + M - 1) / M;
    const int64_t smax = (K + 2047) / 2048;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    const int64_t chunk = (K + S - 1) / S;
    S = (K + chunk - 1) / chunk;
    if (S < 1) S = 1;
    size_t mark = ws ? ws->mark() : 0;
    Acc *part = ws ? (Acc *)ws->take(sizeof(Acc) * (size_t)S * (size_t)M) : nullptr;
    if (!part) return cudaErrorMemoryAllocation;
    count_launch(2);
    gemv_t_partial_kernel<TA, TB, Acc><<<dim3((unsigned)M, (unsigned)S), 256, 0, s>>>(M, K, chunk, A, lda, x, part);
    EOD_CUDA_TRY(cudaGetLastError());
    const int64_t blocks = std::min<int64_t>((M + 255) / 256, 8LL * kNumSMs);
    gemv_t_reduce_kernel<TC, Acc><<<(unsigned)blocks, 256, 0, s>>>(M, (int)S, part, (Acc)alpha, (Acc)beta, y);
    EOD_CUDA_TRY(cudaGetLastError());
    ws->release(mark);
    return cudaSuccess;
}

// Tile size and K split: FP64 issue (a few DFMA per clock per SM) bounds
// every tile, so the plan minimises the DFMA count of the busiest SM,
// ceil(CTAs / SMs) * TS^2 * kchunk, plus the second launch and the partial
// traffic a split costs; smaller tiles carry a small penalty for their lower
// reuse of shared operands, so that large products keep the 64-tiles.
struct SimtPlan {
    int ts;
    int64_t gm, gn, S;
};

inline SimtPlan simt_plan(int64_t M, int64_t N, int64_t K, const GemmExtra &x);

// FP32 arithmetic has 64 times the issue rate, and there shared memory
// bounds the tile instead: per step of K a warp issues TPT^2 FFMA (4 per
// clock per SM) against about 2 TPT shared-memory wavefronts (1 per clock),
// so the per-CTA cost is kch * max(TPT^2 / 4, 2 TPT) and the 128-tiles
// (TPT = 8) are the only ones that keep the FFMA pipes busy -- once there
// are enough of them: with fewer than 128 such tiles (or K < 128) the
// latency of each CTA's K loop dominates and the FP64 plan's smaller tiles
// measured faster (8192 x 64 x 64: 11 us on 32-tiles, 16 us on 128-tiles;
// 8192 x 455 x 455: 126 us on 128-tiles, 259 us on 32-tiles), and with
// fewer than 4096 rows (the 2048^2 image workload's core products ran 2.6x
// slower as a whole on 128-tiles).
inline SimtPlan simt_plan_f32(int64_t M, int64_t N, int64_t K, const GemmExtra &x) {
    // the tile: forced (timing hook), else the autotuner's table, else the rule
    int only = x.force_ts;
    int64_t tv = 0;
    if (!only && tuned_value("f32_tile", M, N, K, &tv) && (tv == 16 || tv == 32 || tv == 64 || tv == 128))
        only = (int)tv;
    if (!only && (((M + 127) / 128) * ((N + 127) / 128) < 128 || K < 128 || M < 4096)) return simt_plan(M, N, K, x);
    SimtPlan best{64, 0, 0, 1};
    double best_cost = -1.0;
    for (int ts = 128; ts >= 16; ts /= 2) {
        if (only && ts != only) continue;
        const int64_t gm = (M + ts - 1) / ts, gn = (N + ts - 1) / ts;
        if (gn > 65535) continue;
        int64_t tiles = gm * gn;
        if (x.upper_only) tiles = (tiles + gm) / 2 + 1;
        const double tpt = ts / 16.0;
        const double per_k = std::max(tpt * tpt / 4.0, 2.0 * tpt);
        for (int64_t kc = BK;; kc *= 2) {
            const int64_t kch = K > 0 ? std::min<int64_t>(kc, K) : 1;
            const int64_t S = K > 0 ? (K + kch - 1) / kch : 1;
            if (S <= x.max_split && S <= 65535) {
                // a 128-tile CTA holds 64 accumulators per thread: one CTA per
                // SM sub-partition set; smaller tiles overlap two
                const int64_t per_sm = ts == 128 ? 1 : 2;
                const int64_t waves = (tiles * S + per_sm * kNumSMs - 1) / (per_sm * kNumSMs);
                double cost = (double)waves * per_sm * (double)kch * per_k * 8.0;
                if (S > 1) cost += 3000.0 + 2.0 * (double)M * (double)N * (double)S * 4.0 / 2400.0;
                if (best_cost < 0.0 || cost < best_cost) {
                    best_cost = cost;
                    best = {ts, gm, gn, S};
                }
            }
            if (kc >= K) break;
        }
    }
    return best;
}

inline SimtPlan simt_plan(int64_t M, int64_t N, int64_t K, const GemmExtra &x) {
    SimtPlan best{64, 0, 0, 1};
    double best_cost = -1.0;
    for (int ts = 64; ts >= 16; ts /= 2) {
        const int64_t gm = (M + ts - 1) / ts, gn = (N + ts - 1) / ts;
        if (gn > 65535) continue;
        int64_t tiles = gm * gn;
        if (x.upper_only) tiles = (tiles + gm) / 2 + 1;
        for (int64_t kc = BK;; kc *= 2) {
            const int64_t kch = K > 0 ? std::min<int64_t>(kc, K) : 1;
            const int64_t S = K > 0 ? (K + kch - 1) / kch : 1;
            if (S <= x.max_split && S <= 65535) {
                const int64_t waves = (tiles * S + kNumSMs - 1) / kNumSMs;
                double cost = (double)waves * ts * ts * (double)kch * 0.5 * (1.0 + 0.05 * (64 / ts - 1));
                if (S > 1) cost += 3000.0 + 2.0 * (double)M * (double)N * (double)S * 8.0 / 2400.0;
                if (best_cost < 0.0 || cost < best_cost) {
                    best_cost = cost;
                    best = {ts, gm, gn, S};
                }
            }
            if (kc >= K) break;
        }
    }
    return best;
}

template <typename TA, typename TB, typename TC, typename Acc, bool TRA, bool TRB, int TS>
cudaError_t launch_store(const SimtPlan &pl, int64_t M, int64_t N, int64_t K, double alpha, const TA *A,
                         int64_t lda, const TB *B, int64_t ldb, double beta, TC *C, int64_t ldc, int flags,
                         const GemmExtra &x, Scratch *ws, cudaStream_t s)
{
    int64_t S = pl.S;
    Acc *part = nullptr;
    size_t mark = ws ? ws->mark() : 0;
    while (S > 1) {
        part = ws ? (Acc *)ws->take(sizeof(Acc) * (size_t)S * (size_t)M * (size_t)N) : nullptr;
        if (part) break;
        S /= 2;
    }
    int64_t kchunk = K > 0 ? K : 1;
    if (S > 1) {
        kchunk = ((K + S - 1) / S + BK - 1) / BK * BK;
        S = (K + kchunk - 1) / kchunk;
    }
    dim3 grid((unsigned)pl.gm, (unsigned)pl.gn, (unsigned)S);
    if (S > 1) {
        // the split's partial sums are folded by the tile's last CTA when the
        // workspace has a counter per tile and that CTA's share is small
        // (at most 64 K partial values), else by a second kernel
        unsigned *cnt = (ws && ws->tile_count && pl.gm * pl.gn <= ws->tile_count_n && (int64_t)TS * TS * S <= 65536)
                            ? ws->tile_count
                            : nullptr;
        count_launch(cnt ? 1 : 2);
        gemm_simt_kernel<TA, TB, TC, Acc, TRA, TRB, EPI_STORE, true, TS><<<grid, NT, 0, s>>>(
            M, N, K, (Acc)alpha, A, lda, B, ldb, (Acc)beta, C, ldc, kchunk, part, flags, nullptr, 0,
            nullptr, cnt);
        EOD_CUDA_TRY(cudaGetLastError());
        if (!cnt) {
            int64_t total = M * N;
            int blocks = (int)((total + 255) / 256);
            if (blocks > 4 * kNumSMs * 8) blocks = 4 * kNumSMs * 8;
            splitk_reduce_kernel<TC, Acc><<<blocks, 256, 0, s>>>(M, N, (int)S, part, (Acc)alpha, (Acc)beta,
                                                                 C, ldc, x.upper_only ? 1 : 0, TS);
            EOD_CUDA_TRY(cudaGetLastError());
        }
        ws->release(mark);
        return cudaSuccess;
    }
    count_launch();
    gemm_simt_kernel<TA, TB, TC, Acc, TRA, TRB, EPI_STORE, false, TS><<<grid, NT, 0, s>>>(
        M, N, K, (Acc)alpha, A, lda, B, ldb, (Acc)beta, C, ldc, kchunk, nullptr, flags, nullptr, 0,
        nullptr, nullptr);
    return cudaGetLastError();
}

template <typename TA, typename TB, typename TC, typename Acc, bool TRA, bool TRB>
cudaError_t launch(int64_t M, int64_t N, int64_t K, double alpha, const TA *A, int64_t lda,
                   const TB *B, int64_t ldb, double beta, TC *C, int64_t ldc, const GemmExtra &x,
                   Scratch *ws, cudaStream_t s)
{
    const int flags = (x.upper_only ? F_UPPER_ONLY : 0) | (x.a_upper ? F_A_UPPER : 0) |
                      (x.b_upper ? F_B_UPPER : 0);
    double frac = 1.0;
    if (x.upper_only) frac *= 0.5;
    if (x.a_upper && x.b_upper) frac /= 6.0;
    else if (x.a_upper || x.b_upper) frac *= 0.5;
    const double flops = 2.0 * (double)M * (double)N * (double)K * frac;
    double bytes = (double)sizeof(TA) * M * K + (double)sizeof(TB) * K * N + (double)sizeof(TC) * M * N;
    if (beta != 0.0 || x.epilogue == EPI_ERR) bytes += (double)sizeof(TC) * M * N;
    ProfScope prof(std::is_same<Acc, float>::value ? PROF_GEMM_SIMT32 : PROF_GEMM_SIMT, flops, bytes, s);
    if (x.epilogue == EPI_ERR) {
        if ((N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
        count_launch();
        dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), 1);
        gemm_simt_kernel<TA, TB, TC, Acc, TRA, TRB, EPI_ERR, false, 64><<<grid, NT, 0, s>>>(
            M, N, K, (Acc)alpha, A, lda, B, ldb, (Acc)beta, C, ldc, K > 0 ? K : 1, nullptr, flags,
            (const TC *)x.ref, x.ldref, x.err_partials, nullptr);
        return cudaGetLastError();
    }
    const bool f32 = std::is_same<Acc, float>::value;
    const SimtPlan pl = f32 ? simt_plan_f32(M, N, K, x) : simt_plan(M, N, K, x);
    if (pl.gm == 0) return cudaErrorInvalidValue;
    if (f32 && pl.ts == 128)
        return launch_store<TA, TB, TC, Acc, TRA, TRB, 128>(pl, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags,
                                                             x, ws, s);
    if (pl.ts == 64)
        return launch_store<TA, TB, TC, Acc, TRA, TRB, 64>(pl, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags,
                                                            x, ws, s);
    if (pl.ts == 32)
        return launch_store<TA, TB, TC, Acc, TRA, TRB, 32>(pl, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags,
                                                            x, ws, s);
    return launch_store<TA, TB, TC, Acc, TRA, TRB, 16>(pl, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, x,
                                                        ws, s);
}

}  // namespace

int64_t gemm_err_ctas(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + BN - 1) / BN); }

// Large FP64 products go to the tensor-core emulation (oz_gemm.cu) unless
// EOD_FP64_GEMM=simt; products below 2^25 multiply-adds stay on the SIMT
// kernel, whose launch and slicing overheads are smaller there.  A skinny
// side (a few columns) does not exclude the emulation: the SIMT tiles waste
// as much, and FP64 issue is what they are short of.
bool fp64_use_emulated(int64_t M, int64_t N, int64_t K) {
    static const int mode = [] {
        const char *v = std::getenv("EOD_FP64_GEMM");
        if (v && std::strcmp(v, "simt") == 0) return 0;
        if (v && std::strcmp(v, "emulated") == 0) return 2;
        return 1;
    }();
    if (mode == 0) return false;
    if (mode == 2) return M >= 1 && N >= 1 && K >= 1;
    return (double)M * (double)N * (double)K >= 33554432.0 && K >= 8 && (M >= 128 || N >= 128);
}

// FP32 products through the emulation only with EOD_FP32_GEMM=emulated: the
// FFMA rate is 64 times the DFMA rate, and at the shapes of the method (one
// side at most a few hundred, FP32 operands sliced on every call) the FFMA
// kernel measured as fast or faster (8192 x 455 x 455: 259 us FFMA against
// 255 us emulated plus 64 us of slicing; 8192 x 256 x 256: 75 against
// 85 + 36 us), so it stays the default.
bool fp32_use_emulated(int64_t M, int64_t N, int64_t K) {
    static const bool on = [] {
        const char *v = std::getenv("EOD_FP32_GEMM");
        return v && std::strcmp(v, "emulated") == 0;
    }();
    return on && M >= 1 && N >= 1 && K >= 1;
}

template <typename TA, typename TB, typename TC, typename Acc>
cudaError_t gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const TA *A,
                 int64_t lda, const TB *B, int64_t ldb, double beta, TC *C, int64_t ldc,
                 const GemmExtra &x, Scratch *ws, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (std::is_same<TA, double>::value && std::is_same<TB, double>::value && std::is_same<TC, double>::value &&
        ws && ws->err_flag && K > 0 && fp64_use_emulated(M, N, K) && (x.epilogue != EPI_ERR || K <= kOzErrMaxK))
        return oz_gemm(ta, tb, M, N, K, alpha, (const double *)A, lda, (const double *)B, ldb, beta, (double *)C,
                       ldc, x, ws->err_flag, s);
    // large FP32 products: the same emulation (more accurate than FP32 FFMA
    // and far faster on this GPU), rounded once to FP32
    if (std::is_same<TA, float>::value && std::is_same<TB, float>::value && std::is_same<TC, float>::value &&
        ws && ws->err_flag && K > 0 && x.epilogue == EPI_STORE && fp32_use_emulated(M, N, K))
        return oz_gemm_f32(ta, tb, M, N, K, alpha, (const float *)A, lda, (const float *)B, ldb, beta, (float *)C,
                           ldc, x, ws->err_flag, s);
    // matrix-vector products: op(B) is one column of K contiguous values
    if (N == 1 && !tb && K > 0 && x.epilogue == EPI_STORE && !x.upper_only && !x.a_upper && !x.b_upper && ws)
        return launch_gemv<TA, TB, TC, Acc>(ta, M, K, alpha, A, lda, B, beta, C, ws, s);
    if (!ta && !tb) return launch<TA, TB, TC, Acc, false, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, ws, s);
    if (ta && !tb) return launch<TA, TB, TC, Acc, true, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, ws, s);
    if (!ta && tb) return launch<TA, TB, TC, Acc, false, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, ws, s);
    return launch<TA, TB, TC, Acc, true, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, ws, s);
}

template cudaError_t gemm<double, double, double, double>(bool, bool, int64_t, int64_t, int64_t, double,
    const double *, int64_t, const double *, int64_t, double, double *, int64_t, const GemmExtra &,
    Scratch *, cudaStream_t);
template cudaError_t gemm<float, float, float, float>(bool, bool, int64_t, int64_t, int64_t, double,
    const float *, int64_t, const float *, int64_t, double, float *, int64_t, const GemmExtra &,
    Scratch *, cudaStream_t);
template cudaError_t gemm<float, float, double, double>(bool, bool, int64_t, int64_t, int64_t, double,
    const float *, int64_t, const float *, int64_t, double, double *, int64_t, const GemmExtra &,
    Scratch *, cudaStream_t);

}  // namespace eod

// ---------------------------------------------------------------------------
// Timing hook of the autotuner: one FP32 product on the SIMT kernel with a
// forced tile (ts = 16, 32, 64, 128) or the library's choice (ts = 0).
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_f32_gemm(int32_t ts, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K,
                                             double alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                                             double beta, float *C, int64_t ldc, void *stream) {
    using namespace eod;
    if (!(ts == 0 || ts == 16 || ts == 32 || ts == 64 || ts == 128)) return EOD_EINVAL;
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || ldc < M) return EOD_EINVAL;
    if (lda < (ta ? K : M) || ldb < (tb ? N : K)) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Arena ar(s);
    Scratch ws;
    eod_status st = ar.get((char **)&ws.base, (size_t)64 << 20);
    if (st != EOD_OK) return st;
    ws.size = (size_t)64 << 20;
    st = ar.get(&ws.tile_count, (size_t)kTileCounters);
    if (st != EOD_OK) return st;
    ws.tile_count_n = kTileCounters;
    if (cudaMemsetAsync(ws.tile_count, 0, sizeof(unsigned) * kTileCounters, s) != cudaSuccess) {
        cudaGetLastError();
        return EOD_ECUDA;
    }
    GemmExtra x;
    x.force_ts = ts;
    cudaError_t e = gemm<float, float, float, float>(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                     x, &ws, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EOD_ECUDA;
    }
    return EOD_OK;
}

// ---------------------------------------------------------------------------
// Test hook: one FP64 GEMM through the SIMT kernel (mode 0) or the tensor-core
// emulation (mode 1), C = alpha op(A) op(B) + beta C, device pointers.
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_f64_gemm(int32_t mode, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K,
                                             double alpha, const double *A, int64_t lda, const double *B,
                                             int64_t ldb, double beta, double *C, int64_t ldc, void *stream) {
    using namespace eod;
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || ldc < M) return EOD_EINVAL;
    if (lda < (ta ? K : M) || ldb < (tb ? N : K)) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    GemmExtra x;
    x.upper_only = (mode & 16) != 0;
    x.a_upper = (mode & 32) != 0;
    x.b_upper = (mode & 64) != 0;
    if ((mode & 3) > 1 || (mode & ~(3 | 16 | 32 | 64 | 128)) != 0) return EOD_EINVAL;
    cudaError_t e;
    if ((mode & 3) == 1) {
        int *flag = nullptr;
        if (cudaMallocAsync((void **)&flag, sizeof(int), s) != cudaSuccess) { cudaGetLastError(); return EOD_ENOMEM; }
        cudaMemsetAsync(flag, 0, sizeof(int), s);
        e = oz_gemm(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, flag, s);
        int h = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(flag, s);
        if (e != cudaSuccess) {
            std::fprintf(stderr, "eod_abe_debug_f64_gemm: %s\n", cudaGetErrorString(e));
            cudaGetLastError();
            return EOD_ECUDA;
        }
        return h ? EOD_ETIMEOUT : EOD_OK;
    }
    Scratch ws;
    if (cudaMallocAsync((void **)&ws.base, (size_t)48 << 20, s) != cudaSuccess) { cudaGetLastError(); return EOD_ENOMEM; }
    ws.size = (size_t)48 << 20;
    if (!(mode & 128)) {   // K splits folded in-kernel (else by the separate reduction)
        if (cudaMallocAsync((void **)&ws.tile_count, sizeof(unsigned) * kTileCounters, s) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(ws.base, s);
            return EOD_ENOMEM;
        }
        cudaMemsetAsync(ws.tile_count, 0, sizeof(unsigned) * kTileCounters, s);
        ws.tile_count_n = kTileCounters;
    }
    e = gemm<double, double, double, double>(ta != 0, tb != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, x, &ws, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(ws.base, s);
    if (ws.tile_count) cudaFreeAsync(ws.tile_count, s);
    if (e != cudaSuccess) { cudaGetLastError(); return EOD_ECUDA; }
    return EOD_OK;
}

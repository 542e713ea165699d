// Gram matrix G = Y^T Y of a tall, skinny panel Y (m x w, w <= 128) in
// FP64 — the Gram of CholQR (Alg. 1 step 5; Alg. 2 step 9 for small r).
//
// Each CTA stages chunks of 64 rows in shared memory (row-major, so the
// threads of a warp read neighbouring columns) and every thread accumulates
// 4 x 4 blocks of the upper triangle over its rows; per-CTA partial Grams are
// summed in a fixed order by a second kernel.
//
// FP64 data: DFMA accumulation.  FP32 data: each product is formed exactly
// as p + e (p = fl(a b), e = fma(a, b, -p)) and the p's are summed with
// Knuth's TwoSum, the e's and the TwoSum errors in plain FP32, all converted
// to FP64 per CTA: the result matches an FP64 accumulation of the exact
// products to about 2^-46 relative, at FP32 ALU rates.
#include "common.cuh"
#include "instrument.cuh"

#include <algorithm>
#include <type_traits>

namespace eod {
namespace {

constexpr int GR = 64;      // rows per chunk
constexpr int GT = 256;     // threads

template <typename T> struct GramAcc;

template <> struct GramAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <> struct GramAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);          // a*b = p + e exactly
        const float t = s + p;                   // TwoSum(s, p)
        const float z = t - s;
        const float err = (s - (t - z)) + (p - z);
        s = t;
        c += err + e;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// MAXB: 4 x 4 blocks per thread, 1 while the upper triangle has at most GT
// blocks (w <= 88), 2 up to 2 GT (w <= 124), else 3 (w <= 128): the
// accumulators of unused blocks would otherwise hold registers and cap the
// CTAs per SM.
template <typename T, int MAXB>
__global__ void __launch_bounds__(GT) gram_partial_kernel(const T *__restrict__ Y, int64_t m, int w, int64_t ldy,
                                                          int64_t rows_per_cta, double *__restrict__ part) {
    extern __shared__ __align__(16) unsigned char gsm[];
    T *sY = (T *)gsm;                      // GR x (w + 1), row-major
    const int ldsm = w + 1;
    const int nb4 = (w + 3) / 4;
    const int nblocks = nb4 * (nb4 + 1) / 2;   // 4x4 blocks of the upper triangle
    // narrow panels: several thread groups share a block, each taking every
    // rsplit-th row of the chunk; their sums are combined in shared memory
    const int rsplit = nblocks * 2 <= GT ? GT / nblocks : 1;
    const int grp = threadIdx.x / nblocks;     // valid when rsplit > 1
    int bi[MAXB], bj[MAXB], nmine = 0;
    {
        int b0 = rsplit > 1 ? threadIdx.x % nblocks : threadIdx.x;
        const bool active = rsplit > 1 ? grp < rsplit : true;
#pragma unroll
        for (int q = 0; q < MAXB; ++q) {
            const int b = b0 + q * GT;
            if (active && b < nblocks && (rsplit == 1 || q == 0)) {
                int j = (int)((sqrtf(8.f * b + 1.f) - 1.f) * 0.5f);
                while ((j + 1) * (j + 2) / 2 <= b) ++j;
                while (j * (j + 1) / 2 > b) --j;
                bi[q] = b - j * (j + 1) / 2;
                bj[q] = j;
                nmine = q + 1;
            } else {
                bi[q] = bj[q] = 0;
            }
        }
    }
    GramAcc<T> acc[MAXB][4][4];

    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    int64_t r1 = r0 + rows_per_cta;
    if (r1 > m) r1 = m;
    const int rstart = rsplit > 1 ? grp : 0, rstep = rsplit;
    for (int64_t c0 = r0; c0 < r1; c0 += GR) {
        const int rows = (int)((r1 - c0) < GR ? (r1 - c0) : GR);
        __syncthreads();
        for (int e = threadIdx.x; e < GR * w; e += GT) {
            const int r = e % GR, c = e / GR;
            sY[r * ldsm + c] = (r < rows) ? Y[(c0 + r) + (int64_t)c * ldy] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXB; ++q) {
            if (q < nmine) {
                const int i0 = 4 * bi[q], j0 = 4 * bj[q];
                for (int r = rstart; r < rows; r += rstep) {
                    const T *row = sY + r * ldsm;
                    T a[4], b[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        a[t] = (i0 + t < w) ? row[i0 + t] : T(0);
                        b[t] = (j0 + t < w) ? row[j0 + t] : T(0);
                    }
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[q][ii][jj].add(a[ii], b[jj]);
                }
            }
        }
    }
    double *dst = part + (int64_t)blockIdx.x * w * w;
    if (rsplit > 1) {
        // combine the row groups in a fixed order
        __syncthreads();
        double *red = (double *)gsm;           // rsplit x nblocks x 16
        if (nmine > 0) {
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    red[((int64_t)grp * nblocks + (threadIdx.x % nblocks)) * 16 + ii * 4 + jj] = acc[0][ii][jj].value();
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nblocks * 16; e += GT) {
            const int blk = e / 16, ii = (e % 16) / 4, jj = e % 4;
            double sum = 0.0;
            for (int g = 0; g < rsplit; ++g) sum += red[((int64_t)g * nblocks + blk) * 16 + ii * 4 + jj];
            int j = (int)((sqrtf(8.f * blk + 1.f) - 1.f) * 0.5f);
            while ((j + 1) * (j + 2) / 2 <= blk) ++j;
            while (j * (j + 1) / 2 > blk) --j;
            const int i0 = 4 * (blk - j * (j + 1) / 2), j0 = 4 * j;
            if (i0 + ii < w && j0 + jj < w) dst[(i0 + ii) + (j0 + jj) * w] = sum;
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < MAXB; ++q) {
        if (q < nmine) {
            const int i0 = 4 * bi[q], j0 = 4 * bj[q];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (i0 + ii < w && j0 + jj < w) dst[(i0 + ii) + (j0 + jj) * w] = acc[q][ii][jj].value();
        }
    }
}

// Sum of the per-CTA partial Grams, upper triangle: a block takes 32
// consecutive entries, its 8 warps each sum every 8th partial (in order), and
// the 8 warp sums are added in order: the FP64 adds of one entry are spread
// over 8 warps and the result does not depend on timing.
__global__ void __launch_bounds__(256) gram_reduce_kernel(const double *__restrict__ part, int nparts, int w,
                                                          double *G, int64_t ldg) {
    __shared__ double red[8][33];
    const int total = w * w;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double sum = 0.0;
    if (e < total && e % w <= e / w)
        for (int z = g; z < nparts; z += 8) sum += part[(int64_t)z * total + e];
    red[g][lane] = sum;
    __syncthreads();
    if (g == 0 && e < total) {
        const int i = e % w, j = e / w;
        if (i <= j) {
            double t = red[0][lane];
#pragma unroll
            for (int q = 1; q < 8; ++q) t += red[q][lane];
            G[i + (int64_t)j * ldg] = t;
        }
    }
}

// Upper triangle of G = W^T W for FP32 W (rows x p, any p), 64 x 64 tiles of
// G, 256 threads with 4 x 4 outputs each, the exact-product / TwoSum
// accumulation of GramAcc<float>; the row range is split over gridDim.z and
// each split writes its FP64 partial tile (or G itself when unsplit).
constexpr int TBM = 64, TBK = 16;

__global__ void __launch_bounds__(GT) gram_tiled_f32_kernel(const float *__restrict__ W, int64_t rows, int64_t p,
                                                             int64_t ldw, int64_t rows_per_split,
                                                             double *__restrict__ out, int64_t ldo,
                                                             int64_t split_stride) {
    __shared__ float As[TBK][TBM + 1];
    __shared__ float Bs[TBK][TBM + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * TBM, n0 = (int64_t)blockIdx.y * TBM;
    if (m0 > n0 + TBM - 1) return;                     // strictly below the diagonal
    const int64_t kb = (int64_t)blockIdx.z * rows_per_split;
    const int64_t ke = kb + rows_per_split < rows ? kb + rows_per_split : rows;
    GramAcc<float> acc[4][4];
    for (int64_t k0 = kb; k0 < ke; k0 += TBK) {
#pragma unroll
        for (int q = 0; q < (TBM * TBK) / GT; ++q) {
            const int e = tid + q * GT;
            const int kk = e % TBK, i = e / TBK;
            const int64_t gk = k0 + kk;
            As[kk][i] = (gk < ke && m0 + i < p) ? W[gk + (m0 + i) * ldw] : 0.f;
            Bs[kk][i] = (gk < ke && n0 + i < p) ? W[gk + (n0 + i) * ldw] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j].add(a[i], b[j]);
        }
        __syncthreads();
    }
    double *dst = out + (int64_t)blockIdx.z * split_stride;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t col = n0 + ty + 16 * j;
        if (col >= p) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = m0 + tx + 16 * i;
            if (row < p) dst[row + col * ldo] = acc[i][j].value();
        }
    }
}

__global__ void gram_split_reduce_kernel(const double *__restrict__ part, int S, int64_t p, double *G, int64_t ldg) {
    const int64_t total = p * p;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % p, j = e / p;
        if ((i / TBM) * TBM > (j / TBM) * TBM + TBM - 1) continue;
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += part[(int64_t)z * total + e];
        G[i + j * ldg] = s;
    }
}

}  // namespace

cudaError_t gram_tiled_f32(const float *W, int64_t rows, int64_t p, int64_t ldw, double *G, int64_t ldg,
                           Scratch *ws, cudaStream_t s) {
    if (p < 1 || rows < 1) return cudaSuccess;
    const int64_t gt = (p + TBM - 1) / TBM;
    const int64_t tiles = gt * (gt + 1) / 2;
    int64_t S = 1;
    if (tiles < 2 * kNumSMs) {
        S = (2 * kNumSMs + tiles - 1) / tiles;
        const int64_t smax = (rows + 4 * TBK - 1) / (4 * TBK);
        if (S > smax) S = smax;
        if (S < 1) S = 1;
    }
    size_t mark = ws->mark();
    double *part = nullptr;
    while (S > 1) {
        part = (double *)ws->take(sizeof(double) * (size_t)S * p * p);
        if (part) break;
        S /= 2;
    }
    const int64_t rows_per = ((rows + S - 1) / S + TBK - 1) / TBK * TBK;
    S = (rows + rows_per - 1) / rows_per;
    ProfScope prof(PROF_GEMM_SIMT32, (double)rows * p * (p + 1), 4.0 * rows * p, s);
    dim3 grid((unsigned)gt, (unsigned)gt, (unsigned)S);
    if (S > 1) {
        count_launch(2);
        gram_tiled_f32_kernel<<<grid, GT, 0, s>>>(W, rows, p, ldw, rows_per, part, p, p * p);
        EOD_CUDA_TRY(cudaGetLastError());
        const int blocks = (int)std::min<int64_t>((p * p + 255) / 256, 4 * kNumSMs * 4);
        gram_split_reduce_kernel<<<blocks, 256, 0, s>>>(part, (int)S, p, G, ldg);
        EOD_CUDA_TRY(cudaGetLastError());
        ws->release(mark);
    } else {
        count_launch();
        gram_tiled_f32_kernel<<<grid, GT, 0, s>>>(W, rows, p, ldw, rows_per, G, ldg, 0);
        EOD_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t gram_skinny(const T *Y, int64_t m, int w, int64_t ldy, double *G, int64_t ldg, Scratch *ws,
                        cudaStream_t s) {
    if (w < 1 || w > 128) return cudaErrorInvalidValue;
    // at least 16 rows per CTA, up to two CTAs per SM: a short panel still
    // spreads its FP64 work over most SMs
    int64_t ctas = (m + 15) / 16;
    if (ctas > 2 * kNumSMs) ctas = 2 * kNumSMs;
    if (ctas < 1) ctas = 1;
    int64_t rows_per = (m + ctas - 1) / ctas;
    ctas = (m + rows_per - 1) / rows_per;
    if (ctas < 1) ctas = 1;
    size_t mark = ws->mark();
    double *part = (double *)ws->take(sizeof(double) * (size_t)ctas * w * w);
    if (!part) return cudaErrorMemoryAllocation;
    size_t smem = sizeof(T) * (size_t)GR * (w + 1);
    if (smem < sizeof(double) * GT * 16) smem = sizeof(double) * GT * 16;   // room for the row-group sums
    const int nb4 = (w + 3) / 4;
    const int nblk = nb4 * (nb4 + 1) / 2;
    const int maxb = nblk <= GT ? 1 : (nblk <= 2 * GT ? 2 : 3);
    EOD_CUDA_TRY(set_smem_once(gram_partial_kernel<T, 1>, (int)(sizeof(double) * GR * 129)));
    EOD_CUDA_TRY(set_smem_once(gram_partial_kernel<T, 2>, (int)(sizeof(double) * GR * 129)));
    EOD_CUDA_TRY(set_smem_once(gram_partial_kernel<T, 3>, (int)(sizeof(double) * GR * 129)));
    ProfScope prof(std::is_same<T, float>::value ? PROF_GEMM_SIMT32 : PROF_GEMM_SIMT, (double)m * w * (w + 1),
                   (double)sizeof(T) * m * w, s);
    count_launch(2);
    if (maxb == 1) gram_partial_kernel<T, 1><<<(unsigned)ctas, GT, smem, s>>>(Y, m > 0 ? m : 0, w, ldy, rows_per, part);
    else if (maxb == 2) gram_partial_kernel<T, 2><<<(unsigned)ctas, GT, smem, s>>>(Y, m > 0 ? m : 0, w, ldy, rows_per, part);
    else gram_partial_kernel<T, 3><<<(unsigned)ctas, GT, smem, s>>>(Y, m > 0 ? m : 0, w, ldy, rows_per, part);
    EOD_CUDA_TRY(cudaGetLastError());
    gram_reduce_kernel<<<(w * w + 31) / 32, 256, 0, s>>>(part, (int)ctas, w, G, ldg);
    EOD_CUDA_TRY(cudaGetLastError());
    ws->release(mark);
    return cudaSuccess;
}

template cudaError_t gram_skinny<double>(const double *, int64_t, int, int64_t, double *, int64_t, Scratch *, cudaStream_t);
template cudaError_t gram_skinny<float>(const float *, int64_t, int, int64_t, double *, int64_t, Scratch *, cudaStream_t);

}  // namespace eod

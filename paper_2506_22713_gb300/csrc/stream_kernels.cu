// Streaming kernels of the EOD-ABE path: the Gaussian test blocks Omega_j
// (Alg. 1 step 3), the Frobenius norm of A with its finiteness check (the
// denominator of RelErr, Sec. 4.1, and eps in relative-tolerance mode), and
// small copy / scale / fill helpers used between the dense steps.
#include "common.cuh"
#include "instrument.cuh"
#include "omega.cuh"

#include <cuda.h>
#include <algorithm>
#include <type_traits>
#include <mutex>

namespace eod {
namespace {

// Columns from blockIdx.y, rows from blockIdx.x: no index division per entry.
template <typename T>
__global__ void omega_kernel(int64_t n, int64_t col0, int64_t ncols, uint64_t seed, uint32_t batch,
                             T *out, int64_t ldo) {
    for (int64_t c = blockIdx.y; c < ncols; c += gridDim.y)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            out[i + c * ldo] = omega_value_fast<T>(seed, (uint32_t)i, (uint32_t)(col0 + c), batch);
}

// ------------------------------------------------------------- norms ----
template <typename T>
__global__ void sumsq_kernel(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                             double *partials, int *flags) {
    // Tasks are (column, chunk of 4 x blockDim rows): one 64-bit division per
    // task, coalesced rows inside it.  Non-finite entries are found on the
    // exponent bits.  FP64 data: FP64 FMA per entry.  FP32 data: the square
    // is formed exactly as p + e (p = x*x, e = fma(x, x, -p)) and summed with
    // TwoSum in FP32, the errors in a second FP32 accumulator, both widened
    // to FP64 at the end (about 2^-48 relative): the FP64 pipe, 64 cycles per
    // warp instruction on this GPU, stays out of the per-entry work.
    __shared__ double red[32];
    constexpr int U = 4;
    const int64_t chunk = (int64_t)blockDim.x * U;
    const int64_t nch = (m + chunk - 1) / chunk;
    const int64_t tasks = nch * n;
    int bad = 0;
    double dacc = 0.0;
    float s = 0.f, c = 0.f;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int64_t j = t / nch, i0 = (t - j * nch) * chunk;
        const T *col = A + j * lda;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * (int64_t)blockDim.x + threadIdx.x;
            if (i < m) {
                const T x = col[i];
                if (sizeof(T) == 8) {
                    const unsigned long long b = (unsigned long long)__double_as_longlong((double)x);
                    bad |= ((b >> 52) & 0x7ff) == 0x7ff;
                    dacc = fma((double)x, (double)x, dacc);
                } else {
                    const float xf = (float)x;
                    bad |= ((__float_as_uint(xf) >> 23) & 0xff) == 0xff;
                    const float pr = xf * xf;
                    const float er = fmaf(xf, xf, -pr);
                    const float tt = s + pr;
                    const float z = tt - s;
                    c += ((s - (tt - z)) + (pr - z)) + er;
                    s = tt;
                }
            }
        }
    }
    const double acc = (sizeof(T) == 8) ? dacc : (double)s + (double)c;
    const double tot = block_sum(acc, red);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        flags[blockIdx.x] = bad;
    }
}

__global__ void finalize_norm_kernel(const double *partials, const int *pflags, int64_t count,
                                     double *out, int *flag) {
    __shared__ double red[32];
    double acc = 0.0;
    int bad = 0;
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
        acc += partials[e];
        if (pflags) bad |= pflags[e];
    }
    const double tot = block_sum(acc, red);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        out[0] = sqrt(tot);
        if (flag) flag[0] |= bad;
    }
}

__global__ void finalize_sqrt_sum_kernel(const double *partials, int64_t count, const double *denom,
                                         double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) acc += partials[e];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) {
        const double d = denom ? denom[0] : 1.0;
        out[0] = d > 0.0 ? sqrt(tot) / d : (tot > 0.0 ? INFINITY : 0.0);
    }
}

// ------------------------------------------------------------- helpers ----
template <typename TS, typename TD>
__global__ void copy_kernel(const TS *__restrict__ src, int64_t lds, TD *__restrict__ dst, int64_t ldd,
                            int64_t rows, int64_t cols, int transpose) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        // dst(i, j) = src(i, j) or src(j, i)
        dst[i + j * ldd] = (TD)(transpose ? src[j + i * lds] : src[i + j * lds]);
    }
}

template <typename T>
__global__ void scale_kernel(T *x, int64_t m, const double *norm) {
    const double inv = 1.0 / norm[0];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        x[e] = (T)((double)x[e] * inv);
}

template <typename T>
__global__ void zero_kernel(T *x, int64_t rows, int64_t cols, int64_t ld) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        x[(e % rows) + (e / rows) * ld] = T(0);
}

constexpr int64_t kGridCap = 8LL * kNumSMs * 4;   // most blocks any streaming launch uses

inline int grid_for(int64_t total, int per = 256) {
    int64_t b = (total + per - 1) / per;
    const int64_t cap = kGridCap;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

template <typename T>
cudaError_t omega_fill(int64_t n, int64_t col0, int64_t ncols, uint64_t seed, uint64_t batch, T *out,
                       int64_t ldo, cudaStream_t s) {
    if (n <= 0 || ncols <= 0) return cudaSuccess;
    ProfScope prof(PROF_OMEGA, 0.0, (double)sizeof(T) * n * ncols, s);
    count_launch();
    const int gx = (int)std::min<int64_t>((n + 255) / 256, 64);
    const int gy = (int)std::min<int64_t>(ncols, std::max<int64_t>(1, 4LL * kNumSMs * 4 / gx));
    omega_kernel<T><<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(n, col0, ncols, seed, (uint32_t)batch, out, ldo);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fro_norm(const T *A, int64_t m, int64_t n, int64_t lda, double *out, int *flag, Scratch *ws,
                     cudaStream_t s) {
    const int blocks = grid_for(m * n, 512);
    size_t mark = ws->mark();
    double *part = (double *)ws->take(sizeof(double) * blocks);
    int *pf = (int *)ws->take(sizeof(int) * blocks);
    if (!part || !pf) return cudaErrorMemoryAllocation;
    ProfScope prof(PROF_STREAM, 2.0 * m * n, (double)sizeof(T) * m * n, s);
    count_launch(2);
    sumsq_kernel<T><<<blocks, 512, 0, s>>>(A, m, n, lda, part, pf);
    EOD_CUDA_TRY(cudaGetLastError());
    finalize_norm_kernel<<<1, 1024, 0, s>>>(part, pf, blocks, out, flag);
    EOD_CUDA_TRY(cudaGetLastError());
    ws->release(mark);
    return cudaSuccess;
}

cudaError_t finalize_norm(const double *partials, const int *flags, int64_t count, double *out, int *flag,
                          cudaStream_t s) {
    count_launch();
    finalize_norm_kernel<<<1, 1024, 0, s>>>(partials, flags, count, out, flag);
    return cudaGetLastError();
}

cudaError_t finalize_sqrt_sum(const double *partials, int64_t count, const double *denom, double *out,
                              cudaStream_t s) {
    count_launch();
    finalize_sqrt_sum_kernel<<<1, 1024, 0, s>>>(partials, count, denom, out);
    return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t copy_matrix(const TS *src, int64_t lds, TD *dst, int64_t ldd, int64_t rows, int64_t cols,
                        bool transpose, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ProfScope prof(PROF_STREAM, 0.0, (double)(sizeof(TS) + sizeof(TD)) * rows * cols, s);
    count_launch();
    copy_kernel<TS, TD><<<grid_for(rows * cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols, transpose ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t scale_column(T *x, int64_t m, const double *norm, cudaStream_t s) {
    count_launch();
    scale_kernel<T><<<grid_for(m), 256, 0, s>>>(x, m, norm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fill_zero(T *x, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    count_launch();
    zero_kernel<T><<<grid_for(rows * cols), 256, 0, s>>>(x, rows, cols, ld);
    return cudaGetLastError();
}

template cudaError_t omega_fill<double>(int64_t, int64_t, int64_t, uint64_t, uint64_t, double *, int64_t, cudaStream_t);
template cudaError_t omega_fill<float>(int64_t, int64_t, int64_t, uint64_t, uint64_t, float *, int64_t, cudaStream_t);
template cudaError_t omega_fill<__nv_bfloat16>(int64_t, int64_t, int64_t, uint64_t, uint64_t, __nv_bfloat16 *, int64_t,
                                               cudaStream_t);
template cudaError_t fro_norm<double>(const double *, int64_t, int64_t, int64_t, double *, int *, Scratch *, cudaStream_t);
template cudaError_t fro_norm<float>(const float *, int64_t, int64_t, int64_t, double *, int *, Scratch *, cudaStream_t);
template cudaError_t copy_matrix<double, double>(const double *, int64_t, double *, int64_t, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t copy_matrix<float, float>(const float *, int64_t, float *, int64_t, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t copy_matrix<double, float>(const double *, int64_t, float *, int64_t, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t copy_matrix<float, double>(const float *, int64_t, double *, int64_t, int64_t, int64_t, bool, cudaStream_t);
template cudaError_t scale_column<double>(double *, int64_t, const double *, cudaStream_t);
template cudaError_t scale_column<float>(float *, int64_t, const double *, cudaStream_t);
template cudaError_t fill_zero<double>(double *, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t fill_zero<float>(float *, int64_t, int64_t, int64_t, cudaStream_t);

}  // namespace eod

// ===========================================================================
// Allocation-free Frobenius norm (eod_abe_fro_norm_noalloc).
//
// Some callers cannot allocate device memory at all: code that runs while
// another framework owns the device allocator, real-time pipelines that
// forbid allocation after start-up, or a host thread that is recording work
// for later replay.  For them the per-block partial sums and non-finite flags
// of the norm reduction live in this fixed device array instead of the
// per-call workspace.  Every GPU that loads the library holds it until the
// process exits.
// ===========================================================================
namespace eod {
namespace {

constexpr int64_t kNoAllocMaxBlocks = kGridCap;                 // 4864 partials
constexpr int64_t kNoAllocMaxElements = (int64_t)1 << 40;       // largest m*n accepted
constexpr size_t kNoAllocScratchBytes = (size_t)kNoAllocMaxBlocks * (sizeof(double) + sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up (with
// that device current) on the first call made in each context of the device.
// The cache is keyed on the context's unique id as well, so a call made after
// cudaDeviceReset (which destroys the context and may move the array) looks
// the address up again instead of using the old one.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};
unsigned long long g_noalloc_ctx[64] = {};
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// id of the calling thread's current context (0 if it cannot be read)
unsigned long long current_context_id() {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return 0;
        }
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

eod_status noalloc_scratch(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return EOD_ECUDA; }
    if (dev < 0 || dev >= 64) return EOD_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return EOD_ECUDA; }
        g_noalloc_addr[dev] = p;
        // the lookup has made the device's primary context current if it was
        // not yet: record its id now (0 again only if it cannot be read, in
        // which case every call looks the address up)
        g_noalloc_ctx[dev] = current_context_id();
    }
    *out = g_noalloc_addr[dev];
    return EOD_OK;
}

template <typename T>
eod_status fro_norm_noalloc(const T *A, int64_t m, int64_t n, int64_t lda, double *norm_out, int *flag_out,
                            cudaStream_t s) {
    const int blocks = grid_for(m * n, 512);
    if (blocks > kNoAllocMaxBlocks) return EOD_EINVAL;
    void *base = nullptr;
    eod_status st = noalloc_scratch(&base);
    if (st != EOD_OK) return st;
    double *part = (double *)base;
    int *pf = (int *)((char *)base + sizeof(double) * kNoAllocMaxBlocks);
    // the flag is OR-ed by the finalize kernel: clear it first; the partials
    // are all rewritten by this call before they are read
    if (cudaMemsetAsync(flag_out, 0, sizeof(int), s) != cudaSuccess) { cudaGetLastError(); return EOD_ECUDA; }
    // never profiled: the per-launch timing would create CUDA events
    count_launch(2);
    sumsq_kernel<T><<<blocks, 512, 0, s>>>(A, m, n, lda, part, pf);
    if (cudaGetLastError() != cudaSuccess) return EOD_ECUDA;
    finalize_norm_kernel<<<1, 1024, 0, s>>>(part, pf, blocks, norm_out, flag_out);
    if (cudaGetLastError() != cudaSuccess) return EOD_ECUDA;
    return EOD_OK;
}

}  // namespace
}  // namespace eod

extern "C" eod_status eod_abe_fro_norm_noalloc(const void *A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                                               double *norm_out, int32_t *nonfinite_out, void *stream) {
    using namespace eod;
    if (!A || !norm_out || !nonfinite_out || m < 1 || n < 1 || lda < m) return EOD_EINVAL;
    if (m > 0x7FFFFFFFLL || n > 0x7FFFFFFFLL || m * n > kNoAllocMaxElements) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == EOD_F64) return fro_norm_noalloc<double>((const double *)A, m, n, lda, norm_out, (int *)nonfinite_out, s);
    if (dtype == EOD_F32) return fro_norm_noalloc<float>((const float *)A, m, n, lda, norm_out, (int *)nonfinite_out, s);
    return EOD_EINVAL;
}

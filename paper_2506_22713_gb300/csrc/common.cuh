// Shared device helpers and the internal (C++) interface between the
// translation units of the EOD-ABE library.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/eod_abe.h"

namespace eod {

#define EOD_CUDA_TRY(...)                                          \
    do {                                                            \
        cudaError_t eod_err_ = (__VA_ARGS__);                              \
        if (eod_err_ != cudaSuccess) return eod_err_;               \
    } while (0)

constexpr double kU64 = 1.1102230246251565e-16;   // 2^-53, unit roundoff of binary64
constexpr double kU32 = 5.9604644775390625e-08;   // 2^-24, unit roundoff of binary32
constexpr int kNumSMs = 152;

// Raises a kernel's dynamic shared-memory limit once per (kernel, device)
// (thread-safe; a failed attempt is retried by the next caller).
inline cudaError_t set_smem_once_ptr(const void *kernel, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == kernel && d.second == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.emplace_back(kernel, dev);
    return e;
}
template <typename K>
inline cudaError_t set_smem_once(K kernel, int bytes) {
    return set_smem_once_ptr((const void *)kernel, bytes);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_or(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, at
// most 1024).  Every thread gets the total.
__device__ __forceinline__ double block_sum(double v, double *sh32) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh32[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = (threadIdx.x < nw) ? sh32[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh32[0] = t;
    __syncthreads();
    return sh32[0];
}

template <typename T> __device__ __forceinline__ double to_f64(T x) { return (double)x; }

// --------------------------------------------------------------------------
// Bump allocator over one device buffer (the per-call workspace).
// --------------------------------------------------------------------------
// counters a workspace holds for in-kernel K-split folding (one per tile)
constexpr int64_t kTileCounters = 65536;

struct Scratch {
    char *base = nullptr;
    size_t size = 0, used = 0, high = 0;
    int *err_flag = nullptr;   // device flag set by a kernel whose bounded wait ran out
    // zeroed counters, one per output tile, for K splits folded in-kernel
    // (each product leaves them zero again); null: a separate reduction
    unsigned *tile_count = nullptr;
    int64_t tile_count_n = 0;
    void *take(size_t bytes) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        if (used > high) high = used;
        return base + off;
    }
    size_t mark() const { return used; }
    void release(size_t m) { used = m; }
};

// --------------------------------------------------------------------------
// Stream-ordered device allocations owned by one call; freed on the stream
// when the call returns unless handed over with keep().
// --------------------------------------------------------------------------
extern int g_fail_alloc_after;   // test hook: n-th allocation from now fails

// Stream-ordered allocation from the library's own memory pool on the
// current device.  The pool keeps up to 64 GiB of freed blocks mapped, so the
// gigabyte-sized per-call buffers (operand slices, the basis) are not mapped
// and unmapped again on every call, and the caller's default pool is left as
// it is.
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);

struct Arena {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Arena(cudaStream_t st) : s(st) {}
    template <typename T>
    eod_status get(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        if (g_fail_alloc_after > 0) {
            if (--g_fail_alloc_after == 0) return EOD_ENOMEM;
        }
        void *q = nullptr;
        cudaError_t e = lib_malloc_async(&q, sizeof(T) * count, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? EOD_ENOMEM : EOD_ECUDA;
        }
        ptrs.push_back(q);
        *p = (T *)q;
        return EOD_OK;
    }
    void keep(void *p) {
        for (auto &q : ptrs)
            if (q == p) q = nullptr;
    }
    ~Arena() {
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, s);
    }
};

// --------------------------------------------------------------------------
// GEMM (SIMT, any of TA/TB/TC in {float, double}, accumulation Acc):
//   C (M x N) = alpha * op(A) * op(B) + beta * C,  column-major,
//   op(X) = X or X^T.  Split-K through the scratch partials when the tile
//   grid would not fill the GPU; the split partials are summed in a fixed
//   order, so results are deterministic.
// --------------------------------------------------------------------------
enum GemmEpilogue { EPI_STORE = 0, EPI_ERR = 1 };

struct GemmExtra {
    bool upper_only = false;   // only tiles that touch the upper triangle of C
    bool a_upper = false;      // op(A) upper triangular: skip its zero K range
    bool b_upper = false;      // op(B) upper triangular: skip its zero K range
    int epilogue = EPI_STORE;
    const void *ref = nullptr; // EPI_ERR: reference matrix R (M x N, type TC)
    int64_t ldref = 0;
    double *err_partials = nullptr; // EPI_ERR: one double per CTA (gridDim.x*gridDim.y)
    int max_split = 64;
    int force_ts = 0;          // SIMT tile forced by the autotuner's timing hook (0 = plan)
};

// A value of the autotuner's table (tuning.cu) for key at (a, b, c); false
// when the table has none.
bool tuned_value(const char *key, int64_t a, int64_t b, int64_t c, int64_t *out);

template <typename TA, typename TB, typename TC, typename Acc>
cudaError_t gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const TA *A, int64_t lda, const TB *B, int64_t ldb, double beta, TC *C,
                 int64_t ldc, const GemmExtra &x, Scratch *ws, cudaStream_t s);

// most CTAs (partials) the EPI_ERR form of gemm() writes for an M x N output;
// clear that many before the call (the emulated FP64 path writes fewer)
int64_t gemm_err_ctas(int64_t M, int64_t N);

// FP64 GEMM emulated on tcgen05 tensor cores (oz_gemm.cu); same contract as
// gemm<double,...> except that the triangular / upper-only hints are ignored
cudaError_t oz_gemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double beta, double *C, int64_t ldc, const GemmExtra &x,
                    int *err_flag, cudaStream_t s);
// Pre-sliced operand of oz_gemm_ops: 8 BF16 slices of op(X) as rows x K
// (K contiguous, leading dimension ldk, slices slice_stride elements apart)
// with a per-row exponent array e, or e == nullptr and one fixed exponent.
struct OzOperand {
    const void *q = nullptr;   // __nv_bfloat16 slices
    const int *e = nullptr;
    int e_fixed = 0;
    int64_t ldk = 0, slice_stride = 0;
};
cudaError_t oz_gemm_ops(const OzOperand &A, const OzOperand &B, int64_t M, int64_t N, int64_t K, double alpha,
                        double beta, double *C, int64_t ldc, const GemmExtra &x, int *err_flag, cudaStream_t s,
                        float *Cf = nullptr);
// FP32 data through the same emulation (FP32 values are exact in FP64), the
// result rounded once to FP32: C = alpha op(A) op(B) + beta C (EPI_STORE only)
cudaError_t oz_gemm_f32(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const float *A, int64_t lda,
                        const float *B, int64_t ldb, double beta, float *C, int64_t ldc, const GemmExtra &x,
                        int *err_flag, cudaStream_t s);
// slices of op(X) (rows x K, X(r, k) at X[r*sr + k*sk]) into q (ld ldk, slices
// slice_stride apart); per-row exponents into e, or the fixed exponent when e
// is null (every |X| must then be below 2^fixed_e)
cudaError_t oz_slice(const double *X, int64_t rows, int64_t K, int64_t sr, int64_t sk, void *q, int *e,
                     int fixed_e, int64_t ldk, int64_t slice_stride, cudaStream_t s);
constexpr int kOzSlices = 8;
// largest K the emulation takes with the fused squared-error epilogue (which
// cannot split K)
constexpr int64_t kOzErrMaxK = 7168;

// whether gemm<double,...> sends an M x N x K product to oz_gemm
bool fp64_use_emulated(int64_t M, int64_t N, int64_t K);
// whether gemm<float,...> sends an M x N x K product to oz_gemm_f32
bool fp32_use_emulated(int64_t M, int64_t N, int64_t K);

// --------------------------------------------------------------------------
// Streaming kernels
// --------------------------------------------------------------------------
// ||A||_F^2 partials (FP64) + non-finite flag; then finalize into out[0] =
// ||A||_F, flag[0] |= 1 if a NaN/Inf was seen.
template <typename T>
cudaError_t fro_norm(const T *A, int64_t m, int64_t n, int64_t lda, double *out,
                     int *flag, Scratch *ws, cudaStream_t s);
// out = sqrt(sum(partials[0..count))) / denom (denom read from device pointer or 1)
// out[0] = sqrt(sum of the count partials); flag[0] |= any of the flags
cudaError_t finalize_norm(const double *partials, const int *flags, int64_t count, double *out, int *flag,
                          cudaStream_t s);
cudaError_t finalize_sqrt_sum(const double *partials, int64_t count, const double *denom,
                              double *out, cudaStream_t s);
// Omega columns col0.. into out (n x ncols, ld n) in type T (values are BF16-exact)
template <typename T>
cudaError_t omega_fill(int64_t n, int64_t col0, int64_t ncols, uint64_t seed, uint64_t batch,
                       T *out, int64_t ldo, cudaStream_t s);
template <typename TS, typename TD>
cudaError_t copy_matrix(const TS *src, int64_t lds, TD *dst, int64_t ldd, int64_t rows,
                        int64_t cols, bool transpose, cudaStream_t s);
template <typename T>
cudaError_t scale_column(T *x, int64_t m, const double *inv_norm_src, cudaStream_t s);
template <typename T>
cudaError_t fill_zero(T *x, int64_t rows, int64_t cols, int64_t ld, cudaStream_t s);

// G (w x w, upper triangle, FP64, ld ldg) = Y^T Y for a tall panel Y (m x w,
// w <= 128); FP64 accumulation of the exact products (gram.cu).
template <typename T>
cudaError_t gram_skinny(const T *Y, int64_t m, int w, int64_t ldy, double *G, int64_t ldg, Scratch *ws,
                        cudaStream_t s);

// Upper triangle of G (p x p, FP64, ld ldg) = W^T W for FP32 W (rows x p,
// any p): exact products and TwoSum accumulation in FP32, FP64 per tile.
cudaError_t gram_tiled_f32(const float *W, int64_t rows, int64_t p, int64_t ldw, double *G, int64_t ldg,
                           Scratch *ws, cudaStream_t s);

// --------------------------------------------------------------------------
// Small dense factorisations (one CTA)
// --------------------------------------------------------------------------
enum CholCode { CHOL_ALL = 0, CHOL_BELOW = 1, CHOL_UNCERTAIN = 2, CHOL_FAIL = 3 };

// Cholesky G = R^T R of the w x w matrix G (upper triangle read, FP64; one
// CTA, computed as L D L^T) with the rank decision of Alg. 1 steps 6-11 when
// decide != 0:
//   info[0] = p (leading columns factored), info[1] = CholCode,
// R (p x p upper, ld ldr) and its inverse Rinv (ld ldr); the original
// diagonal of G is used for the rounding margin.
// ni_tau2 > 0 (only with decide == 0 and shift == 0): when ||G - I||_F^2 <=
// ni_tau2 the factor is taken to first order, R = I + Phi(G - I), R^{-1} =
// I - Phi(G - I) (Phi: strict upper part plus half the diagonal; error
// O(||G - I||^2)), without the factorisation.
cudaError_t chol_small(const double *G, int64_t ldg, int w, int decide, double eps2,
                       double delta_coef, double rho, double shift, double *R, int64_t ldr,
                       double *Rinv, int64_t ldinv, int *info, cudaStream_t s, double ni_tau2 = 0.0,
                       bool classic = false);
// out[0] = ||G - I||_F^2 of the symmetric p x p matrix G (upper triangle
// read), through kOffIdMaxBlocks partial sums in `part`
constexpr int kOffIdMaxBlocks = 608;
cudaError_t offidentity_sumsq(const double *G, int64_t ldg, int64_t p, double *part, double *out, cudaStream_t s);
// the first-order factor of a near-identity G (see chol_small): R (p x p,
// ld ldr, zeros below the diagonal) and the inverses of its diagonal panels
// of width pb at RiD + J pb^2 (ld pb)
cudaError_t near_identity_factor(const double *G, int64_t ldg, int64_t p, double *R, int64_t ldr, double *RiD,
                                 int pb, cudaStream_t s);
// tdiag[j] = |R1(j,j) * R2(j,j)|, j < p
cudaError_t tdiag_product(const double *R1, const double *R2, int64_t ldr, const int *p_dev,
                          double *tdiag, cudaStream_t s);
// trace(G) for the shift of shifted CholQR
cudaError_t trace_sum(const double *G, int64_t ldg, int64_t p, double *out, cudaStream_t s);

}  // namespace eod

// Tensor-core contractions of the mixed path on sm_103a: tcgen05.mma
// (kind::f16 with BF16 operands, or kind::tf32 with FP32-stored TF32
// operands; FP32 accumulation in TMEM) fed by TMA.
//
//   sketch          Y   = (A_hi + A_lo + A_3) Omega   Alg. 1 step 4
//   projection      C^T = A_hi^T Q_hi + A_hi^T Q_lo + A_lo^T Q_hi    Alg. 2 step 8
//   reconstruction  sum (A - Q C)^2 over a tile       Sec. 4.1 RelErr, with
//                   Q C = Q_hi C_hi + Q_hi C_lo + Q_lo C_hi
//
// A FP32 matrix X is split as X_hi = bf16(X), X_lo = bf16(X - X_hi) (round
// to nearest even); the dropped X_lo Y_lo term and the split's own residual
// are about 2^-16 relative.  For the sketch A gets a third term A_3 =
// bf16(A - A_hi - A_lo), which makes the split exact for FP32 data; Omega is
// BF16-exact, so the sketch is then as accurate as an FP32 GEMM.
// The TF32 form splits X as X_hi = X with its 13 low significand bits
// cleared (exact in TF32) and X_lo = X - X_hi (exact in FP32, at most 13
// significant bits, of which TF32 keeps 11): the dropped terms are about
// 2^-21 relative, at half the BF16 MMA rate and twice the operand bytes.
// TF32 operands are K-major only (the sketch reads a transposed copy of A).
//
// One CTA computes a 128 x BN tile of D.  Warp 0 issues TMA loads into a
// ring of shared-memory stages (128-byte swizzle), warp 1 allocates TMEM and
// one of its threads issues the MMAs (4 per 64-wide K block), warps 2-5 read
// the accumulator back with tcgen05.ld (warp w owns TMEM lanes 32*(w%4) ..)
// and run the epilogue.  A tile is "pairs" of (A operand, B operand) tensor
// maps accumulated into the same TMEM columns, interleaved per K block so a
// re-read A tile hits L2.  Every mbarrier wait is bounded; a wait that runs
// out sets an error flag the host turns into EOD_ETIMEOUT, and the CTA still
// releases its TMEM and exits.
#include "common.cuh"
#include "instrument.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace eod {
namespace tc {

constexpr int BM = 128;           // MMA M (one CTA, cta_group::1)
constexpr int BK = 64;            // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int UMMA_K = 16;        // K per tcgen05.mma (kind::f16)
constexpr int BK_TF32 = 32;       // K per stage in the TF32 form: 32 FP32 = one 128-byte row
constexpr int NTHREADS = 192;
// Both forms advance 32 bytes of K per MMA (16 BF16 or 8 TF32 elements) and
// 128 bytes per stage, so the shared-memory layout and descriptors are shared.

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 2-D FP32 map, 128-byte swizzle: the BF16 map's geometry in 4-byte elements
inline bool make_map_f32(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint64_t ld,
                         uint32_t box_in, uint32_t box_out) {
    auto fn = encode_fn();
    if (!fn) return false;
    if (((uintptr_t)base & 15) || ((ld * 4) & 15)) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {box_in, box_out};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- kernel ----
struct Maps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

struct Params {
    int64_t M, N;          // output size
    int64_t kblocks;       // K blocks (of 64) in the whole K range
    int64_t kblocks_per_split;
    int npairs;
    float *D;              // EPI_STORE: output (or split partial base), column-major
    int64_t ldd;
    float alpha, beta;     // EPI_STORE: D = alpha acc + beta D (split partials: 1, 0)
    int64_t split_stride;  // elements between split partials (0: no split)
    const float *R;        // EPI_ERR: reference
    int64_t ldr;
    double *errp;          // EPI_ERR: one partial per CTA
    int *err_flag;         // timeout flag
};

template <bool A_MN, int BN_, int EPI>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;          // 16 KB
    static constexpr int B_BYTES = BN_ * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // The fused error epilogue reads a tile of A after the MMAs; two stages
    // leave room for a second CTA on the SM, whose MMAs overlap that read.
    static constexpr int STAGES = (EPI == EPI_ERR) ? 2 : ((BN_ >= 256) ? 4 : (BN_ >= 128 ? 6 : 8));
    static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr uint32_t TMEM_COLS = BN_ < 32 ? 32 : BN_;
};

template <bool A_MN, int BN_, int EPI, bool TF32>
__global__ void __launch_bounds__(NTHREADS, EPI == EPI_ERR ? 2 : 1) tc_gemm_kernel(const __grid_constant__ Maps maps,
                                                                                   Params p) {
    static_assert(!(TF32 && A_MN), "TF32 operands are K-major");
    using C = Cfg<A_MN, BN_, EPI>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + C::STAGES * C::STAGE);
    uint64_t *empty = full + C::STAGES;
    uint64_t *tmem_full = empty + C::STAGES;
    uint32_t *tmem_slot = (uint32_t *)(tmem_full + 1);
    int *abort_sh = (int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN_;
    const int64_t kb0 = (int64_t)blockIdx.z * p.kblocks_per_split;
    int64_t kb1 = kb0 + p.kblocks_per_split;
    if (kb1 > p.kblocks) kb1 = p.kblocks;
    const int64_t iters = (kb1 > kb0 ? kb1 - kb0 : 0) * p.npairs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tmem_full, 1);
        *abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        // Warp-uniform loop, one elected lane issues (single-thread divergent
        // control flow around the async instructions slows their issue).
        const bool leader = elect_one();
        for (int64_t it = 0; it < iters; ++it) {
            const int s = (int)(it % C::STAGES);
            const uint32_t round = (uint32_t)(it / C::STAGES);
            if (it >= C::STAGES && !warp_wait(&empty[s], (round - 1) & 1)) {
                if (leader) {
                    atomicExch(p.err_flag, 1);
                    *abort_sh = 1;
                }
                break;
            }
            if (__any_sync(0xffffffffu, *(volatile int *)abort_sh != 0)) break;
            if (leader) {
                const int pair = (int)(it % p.npairs);
                const int64_t kb = kb0 + it / p.npairs;
                uint8_t *sa = smem + s * C::STAGE;
                uint8_t *sb = sa + C::A_BYTES;
                mbar_expect_tx(&full[s], C::STAGE);
                const int k_el = (int)(kb * (TF32 ? BK_TF32 : BK));
                if (A_MN) {
                    // A stored M-contiguous: two 64 (M) x 64 (K) boxes
                    tma_load_2d(sa, &maps.a[pair], &full[s], (int)m0, k_el);
                    tma_load_2d(sa + BM * BK, &maps.a[pair], &full[s], (int)m0 + 64, k_el);
                } else {
                    tma_load_2d(sa, &maps.a[pair], &full[s], k_el, (int)m0);
                }
                tma_load_2d(sb, &maps.b[pair], &full[s], k_el, (int)n0);
            }
            __syncwarp();
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        const bool leader = elect_one();
        constexpr uint32_t idesc = TF32 ? idesc_tf32(BM, BN_) : idesc_bf16(BM, BN_, A_MN, false);
        for (int64_t it = 0; it < iters; ++it) {
            const int s = (int)(it % C::STAGES);
            const uint32_t round = (uint32_t)(it / C::STAGES);
            if (!warp_wait(&full[s], round & 1)) {
                if (leader) {
                    atomicExch(p.err_flag, 1);
                    *abort_sh = 1;
                }
                break;
            }
            if (__any_sync(0xffffffffu, *(volatile int *)abort_sh != 0)) break;
            tc_fence_after();
            if (leader) {
                const uint32_t sa = smem_u32(smem + s * C::STAGE);
                const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                    uint64_t ad, bd;
                    if (A_MN) ad = sdesc(sa + kk * (UMMA_K * 128), BM * BK, 1024);   // LBO: next 64-row M block
                    else ad = sdesc(sa + kk * (UMMA_K * 2), 16, 1024);
                    bd = sdesc(sb + kk * (UMMA_K * 2), 16, 1024);
                    if (TF32) umma_tf32(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                    else umma_bf16(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            __syncwarp();
        }
        if (leader) umma_commit(tmem_full);   // completes once every MMA issued above has finished
    } else if (warp >= 2 && EPI == EPI_ERR) {
        // ---------------- error epilogue ----------------
        // Each thread owns one row of the tile.  The reference entries of a
        // chunk of 32 columns are loaded before the accumulators are ready (the
        // first chunk while the MMAs still run) and one chunk ahead of the
        // arithmetic afterwards, so their latency overlaps the TMEM reads
        // and the sums instead of following them.
        constexpr int CW = 32;
        const int q = warp & 3;
        const int64_t row = m0 + 32 * q + lane;
        const bool rin = row < p.M;
        float rn[CW];
        auto load_ref = [&](int c) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const int64_t col = n0 + c + j;
                rn[j] = (rin && col < p.N) ? __ldcs(p.R + row + col * p.ldr) : 0.0f;
            }
        };
        load_ref(0);
        const bool got = __all_sync(0xffffffffu, mbar_wait(tmem_full, 0) ? 1 : 0) != 0;
        if (!got) atomicExch(p.err_flag, 1);
        tc_fence_after();
        double local = 0.0;
        if (got && iters > 0) {
#pragma unroll 1
            for (int c = 0; c < BN_; c += CW) {
                float rc[CW];
#pragma unroll
                for (int j = 0; j < CW; ++j) rc[j] = rn[j];
                if (c + CW < BN_) load_ref(c + CW);
                float v[CW];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c + 16), v + 16);
                // residual in FP32 (the difference of two FP32 values), squares
                // summed in FP32 over the 32 columns, FP64 across chunks
                float part = 0.f;
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const float d = (n0 + c + j < p.N) ? rc[j] - v[j] : 0.0f;
                    part = fmaf(d, d, part);
                }
                if (rin) local += (double)part;
            }
        }
        local = warp_sum(local);
        __shared__ double red[4];
        if (lane == 0) red[q] = local;
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps
        if (warp == 2 && lane == 0) p.errp[blockIdx.x + (int64_t)blockIdx.y * gridDim.x] = red[0] + red[1] + red[2] + red[3];
    } else if (warp >= 2) {
        // ---------------- store epilogue ----------------
        const int q = warp & 3;   // TMEM lane quarter this warp may access
        const bool got = __all_sync(0xffffffffu, mbar_wait(tmem_full, 0) ? 1 : 0) != 0;
        if (!got) atomicExch(p.err_flag, 1);
        tc_fence_after();
        const int64_t row = m0 + 32 * q + lane;
        if (got && iters > 0) {
#pragma unroll 1
            for (int c = 0; c < BN_; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
                if (row < p.M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t col = n0 + c + j;
                        if (col < p.N) {
                            float *d = p.D + (int64_t)blockIdx.z * p.split_stride + row + col * p.ldd;
                            *d = p.beta != 0.f ? fmaf(p.alpha, v[j], p.beta * *d) : p.alpha * v[j];
                        }
                    }
                }
            }
        } else if (iters == 0 && row < p.M) {
            for (int c = 0; c < BN_; ++c) {
                const int64_t col = n0 + c;
                if (col < p.N) {
                    float *d = p.D + (int64_t)blockIdx.z * p.split_stride + row + col * p.ldd;
                    *d = p.beta != 0.f ? p.beta * *d : 0.0f;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

__global__ void split_reduce_kernel(const float *__restrict__ part, int64_t M, int64_t N, int S, float *D,
                                    int64_t ldd, float alpha, float beta) {
    const int64_t total = M * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < S; ++z) s += part[(int64_t)z * total + e];
        float *d = D + (e % M) + (e / M) * ldd;
        *d = beta != 0.f ? fmaf(alpha, s, beta * *d) : alpha * s;
    }
}

// --------------------------------------------------------- split kernels ----
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// X (rows x cols, ldx, FP32) -> X_hi, X_lo (same shape, ld ldo) and, when
// x3 != nullptr, X_3 = bf16(X - X_hi - X_lo), so that X_hi + X_lo + X_3 == X
// exactly for normal FP32 values (three 8-bit significands); with partials
// != nullptr also the S0 sums of squares and non-finite flags per block.
__global__ void split_norm_kernel(const float *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                  __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                                  __nv_bfloat16 *__restrict__ x3, int64_t ldo, double *partials, int *flags) {
    // (column, chunk of 4 x blockDim rows) tasks: one 64-bit division per
    // task; the sum of squares compensated in FP32 (exact squares p + e,
    // TwoSum), widened to FP64 per thread; non-finite entries on the bits
    __shared__ double red[32];
    constexpr int U = 4;
    const int64_t chunk = (int64_t)blockDim.x * U;
    const int64_t nch = (rows + chunk - 1) / chunk;
    const int64_t tasks = nch * cols;
    int bad = 0;
    float sacc = 0.f, cacc = 0.f;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const int64_t j = t / nch, i0 = (t - j * nch) * chunk;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * (int64_t)blockDim.x + threadIdx.x;
            if (i < rows) {
                const float x = X[i + j * ldx];
                bad |= ((__float_as_uint(x) >> 23) & 0xff) == 0xff;
                const float pr = x * x;
                const float er = fmaf(x, x, -pr);
                const float tt = sacc + pr;
                const float z = tt - sacc;
                cacc += ((sacc - (tt - z)) + (pr - z)) + er;
                sacc = tt;
                __nv_bfloat16 h, l;
                split_bf16(x, h, l);
                hi[i + j * ldo] = h;
                lo[i + j * ldo] = l;
                if (x3) x3[i + j * ldo] = __float2bfloat16_rn((x - __bfloat162float(h)) - __bfloat162float(l));
            }
        }
    }
    if (partials) {
        const double tot = block_sum((double)sacc + (double)cacc, red);
        bad = __syncthreads_or(bad);
        if (threadIdx.x == 0) {
            partials[blockIdx.x] = tot;
            flags[blockIdx.x] = bad;
        }
    }
}

// Xt_hi/lo (cols x rows, ld ldt) = split(X^T), X rows x cols (ldx), FP32.
__global__ void split_transpose_kernel(const float *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                       __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo, int64_t ldt) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t i = i0 + threadIdx.x, j = j0 + dy;
        tile[dy][threadIdx.x] = (i < rows && j < cols) ? X[i + j * ldx] : 0.f;
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t j = j0 + threadIdx.x, i = i0 + dy;   // output (j, i) = X(i, j)
        if (i < rows && j < cols) {
            __nv_bfloat16 h, l;
            split_bf16(tile[threadIdx.x][dy], h, l);
            hi[j + i * ldt] = h;
            lo[j + i * ldt] = l;
        }
    }
}

// TF32 split of one FP32 value: hi = x with its 13 low significand bits
// cleared (exactly a TF32 value), lo = x - hi (exact in FP32).
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

// X (rows x cols, ldx) -> X_hi, X_lo (same shape, ld ldo), FP32 storage.
// (FP64 input is rounded to FP32 first)
template <typename TI>
__global__ void split_tf32_kernel(const TI *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                  float *__restrict__ hi, float *__restrict__ lo, int64_t ldo) {
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / rows, i = e - j * rows;
        float h, l;
        split_tf32((float)X[i + j * ldx], h, l);
        hi[i + j * ldo] = h;
        lo[i + j * ldo] = l;
    }
}

// Xt_hi / Xt_lo (cols x rows, ld ldt) = TF32 split of X^T, X rows x cols (ldx).
__global__ void split_transpose_tf32_kernel(const float *__restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                            float *__restrict__ hi, float *__restrict__ lo, int64_t ldt) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t i = i0 + threadIdx.x, j = j0 + dy;
        tile[dy][threadIdx.x] = (i < rows && j < cols) ? X[i + j * ldx] : 0.f;
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t j = j0 + threadIdx.x, i = i0 + dy;   // output (j, i) = X(i, j)
        if (i < rows && j < cols) {
            float h, l;
            split_tf32(tile[threadIdx.x][dy], h, l);
            hi[j + i * ldt] = h;
            lo[j + i * ldt] = l;
        }
    }
}

template <bool A_MN, int BN_, int EPI, bool TF32>
cudaError_t launch_tc(const Maps &maps, Params p, int splits, cudaStream_t s) {
    using C = Cfg<A_MN, BN_, EPI>;
    EOD_CUDA_TRY(set_smem_once(tc_gemm_kernel<A_MN, BN_, EPI, TF32>, C::SMEM));
    dim3 grid((unsigned)((p.M + BM - 1) / BM), (unsigned)((p.N + BN_ - 1) / BN_), (unsigned)splits);
    count_launch();
    tc_gemm_kernel<A_MN, BN_, EPI, TF32><<<grid, NTHREADS, C::SMEM, s>>>(maps, p);
    return cudaGetLastError();
}

template <bool A_MN, int EPI, bool TF32>
cudaError_t launch_bn(int bn, const Maps &maps, const Params &p, int splits, cudaStream_t s) {
    switch (bn) {
    case 32: return launch_tc<A_MN, 32, EPI, TF32>(maps, p, splits, s);
    case 64: return launch_tc<A_MN, 64, EPI, TF32>(maps, p, splits, s);
    case 128: return launch_tc<A_MN, 128, EPI, TF32>(maps, p, splits, s);
    default: return launch_tc<A_MN, 256, EPI, TF32>(maps, p, splits, s);
    }
}

int pick_bn(int64_t N) {
    if (N <= 32) return 32;
    if (N <= 64) return 64;
    if (N <= 128) return 128;
    return 256;
}

}  // namespace tc

// Runs one tensor-core contraction (see tc_gemm.cuh).
cudaError_t tc_gemm_run(const TcGemmDesc &g, Scratch *ws, cudaStream_t s) {
    using namespace tc;
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const int bn = g.bn > 0 ? g.bn : pick_bn(g.N);
    if (g.tf32 && g.a_mn_major) return cudaErrorInvalidValue;
    Maps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int i = 0; i < g.npairs; ++i) {
        const TcOperand &a = g.a[i], &b = g.b[i];
        bool ok;
        if (g.tf32) {
            ok = make_map_f32(&maps.a[i], a.ptr, a.inner, a.outer, a.ld, BK_TF32, BM) &&
                 make_map_f32(&maps.b[i], b.ptr, b.inner, b.outer, b.ld, BK_TF32, (uint32_t)bn);
        } else {
            ok = g.a_mn_major ? make_map(&maps.a[i], a.ptr, a.inner, a.outer, a.ld, 64, 64)
                              : make_map(&maps.a[i], a.ptr, a.inner, a.outer, a.ld, 64, BM);
            ok = ok && make_map(&maps.b[i], b.ptr, b.inner, b.outer, b.ld, 64, (uint32_t)bn);
        }
        if (!ok) return cudaErrorInvalidValue;
    }
    Params p;
    p.M = g.M;
    p.N = g.N;
    p.kblocks = (g.K + (g.tf32 ? BK_TF32 : BK) - 1) / (g.tf32 ? BK_TF32 : BK);
    p.npairs = g.npairs;
    p.err_flag = g.err_flag;
    p.R = g.ref;
    p.ldr = g.ldref;
    p.errp = g.err_partials;
    const int64_t tiles = ((g.M + BM - 1) / BM) * ((g.N + bn - 1) / bn);
    int splits = 1;
    if (g.epilogue == EPI_STORE && tiles < kNumSMs && p.kblocks >= 8) {
        splits = (int)((kNumSMs + tiles - 1) / tiles);
        if (splits > p.kblocks / 4) splits = (int)(p.kblocks / 4);
        if (splits > 8) splits = 8;
        if (splits < 1) splits = 1;
    }
    float *part = nullptr;
    size_t mark = ws ? ws->mark() : 0;
    if (splits > 1) {
        part = ws ? (float *)ws->take(sizeof(float) * (size_t)splits * g.M * g.N) : nullptr;
        if (!part) splits = 1;
    }
    p.kblocks_per_split = (p.kblocks + splits - 1) / splits;
    // the method's flops: one product (the split's extra pairs are the
    // implementation's overhead, not counted)
    const double flops = 2.0 * g.M * g.N * g.K;
    const double bytes = (g.tf32 ? 4.0 : 2.0) * g.npairs * ((double)g.M * g.K + (double)g.K * g.N) +
                         (g.epilogue == EPI_ERR ? 4.0 * g.M * g.N : 4.0 * g.M * g.N);
    ProfScope prof(PROF_TC_GEMM, flops, bytes, s);
    if (splits > 1) {
        p.D = part;
        p.ldd = g.M;
        p.split_stride = g.M * g.N;
        p.alpha = 1.f;
        p.beta = 0.f;
    } else {
        p.D = g.D;
        p.ldd = g.ldd;
        p.split_stride = 0;
        p.alpha = g.alpha;
        p.beta = g.beta;
    }
    cudaError_t e;
    if (g.tf32)
        e = g.epilogue == EPI_ERR ? launch_bn<false, EPI_ERR, true>(bn, maps, p, 1, s)
                                  : launch_bn<false, EPI_STORE, true>(bn, maps, p, splits, s);
    else if (g.epilogue == EPI_ERR)
        e = g.a_mn_major ? launch_bn<true, EPI_ERR, false>(bn, maps, p, 1, s)
                         : launch_bn<false, EPI_ERR, false>(bn, maps, p, 1, s);
    else
        e = g.a_mn_major ? launch_bn<true, EPI_STORE, false>(bn, maps, p, splits, s)
                         : launch_bn<false, EPI_STORE, false>(bn, maps, p, splits, s);
    if (e != cudaSuccess) return e;
    if (splits > 1) {
        int blocks = (int)std::min<int64_t>((g.M * g.N + 255) / 256, 4 * kNumSMs * 8);
        count_launch();
        split_reduce_kernel<<<blocks, 256, 0, s>>>(part, g.M, g.N, splits, g.D, g.ldd, g.alpha, g.beta);
        EOD_CUDA_TRY(cudaGetLastError());
        ws->release(mark);
    }
    return cudaSuccess;
}

int64_t tc_gemm_err_ctas(int64_t M, int64_t N, int bn) {
    if (bn <= 0) bn = tc::pick_bn(N);
    return ((M + tc::BM - 1) / tc::BM) * ((N + bn - 1) / bn);
}

cudaError_t split_norm(const float *X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16 *hi,
                       __nv_bfloat16 *lo, int64_t ldo, double *partials, int *flags, int blocks, cudaStream_t s,
                       __nv_bfloat16 *x3) {
    ProfScope prof(PROF_STREAM, 2.0 * rows * cols, (x3 ? 10.0 : 8.0) * rows * cols, s);
    count_launch();
    tc::split_norm_kernel<<<blocks, 512, 0, s>>>(X, rows, cols, ldx, hi, lo, x3, ldo, partials, flags);
    return cudaGetLastError();
}

cudaError_t split_tf32(const float *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo, int64_t ldo,
                       cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ProfScope prof(PROF_STREAM, 0.0, 12.0 * rows * cols, s);
    count_launch();
    const int64_t blocks = std::min<int64_t>((rows * cols + 255) / 256, 8LL * kNumSMs * 4);
    tc::split_tf32_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(X, rows, cols, ldx, hi, lo, ldo);
    return cudaGetLastError();
}

cudaError_t split_tf32_f64(const double *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo,
                           int64_t ldo, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ProfScope prof(PROF_STREAM, 0.0, 16.0 * rows * cols, s);
    count_launch();
    const int64_t blocks = std::min<int64_t>((rows * cols + 255) / 256, 8LL * kNumSMs * 4);
    tc::split_tf32_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(X, rows, cols, ldx, hi, lo, ldo);
    return cudaGetLastError();
}

cudaError_t split_transpose_tf32(const float *X, int64_t rows, int64_t cols, int64_t ldx, float *hi, float *lo,
                                 int64_t ldt, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ProfScope prof(PROF_STREAM, 0.0, 12.0 * rows * cols, s);
    count_launch();
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    tc::split_transpose_tf32_kernel<<<grid, dim3(32, 8), 0, s>>>(X, rows, cols, ldx, hi, lo, ldt);
    return cudaGetLastError();
}

cudaError_t split_transpose(const float *X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16 *hi,
                            __nv_bfloat16 *lo, int64_t ldt, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    ProfScope prof(PROF_STREAM, 0.0, 8.0 * rows * cols, s);
    count_launch();
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    tc::split_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(X, rows, cols, ldx, hi, lo, ldt);
    return cudaGetLastError();
}

}  // namespace eod

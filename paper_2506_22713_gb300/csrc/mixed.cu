// The mixed-precision forms of the three O(mnr) contractions of power-free
// EOD-ABE, on tcgen05 tensor cores (tc_gemm.cu):
//
//  * sketch (Alg. 1 step 4): A Omega for a window of global Omega columns
//    computed in one pass over A.  A Omega_j does not depend on the basis
//    kept so far, so sketching several blocks at once and deflating each
//    block when its turn comes gives exactly the blocks of Alg. 1; the
//    window starts at 2k columns and doubles (up to 1024) while no break
//    occurs, so a rank-r run reads A about log2(r/k) times for the sketch.
//  * projection (Alg. 2 step 8): C^T = A^T Q.
//  * reconstruction error (Sec. 4.1): sum (A - Q C)^2, never storing Q C.
//
// BF16 form: A is split once into BF16 A_hi + A_lo + A_3 (exact for FP32
// data; the sketch uses all three terms, the projection and the error the
// first two); Q and C are split into two terms before their products.
// TF32 form: A, Q and C are split into two TF32 terms in FP32 storage (hi =
// the value with 13 low significand bits cleared, lo = the exact rest), and
// the sketch multiplies a transposed copy of A's terms (kind::tf32 operands
// are K-major); the same three pair products per contraction, two for the
// sketch (Omega is exact in TF32).  Deflation, CholQR, the rank test and the
// core stay on the FP32 SIMT / FP64 kernels of the plain path.
#include "common.cuh"
#include "instrument.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace eod {

#define MX_TRY(...)                                                     \
    do {                                                                \
        cudaError_t mx_e_ = (__VA_ARGS__);                              \
        if (mx_e_ != cudaSuccess) {                                     \
            cudaGetLastError();                                         \
            return mx_e_ == cudaErrorMemoryAllocation ? EOD_ENOMEM : EOD_ECUDA; \
        }                                                               \
    } while (0)
#define MX_ST(...)                                                      \
    do {                                                                \
        eod_status mx_s_ = (__VA_ARGS__);                               \
        if (mx_s_ != EOD_OK) return mx_s_;                              \
    } while (0)

static int stream_blocks(int64_t total) {
    int64_t b = (total + 511) / 512;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8LL * kNumSMs * 4));
}

eod_status MixedOps<float>::prepare(const float *A_, int64_t m_, int64_t n_, int64_t lda_, int64_t k_, Arena &ar_,
                                    Scratch *ws_, cudaStream_t s, bool tf32_, double *d_norm, int *d_flag) {
    A = A_;
    m = m_;
    n = n_;
    lda = lda_;
    k = k_;
    ar = &ar_;
    ws = ws_;
    tf32 = tf32_;
    cap = std::min(m, n);
    ldm8 = round_up(m, 8);
    ldn8 = round_up(n, 8);
    MX_ST(ar->get(&err_flag, 1));
    MX_TRY(cudaMemsetAsync(err_flag, 0, sizeof(int), s));
    win_cap = std::min<int64_t>(cap, 1024);
    next_w = std::min<int64_t>(std::max<int64_t>(2 * k, 64), win_cap);
    MX_ST(ar->get(&Yw, (size_t)m * win_cap));
    if (tf32) {
        MX_ST(ar->get(&Th, (size_t)ldm8 * n));
        MX_ST(ar->get(&Tl, (size_t)ldm8 * n));
        MX_ST(ar->get(&Tth, (size_t)ldn8 * m));
        MX_ST(ar->get(&Ttl, (size_t)ldn8 * m));
        MX_TRY(split_tf32(A, m, n, lda, Th, Tl, ldm8, s));
        MX_TRY(split_transpose_tf32(A, m, n, lda, Tth, Ttl, ldn8, s));
        MX_ST(ar->get(&Om32, (size_t)ldn8 * win_cap));
        return EOD_OK;
    }
    MX_ST(ar->get(&Ahi, (size_t)ldm8 * n));
    MX_ST(ar->get(&Alo, (size_t)ldm8 * n));
    MX_ST(ar->get(&A3, (size_t)ldm8 * n));
    const int blocks = stream_blocks(m * n);
    double *part = nullptr;
    int *pflag = nullptr;
    if (d_norm) {
        MX_ST(ar->get(&part, (size_t)blocks));
        MX_ST(ar->get(&pflag, (size_t)blocks));
    }
    MX_TRY(split_norm(A, m, n, lda, Ahi, Alo, ldm8, part, pflag, blocks, s, A3));
    if (d_norm) MX_TRY(finalize_norm(part, pflag, blocks, d_norm, d_flag, s));
    MX_ST(ar->get(&Om, (size_t)ldn8 * win_cap));
    return EOD_OK;
}

eod_status MixedOps<float>::sketch(int64_t col0, int64_t f, uint64_t seed, uint64_t batch, float *Y, int64_t ldy,
                                   cudaStream_t s) {
    if (win_c0 < 0 || col0 < win_c0 || col0 + f > win_c0 + win_w) {
        // a new window of Omega columns starting at col0
        int64_t w = std::max(next_w, f);
        w = std::min(w, std::min(win_cap, cap - col0));
        w = std::max(w, f);
        TcGemmDesc g;
        g.M = m;
        g.N = w;
        g.K = n;
        if (tf32) {
            MX_TRY(omega_fill<float>(n, col0, w, seed, batch, Om32, ldn8, s));
            g.tf32 = true;
            g.npairs = 2;
            g.a[0] = {Tth, n, m, ldn8};
            g.a[1] = {Ttl, n, m, ldn8};
            g.b[0] = {Om32, n, w, ldn8};
            g.b[1] = g.b[0];
        } else {
            MX_TRY(omega_fill<__nv_bfloat16>(n, col0, w, seed, batch, Om, ldn8, s));
            g.a_mn_major = true;
            g.npairs = 3;
            g.a[0] = {Ahi, m, n, ldm8};
            g.a[1] = {Alo, m, n, ldm8};
            g.a[2] = {A3, m, n, ldm8};
            g.b[0] = {Om, n, w, ldn8};
            g.b[1] = g.b[0];
            g.b[2] = g.b[0];
        }
        g.D = Yw;
        g.ldd = m;
        g.err_flag = err_flag;
        MX_TRY(tc_gemm_run(g, ws, s));
        win_c0 = col0;
        win_w = w;
        next_w = std::min<int64_t>(2 * w, win_cap);
    }
    MX_TRY((copy_matrix<float, float>(Yw + (col0 - win_c0) * m, m, Y, ldy, m, f, false, s)));
    return EOD_OK;
}

eod_status MixedOps<float>::project(const float *Q, int64_t r, float *Ct, cudaStream_t s) {
    if (tf32) {
        float *Qh, *Ql;
        MX_ST(ar->get(&Qh, (size_t)ldm8 * r));
        MX_ST(ar->get(&Ql, (size_t)ldm8 * r));
        MX_TRY(split_tf32(Q, m, r, m, Qh, Ql, ldm8, s));
        TcGemmDesc g;
        g.M = n;
        g.N = r;
        g.K = m;
        g.tf32 = true;
        g.npairs = 3;
        const TcOperand ah{Th, m, n, ldm8}, al{Tl, m, n, ldm8};
        const TcOperand qh{Qh, m, r, ldm8}, ql{Ql, m, r, ldm8};
        g.a[0] = ah; g.b[0] = qh;
        g.a[1] = ah; g.b[1] = ql;
        g.a[2] = al; g.b[2] = qh;
        g.D = Ct;
        g.ldd = n;
        g.err_flag = err_flag;
        MX_TRY(tc_gemm_run(g, ws, s));
        return EOD_OK;
    }
    __nv_bfloat16 *Qh, *Ql;
    MX_ST(ar->get(&Qh, (size_t)ldm8 * r));
    MX_ST(ar->get(&Ql, (size_t)ldm8 * r));
    MX_TRY(split_norm(Q, m, r, m, Qh, Ql, ldm8, nullptr, nullptr, stream_blocks(m * r), s));
    TcGemmDesc g;
    g.M = n;
    g.N = r;
    g.K = m;
    g.a_mn_major = false;
    g.npairs = 3;
    const TcOperand ah{Ahi, m, n, ldm8}, al{Alo, m, n, ldm8};
    const TcOperand qh{Qh, m, r, ldm8}, ql{Ql, m, r, ldm8};
    g.a[0] = ah; g.b[0] = qh;
    g.a[1] = ah; g.b[1] = ql;
    g.a[2] = al; g.b[2] = qh;
    g.D = Ct;
    g.ldd = n;
    g.err_flag = err_flag;
    MX_TRY(tc_gemm_run(g, ws, s));
    return EOD_OK;
}

eod_status MixedOps<float>::recon_error(const float *Q, int64_t r, const float *Ct, const double *d_norm,
                                        double *d_err, cudaStream_t s, cudaStream_t run) {
    const int64_t r8 = round_up(r, 8);
    void *Qth, *Qtl, *Chh, *Chl;
    const size_t es = tf32 ? sizeof(float) : sizeof(__nv_bfloat16);
    MX_ST(ar->get((char **)&Qth, es * (size_t)r8 * m));
    MX_ST(ar->get((char **)&Qtl, es * (size_t)r8 * m));
    MX_ST(ar->get((char **)&Chh, es * (size_t)r8 * n));
    MX_ST(ar->get((char **)&Chl, es * (size_t)r8 * n));
    const int64_t nct = tc_gemm_err_ctas(m, n, 256);
    double *part;
    MX_ST(ar->get(&part, (size_t)nct));
    // the buffers come from `s`'s stream-ordered pool: `run` starts after them
    if (run != s) {
        cudaEvent_t ev = nullptr;
        MX_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(run, ev, 0);
        cudaEventDestroy(ev);
        MX_TRY(e);
        s = run;
    }
    if (tf32) {
        MX_TRY(split_transpose_tf32(Q, m, r, m, (float *)Qth, (float *)Qtl, r8, s));    // (r x m)
        MX_TRY(split_transpose_tf32(Ct, n, r, n, (float *)Chh, (float *)Chl, r8, s));   // C = (C^T)^T, r x n
    } else {
        MX_TRY(split_transpose(Q, m, r, m, (__nv_bfloat16 *)Qth, (__nv_bfloat16 *)Qtl, r8, s));
        MX_TRY(split_transpose(Ct, n, r, n, (__nv_bfloat16 *)Chh, (__nv_bfloat16 *)Chl, r8, s));
    }
    TcGemmDesc g;
    g.tf32 = tf32;
    g.M = m;
    g.N = n;
    g.K = r;
    g.a_mn_major = false;
    g.npairs = 3;
    const TcOperand qh{Qth, r, m, r8}, ql{Qtl, r, m, r8}, ch{Chh, r, n, r8}, cl{Chl, r, n, r8};
    g.a[0] = qh; g.b[0] = ch;
    g.a[1] = qh; g.b[1] = cl;
    g.a[2] = ql; g.b[2] = ch;
    g.epilogue = EPI_ERR;
    g.bn = 256;
    g.ref = A;
    g.ldref = lda;
    g.err_partials = part;
    g.err_flag = err_flag;
    MX_TRY(tc_gemm_run(g, ws, s));
    MX_TRY(finalize_sqrt_sum(part, nct, d_norm, d_err, s));
    return EOD_OK;
}

eod_status MixedOps<float>::check(cudaStream_t s) {
    if (!err_flag) return EOD_OK;
    int h = 0;
    MX_TRY(cudaMemcpyAsync(&h, err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    return h ? EOD_ETIMEOUT : EOD_OK;
}

}  // namespace eod

namespace eod {
namespace {
// One CTA waits on an mbarrier of one expected arrival, with the same bounded
// wait the tcgen05 kernels use; the arrival is made only when `arrive` is
// set.  No copy or MMA is in flight, so a wait that runs out leaves nothing
// behind: the kernel records the time-out in *flag and returns.
__global__ void bounded_wait_kernel(long long budget, int arrive, int *flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && arrive) tc::mbar_arrive(&bar);
    const bool ok = tc::mbar_wait(&bar, 0, budget);
    if (!__all_sync(0xffffffffu, ok ? 1 : 0) && threadIdx.x == 0) atomicExch(flag, 1);
}
}  // namespace
}  // namespace eod

// Test hook of the bounded waits (EOD_ETIMEOUT path).
extern "C" eod_status eod_abe_debug_bounded_wait(int64_t budget_cycles, int32_t arrive, void *stream) {
    using namespace eod;
    if (budget_cycles < 1 || budget_cycles > tc::kWaitBudget) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Arena ar(s);
    int *flag;
    MX_ST(ar.get(&flag, 1));
    MX_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    count_launch(1);
    bounded_wait_kernel<<<1, 32, 0, s>>>((long long)budget_cycles, arrive ? 1 : 0, flag);
    MX_TRY(cudaGetLastError());
    int h = 0;
    MX_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    return h ? EOD_ETIMEOUT : EOD_OK;
}

// ---------------------------------------------------------------------------
// Test hook: one tensor-core contraction in each of the three forms.
// ---------------------------------------------------------------------------
extern "C" eod_status eod_abe_debug_tc_gemm(int32_t form, int64_t M, int64_t N, int64_t K, const float *X,
                                            int64_t ldx, const float *Y, int64_t ldy, float *D, int64_t ldd,
                                            double *err_out, void *stream) {
    using namespace eod;
    if (M < 1 || N < 1 || K < 1 || !X || !Y) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Arena ar(s);
    Scratch ws;
    MX_ST(ar.get((char **)&ws.base, (size_t)64 << 20));
    ws.size = (size_t)64 << 20;
    int *flag;
    MX_ST(ar.get(&flag, 1));
    MX_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    TcGemmDesc g;
    g.err_flag = flag;
    if (form & 8) {
        // the TF32 form of forms 0-2 (X and Y split into two TF32 terms)
        const int f = form & ~8;
        const int64_t lk = round_up(K, 8);
        float *xh, *xl, *yh, *yl;
        MX_ST(ar.get(&xh, (size_t)lk * M));
        MX_ST(ar.get(&xl, (size_t)lk * M));
        MX_ST(ar.get(&yh, (size_t)lk * N));
        MX_ST(ar.get(&yl, (size_t)lk * N));
        g.M = M; g.N = N; g.K = K;
        g.tf32 = true;
        if (f == 0) {
            if (!D || ldx < M || ldy < K || ldd < M) return EOD_EINVAL;
            MX_TRY(split_transpose_tf32(X, M, K, ldx, xh, xl, lk, s));
            MX_TRY(split_tf32(Y, K, N, ldy, yh, yl, lk, s));
            g.npairs = 2;   // Y holds TF32-exact values: its low term is zero
            g.a[0] = {xh, K, M, lk}; g.b[0] = {yh, K, N, lk};
            g.a[1] = {xl, K, M, lk}; g.b[1] = {yh, K, N, lk};
            g.D = D;
            g.ldd = ldd;
        } else if (f == 1 || f == 2) {
            if (f == 1 && (!D || ldx < K || ldy < K || ldd < M)) return EOD_EINVAL;
            if (f == 2 && (!D || !err_out || ldx < M || ldy < N || ldd < M)) return EOD_EINVAL;
            if (f == 1) {
                MX_TRY(split_tf32(X, K, M, ldx, xh, xl, lk, s));
                MX_TRY(split_tf32(Y, K, N, ldy, yh, yl, lk, s));
            } else {
                MX_TRY(split_transpose_tf32(X, M, K, ldx, xh, xl, lk, s));
                MX_TRY(split_transpose_tf32(Y, N, K, ldy, yh, yl, lk, s));
            }
            g.npairs = 3;
            const TcOperand a_h{xh, K, M, lk}, a_l{xl, K, M, lk}, b_h{yh, K, N, lk}, b_l{yl, K, N, lk};
            g.a[0] = a_h; g.b[0] = b_h;
            g.a[1] = a_h; g.b[1] = b_l;
            g.a[2] = a_l; g.b[2] = b_h;
            if (f == 1) {
                g.D = D;
                g.ldd = ldd;
            } else {
                g.epilogue = EPI_ERR;
                g.bn = 256;
                g.ref = D;
                g.ldref = ldd;
                const int64_t nct = tc_gemm_err_ctas(M, N, g.bn);
                double *part;
                MX_ST(ar.get(&part, (size_t)nct));
                g.err_partials = part;
                MX_TRY(tc_gemm_run(g, &ws, s));
                MX_TRY(finalize_sqrt_sum(part, nct, nullptr, err_out, s));
                int h = 0;
                MX_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
                MX_TRY(cudaStreamSynchronize(s));
                return h ? EOD_ETIMEOUT : EOD_OK;
            }
        } else {
            return EOD_EINVAL;
        }
    } else if (form == 0) {
        // D (M x N) = split(X) * bf16(Y): X is M x K (ld ldx), Y is K x N with BF16-exact values
        if (!D || ldx < M || ldy < K || ldd < M) return EOD_EINVAL;
        const int64_t lm = round_up(M, 8), lk = round_up(K, 8);
        __nv_bfloat16 *xh, *xl, *x3, *yh, *yl;
        MX_ST(ar.get(&xh, (size_t)lm * K));
        MX_ST(ar.get(&xl, (size_t)lm * K));
        MX_ST(ar.get(&x3, (size_t)lm * K));
        MX_ST(ar.get(&yh, (size_t)lk * N));
        MX_ST(ar.get(&yl, (size_t)lk * N));
        MX_TRY(split_norm(X, M, K, ldx, xh, xl, lm, nullptr, nullptr, 1024, s, x3));
        MX_TRY(split_norm(Y, K, N, ldy, yh, yl, lk, nullptr, nullptr, 1024, s));
        g.M = M; g.N = N; g.K = K;
        g.a_mn_major = true;
        g.npairs = 3;
        g.a[0] = {xh, M, K, lm};
        g.a[1] = {xl, M, K, lm};
        g.a[2] = {x3, M, K, lm};
        g.b[0] = {yh, K, N, lk};
        g.b[1] = g.b[0];
        g.b[2] = g.b[0];
        g.D = D;
        g.ldd = ldd;
    } else if (form == 1) {
        // D (M x N) = split(X)^T split(Y): X is K x M (ld ldx), Y is K x N (ld ldy)
        if (!D || ldx < K || ldy < K || ldd < M) return EOD_EINVAL;
        const int64_t lk = round_up(K, 8);
        __nv_bfloat16 *xh, *xl, *yh, *yl;
        MX_ST(ar.get(&xh, (size_t)lk * M));
        MX_ST(ar.get(&xl, (size_t)lk * M));
        MX_ST(ar.get(&yh, (size_t)lk * N));
        MX_ST(ar.get(&yl, (size_t)lk * N));
        MX_TRY(split_norm(X, K, M, ldx, xh, xl, lk, nullptr, nullptr, 1024, s));
        MX_TRY(split_norm(Y, K, N, ldy, yh, yl, lk, nullptr, nullptr, 1024, s));
        g.M = M; g.N = N; g.K = K;
        g.npairs = 3;
        const TcOperand a_h{xh, K, M, lk}, a_l{xl, K, M, lk}, b_h{yh, K, N, lk}, b_l{yl, K, N, lk};
        g.a[0] = a_h; g.b[0] = b_h;
        g.a[1] = a_h; g.b[1] = b_l;
        g.a[2] = a_l; g.b[2] = b_h;
        g.D = D;
        g.ldd = ldd;
    } else if (form == 2) {
        // *err_out = sum (D - X Y^T)^2: X is M x K (ld ldx), Y is N x K (ld ldy), D the reference (M x N, ldd)
        if (!D || !err_out || ldx < M || ldy < N || ldd < M) return EOD_EINVAL;
        const int64_t lk = round_up(K, 8);
        __nv_bfloat16 *xh, *xl, *yh, *yl;
        MX_ST(ar.get(&xh, (size_t)lk * M));
        MX_ST(ar.get(&xl, (size_t)lk * M));
        MX_ST(ar.get(&yh, (size_t)lk * N));
        MX_ST(ar.get(&yl, (size_t)lk * N));
        MX_TRY(split_transpose(X, M, K, ldx, xh, xl, lk, s));
        MX_TRY(split_transpose(Y, N, K, ldy, yh, yl, lk, s));
        g.M = M; g.N = N; g.K = K;
        g.npairs = 3;
        const TcOperand a_h{xh, K, M, lk}, a_l{xl, K, M, lk}, b_h{yh, K, N, lk}, b_l{yl, K, N, lk};
        g.a[0] = a_h; g.b[0] = b_h;
        g.a[1] = a_h; g.b[1] = b_l;
        g.a[2] = a_l; g.b[2] = b_h;
        g.epilogue = EPI_ERR;
        g.bn = 256;
        g.ref = D;
        g.ldref = ldd;
        const int64_t nct = tc_gemm_err_ctas(M, N, g.bn);
        double *part;
        MX_ST(ar.get(&part, (size_t)nct));
        g.err_partials = part;
        MX_TRY(tc_gemm_run(g, &ws, s));
        MX_TRY(finalize_sqrt_sum(part, nct, nullptr, err_out, s));
        int h = 0;
        MX_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        MX_TRY(cudaStreamSynchronize(s));
        return h ? EOD_ETIMEOUT : EOD_OK;
    } else {
        return EOD_EINVAL;
    }
    MX_TRY(tc_gemm_run(g, &ws, s));
    int h = 0;
    MX_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MX_TRY(cudaStreamSynchronize(s));
    return h ? EOD_ETIMEOUT : EOD_OK;
}

// Host orchestration of power-free EOD-ABE on one GPU and the exported C ABI
// (include/eod_abe.h).
//
//   Alg. 1 (BasisExt)      omega_fill -> gemm (Y = A Omega_j)
//                          -> 2 x [gemm (S = Q^T Y), gemm (Y -= Q S)]
//                          -> gemm (G = Y^T Y) -> chol_small (pivots + rank test)
//                          -> gemm (P1 = Y R1^{-1}) -> gemm (G2) -> chol_small
//                          -> gemm (P = P1 R2^{-1}) appended to Q
//                          undecided pivots: explicit CGS2 residual of that column
//   Alg. 2 steps 8-11      gemm (C^T = A^T Q), [gemm with fused error: Q C vs A],
//                          CholQR2 (C^T = V R), CholQR2 (R^T = Qh D), gemm (U = Q Qh)
//
// The kernels live in oz_gemm.cu (FP64 products emulated on tcgen05),
// gemm_simt.cu, gram.cu, stream_kernels.cu and chol.cu (plain paths) and
// tc_gemm.cu / mixed.cu (the BF16 and TF32 mixed paths); tau >= 1 adds Alg. 2
// steps 2-7 (subspace iteration) between the two algorithms.  The rank test
// reads a pivot decision back to the host once per sub-panel; everything else
// stays on the device.
#include "common.cuh"
#include "tc_gemm.cuh"
#include "instrument.cuh"
#include "batch.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <thread>
#include <vector>

namespace eod {

int g_fail_alloc_after = 0;

#define EOD_TRY(...)                                    \
    do {                                                 \
        eod_status eod_st_ = (__VA_ARGS__);                     \
        if (eod_st_ != EOD_OK) return eod_st_;           \
    } while (0)
#define EOD_CU(...)                                     \
    do {                                                 \
        cudaError_t eod_ce_ = (__VA_ARGS__);                    \
        if (eod_ce_ != cudaSuccess) {                    \
            return cuda_status(eod_ce_);                 \
        }                                                \
    } while (0)

static eod_status cuda_status(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? EOD_ENOMEM : EOD_ECUDA;
}

// Pinned host mirror of the small device results read once per decision.
struct HostMirror {
    int *info = nullptr;      // [2]
    double *val = nullptr;    // [4]
    int *flag = nullptr;      // [1]
    eod_status init() {
        void *p = nullptr;
        if (cudaMallocHost(&p, 64) != cudaSuccess) { cudaGetLastError(); return EOD_ENOMEM; }
        info = (int *)p;
        flag = info + 2;
        val = (double *)((char *)p + 16);
        return EOD_OK;
    }
    ~HostMirror() { if (info) cudaFreeHost(info); }
};

inline int64_t round_up8(int64_t x) { return (x + 7) / 8 * 8; }

// largest tau (subspace iterations of Alg. 2) accepted
constexpr int kMaxPowerIters = 16;

// Second CholQR pass on a near-identity Gram I + E: the first-order factor
// I + Phi(E) is exact to O(||E||^2) and replaces the factorisation (see
// chol_small) when that is at or below the data's rounding: ||E||_F <= 1e-8
// for FP64 data (O(E^2) <= 1e-16), ||E||_F <= 2e-4 for FP32 data (O(E^2) <=
// 4e-8, the FP32 unit roundoff being 6e-8).
template <typename T> constexpr double near_id_tau2() { return std::is_same<T, double>::value ? 1e-16 : 4e-8; }

// smallest eps / ||A||_F the FP32-data paths accept (see factor_impl)
constexpr double kMixedFloor = 1e-5;
constexpr double kF32Floor = kPF32Floor;   // the persistent batched launch applies the same

template <typename T> struct Traits;
template <> struct Traits<double> { static constexpr int dtype = EOD_F64; static constexpr double rho = 1e-10; };
template <> struct Traits<float> { static constexpr int dtype = EOD_F32; static constexpr double rho = 1e-6; };

// ---------------------------------------------------------------------------
// Blocked CholQR pass on W (rows x p, FP64 Gram, FP64 R):  G = W^T W,
// R = chol(G + shift I), W <- W R^{-1}.
// The Cholesky runs right-looking over panels of kPB columns: each diagonal
// panel is factored left-looking over 64-column leaves (one CTA each, the
// leaf inverses kept), its triangular inverse formed, then the panel row of R
// and the trailing Gram update are two large products.  The solve
// W <- W R^{-1} runs over the same panels (diagonal inverse, then the
// trailing columns of W), so every large product is a plain GEMM.
// Returns EOD_EPRECISION (without touching W) if a pivot is not positive.
// ---------------------------------------------------------------------------
template <typename T>
struct CoreWork {
    double *G = nullptr, *R = nullptr, *Rp = nullptr, *RiD = nullptr, *RiT = nullptr,
           *trace = nullptr, *part = nullptr;
    T *InvT = nullptr, *Tmp = nullptr;
    int *info = nullptr;
    int64_t pcap = 0, rows_cap = 0;
    int nb = 64;       // leaf width of the current Cholesky (divides kPB)
    bool tc = false;   // mixed forms: the solves' products on the tensor cores
};

// rows from which the mixed forms form U = Q Qh on the tensor cores
static constexpr int64_t kTfMinRows = 1024;
static constexpr int kNBMin = 16;   // narrowest leaf (sizes the leaves' status array)
static constexpr int kPB = 256;     // panel width of the core Cholesky and triangular solve

// Leaf width for the Cholesky of a p x p Gram: the tuned value (key
// core_leaf, a = p), else 64.  A narrower leaf spends less time per pivot
// (its in-CTA trailing update competes less with the pivot chain for the
// SM's FP64 unit) at the price of more small panel products between leaves.
static int core_leaf_width(int64_t p) {
    int64_t v = 0;
    if (tuned_value("core_leaf", p, 0, 0, &v) && (v == 16 || v == 32 || v == 64 || v == 128)) return (int)v;
    return 64;
}

template <typename T>
static eod_status chol_panel_leaves(CoreWork<T> &w, int64_t p, int64_t j0, int64_t pe, double shift, Scratch *ws,
                                    cudaStream_t s, double *Rout, double *RiJ) {
    GemmExtra ex;
    for (int64_t l0 = j0; l0 < pe; l0 += w.nb) {
        const int64_t lb = std::min<int64_t>(w.nb, pe - l0), L = l0 / w.nb;
        double *RiL = RiJ + (l0 - j0) * (1 + kPB);   // the leaf's inverse, on the diagonal of R_JJ^{-1}
        if (l0 > j0)   // G(l, l:pe) -= R(j0:l0, l)^T R(j0:l0, l:pe)
            EOD_CU((gemm<double, double, double, double>(true, false, lb, pe - l0, l0 - j0, -1.0, Rout + j0 + l0 * p,
                                                          p, Rout + j0 + l0 * p, p, 1.0, w.G + l0 + l0 * p, p, ex,
                                                          ws, s)));
        EOD_CU(chol_small(w.G + l0 + l0 * p, p, (int)lb, 0, 0.0, 0.0, 0.0, shift, Rout + l0 + l0 * p, p, RiL, kPB,
                          w.info + 2 * L, s));
        if (l0 + lb < pe)   // R(l, l+1:pe) = R_ll^{-T} G(l, l+1:pe)
            EOD_CU((gemm<double, double, double, double>(true, false, lb, pe - l0 - lb, lb, 1.0, RiL, kPB,
                                                          w.G + l0 + (l0 + lb) * p, p, 0.0, Rout + l0 + (l0 + lb) * p,
                                                          p, ex, ws, s)));
    }
    return EOD_OK;
}

// RiJ (jb x jb, ld kPB) = R_JJ^{-1} for the diagonal panel at j0, from its
// leaves' inverses (already on its diagonal) by doubling:
// inv([A B; 0 C]) = [A^-1, -A^-1 B C^-1; 0, C^-1].
template <typename T>
static eod_status panel_inverse(CoreWork<T> &w, int64_t p, int64_t j0, int64_t jb, const double *Rout, double *RiJ,
                                Scratch *ws, cudaStream_t s) {
    GemmExtra au, bu;
    au.a_upper = true;
    bu.b_upper = true;
    for (int64_t h = w.nb; h < jb; h *= 2) {
        for (int64_t a0 = 0; a0 + h < jb; a0 += 2 * h) {
            const int64_t b0 = a0 + h, bl = std::min<int64_t>(h, jb - b0);
            // T = A^-1 B;  RiJ(a, b) = -T C^-1
            EOD_CU((gemm<double, double, double, double>(false, false, h, bl, h, 1.0, RiJ + a0 + a0 * kPB, kPB,
                                                          Rout + (j0 + a0) + (j0 + b0) * p, p, 0.0, w.RiT, h, au,
                                                          ws, s)));
            EOD_CU((gemm<double, double, double, double>(false, false, h, bl, bl, -1.0, w.RiT, h,
                                                          RiJ + b0 + b0 * kPB, kPB, 0.0, RiJ + a0 + b0 * kPB, kPB, bu,
                                                          ws, s)));
        }
    }
    return EOD_OK;
}

template <typename T>
static eod_status chol_panels(CoreWork<T> &w, int64_t p, double shift, HostMirror &hm, Scratch *ws,
                              cudaStream_t s, double *Rout) {
    GemmExtra ex, sym;
    sym.upper_only = true;
    EOD_CU(fill_zero<double>(Rout, p, p, p, s));
    for (int64_t j0 = 0; j0 < p; j0 += kPB) {
        const int64_t pe = std::min<int64_t>(p, j0 + kPB), jb = pe - j0;
        double *RiJ = w.RiD + (j0 / kPB) * kPB * kPB;   // ld kPB
        EOD_CU(fill_zero<double>(RiJ, jb, jb, kPB, s));
        EOD_TRY(chol_panel_leaves(w, p, j0, pe, shift, ws, s, Rout, RiJ));
        EOD_TRY(panel_inverse(w, p, j0, jb, Rout, RiJ, ws, s));
        if (pe < p) {
            // R(J, pe:p) = R_JJ^{-T} G(J, pe:p);  G(pe:p, pe:p) -= R(J, pe:p)^T R(J, pe:p)
            EOD_CU((gemm<double, double, double, double>(true, false, jb, p - pe, jb, 1.0, RiJ, kPB,
                                                          w.G + j0 + pe * p, p, 0.0, Rout + j0 + pe * p, p, ex, ws,
                                                          s)));
            EOD_CU((gemm<double, double, double, double>(true, false, p - pe, p - pe, jb, -1.0, Rout + j0 + pe * p,
                                                          p, Rout + j0 + pe * p, p, 1.0, w.G + pe + pe * p, p, sym,
                                                          ws, s)));
        }
    }
    const int64_t nblk = (p + w.nb - 1) / w.nb;
    std::vector<int> infos(2 * nblk);
    EOD_CU(cudaMemcpyAsync(infos.data(), w.info, sizeof(int) * 2 * nblk, cudaMemcpyDeviceToHost, s));
    EOD_CU(cudaStreamSynchronize(s));
    for (int64_t J = 0; J < nblk; ++J) {
        const int64_t jb = std::min<int64_t>(w.nb, p - J * w.nb);
        if (infos[2 * J] != jb || infos[2 * J + 1] != CHOL_ALL) return EOD_EPRECISION;
    }
    return EOD_OK;
}

// W <- W R^{-1} on the tensor cores (the mixed forms, FP32 data): per panel
// J, X_J = W_J R_JJ^{-1} written over W_J, then W(:, pe:p) -= X_J R(J, pe:p),
// each as three TF32 products of split operands (X = X_hi + X_lo: about
// 2^-21 relative, the accuracy of an FP32 product).  TF32 operands are
// K-major, so W_J and X_J are split transposed; the FP64 blocks of R and of
// R_JJ^{-1} (zero below the diagonal) are rounded to FP32 and split.
// EOD_EUNSUPPORTED, with nothing launched, when the scratch has no room.
static eod_status trsm_panels_tc(const double *RiD, float *W, int64_t rows, int64_t ldw, int64_t p,
                                 const double *R, Scratch *ws, cudaStream_t s) {
    const int64_t pb = round_up(std::min<int64_t>(p, kPB), 4);   // ld of the split blocks
    const size_t mark = ws->mark();
    float *wth = (float *)ws->take(sizeof(float) * (size_t)(pb * rows));
    float *wtl = (float *)ws->take(sizeof(float) * (size_t)(pb * rows));
    float *bh = (float *)ws->take(sizeof(float) * (size_t)(pb * p));
    float *bl = (float *)ws->take(sizeof(float) * (size_t)(pb * p));
    if (!wth || !wtl || !bh || !bl) {
        ws->release(mark);
        return EOD_EUNSUPPORTED;
    }
    // W(:, c0 : c0+N) = alpha (W_J or X_J, split in wth/wtl) (the split block in bh/bl) + beta W(:, c0 : c0+N)
    auto product = [&](int64_t N, int64_t K, float *D, float alpha, float beta) -> cudaError_t {
        TcGemmDesc g;
        g.M = rows;
        g.N = N;
        g.K = K;
        g.tf32 = true;
        g.npairs = 3;
        const TcOperand ah{wth, K, rows, pb}, al{wtl, K, rows, pb}, b_h{bh, K, N, pb}, b_l{bl, K, N, pb};
        g.a[0] = ah, g.b[0] = b_h;
        g.a[1] = ah, g.b[1] = b_l;
        g.a[2] = al, g.b[2] = b_h;
        g.D = D;
        g.ldd = ldw;
        g.alpha = alpha;
        g.beta = beta;
        g.err_flag = ws->err_flag;
        return tc_gemm_run(g, ws, s);
    };
    for (int64_t j0 = 0; j0 < p; j0 += kPB) {
        const int64_t pe = std::min<int64_t>(p, j0 + kPB), jb = pe - j0;
        const double *RiJ = RiD + (j0 / kPB) * kPB * kPB;
        EOD_CU(split_transpose_tf32(W + j0 * ldw, rows, jb, ldw, wth, wtl, pb, s));
        EOD_CU(split_tf32_f64(RiJ, jb, jb, kPB, bh, bl, pb, s));
        EOD_CU(product(jb, jb, W + j0 * ldw, 1.f, 0.f));   // X_J over W_J (read from its split copy)
        if (pe < p) {
            EOD_CU(split_transpose_tf32(W + j0 * ldw, rows, jb, ldw, wth, wtl, pb, s));
            EOD_CU(split_tf32_f64(R + j0 + pe * p, jb, p - pe, p, bh, bl, pb, s));
            EOD_CU(product(p - pe, jb, W + pe * ldw, -1.f, 1.f));
        }
    }
    ws->release(mark);
    return EOD_OK;
}

// W <- W R^{-1}, R upper p x p (ld p) with the diagonal panels' inverses in w.RiD.
// With allow_tc, the mixed forms' products run on the tensor cores.
template <typename T>
static eod_status trsm_panels(CoreWork<T> &w, T *W, int64_t rows, int64_t ldw, int64_t p, const double *R,
                              Scratch *ws, cudaStream_t s, bool allow_tc) {
    if (allow_tc && w.tc && std::is_same<T, float>::value && rows >= kTfMinRows && p >= 128) {
        const eod_status st = trsm_panels_tc(w.RiD, (float *)W, rows, ldw, p, R, ws, s);
        if (st != EOD_EUNSUPPORTED) return st;
    }
    GemmExtra ex, exb;
    exb.b_upper = true;
    for (int64_t j0 = 0; j0 < p; j0 += kPB) {
        const int64_t pe = std::min<int64_t>(p, j0 + kPB), jb = pe - j0;
        const double *RiJ = w.RiD + (j0 / kPB) * kPB * kPB;
        const T *Ri = (const T *)RiJ;
        if (!std::is_same<T, double>::value) {
            EOD_CU((copy_matrix<double, T>(RiJ, kPB, w.InvT, kPB, jb, jb, false, s)));
            Ri = w.InvT;
        }
        // X_J = W_J R_JJ^{-1}
        EOD_CU((gemm<T, T, T, T>(false, false, rows, jb, jb, 1.0, W + j0 * ldw, ldw, Ri, kPB, 0.0, w.Tmp, rows, exb,
                                 ws, s)));
        EOD_CU((copy_matrix<T, T>(w.Tmp, rows, W + j0 * ldw, ldw, rows, jb, false, s)));
        if (pe < p) {
            // W(:, pe:p) -= X_J R(J, pe:p)
            const T *Rb = (const T *)(R + j0 + pe * p);
            int64_t ldb = p;
            if (!std::is_same<T, double>::value) {
                EOD_CU((copy_matrix<double, T>(R + j0 + pe * p, p, w.InvT, jb, jb, p - pe, false, s)));
                Rb = w.InvT;
                ldb = jb;
            }
            EOD_CU((gemm<T, T, T, T>(false, false, rows, p - pe, jb, -1.0, W + j0 * ldw, ldw, Rb, ldb, 1.0,
                                     W + pe * ldw, ldw, ex, ws, s)));
        }
    }
    return EOD_OK;
}

// G (p x p, upper, FP64) = W^T W: the skinny kernel for p <= 128, else the
// FP64 GEMM (tensor-core emulation for large products; FP32 data is widened
// to FP64 first, exactly), else for FP32 data the exact-product FP32 sums.
template <typename T>
static eod_status gram_full(const T *W, int64_t rows, int64_t p, int64_t ldw, double *G, const GemmExtra &sym,
                            Scratch *ws, cudaStream_t s) {
    if (p <= 128) {
        EOD_CU(gram_skinny<T>(W, rows, (int)p, ldw, G, p, ws, s));
    } else if (std::is_same<T, double>::value) {
        EOD_CU((gemm<T, T, double, double>(true, false, p, p, rows, 1.0, W, ldw, W, ldw, 0.0, G, p, sym, ws, s)));
    } else if (fp64_use_emulated(p, p, rows)) {
        double *Wd = nullptr;
        EOD_CU(lib_malloc_async((void **)&Wd, sizeof(double) * (size_t)rows * p, s));
        cudaError_t e = copy_matrix<T, double>(W, ldw, Wd, rows, rows, p, false, s);
        if (e == cudaSuccess)
            e = gemm<double, double, double, double>(true, false, p, p, rows, 1.0, Wd, rows, Wd, rows, 0.0, G, p, sym,
                                                     ws, s);
        cudaFreeAsync(Wd, s);
        EOD_CU(e);
    } else {
        EOD_CU(gram_tiled_f32((const float *)W, rows, p, ldw, G, p, ws, s));
    }
    return EOD_OK;
}

// CholQR2 (shifted CholQR3 when the first Cholesky breaks down; Fukaya,
// Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SISC 2020): W (rows x p) is
// replaced by its orthonormal factor and Rout (p x p, ld p) by R with
// W_in = W_out R, diag(R) > 0.
template <typename T>
static eod_status cholqr2(CoreWork<T> &w, T *W, int64_t rows, int64_t ldw, int64_t p, double *Rout,
                          HostMirror &hm, Scratch *ws, cudaStream_t s) {
    GemmExtra sym;
    sym.upper_only = true;
    double *Racc = w.R;  // running product
    w.nb = core_leaf_width(p);
    int passes = 2;
    double shift = 0.0;
    for (int pass = 0; pass < passes; ++pass) {
        EOD_TRY(gram_full(W, rows, p, ldw, w.G, sym, ws, s));
        double *Rpass = (pass == 0) ? Rout : w.Rp;  // pass factor storage
        eod_status st = EOD_OK;
        bool near_id = false;
        if (pass > 0 && shift == 0.0) {
            EOD_CU(offidentity_sumsq(w.G, p, p, w.part, w.trace, s));
            EOD_CU(cudaMemcpyAsync(hm.val, w.trace, sizeof(double), cudaMemcpyDeviceToHost, s));
            EOD_CU(cudaStreamSynchronize(s));
            near_id = hm.val[0] <= near_id_tau2<T>();
        }
        if (near_id) EOD_CU(near_identity_factor(w.G, p, p, Rpass, p, w.RiD, kPB, s));
        else st = chol_panels(w, p, shift, hm, ws, s, Rpass);
        if (st == EOD_EPRECISION && pass == 0 && shift == 0.0) {
            // shifted CholQR: shift = 11 (rows p + p (p+1)) u ||W||_2^2, ||W||_2^2 <= trace(G)
            EOD_CU(trace_sum(w.G, p, p, w.trace, s));
            EOD_CU(cudaMemcpyAsync(hm.val, w.trace, sizeof(double), cudaMemcpyDeviceToHost, s));
            EOD_CU(cudaStreamSynchronize(s));
            const double u = std::is_same<T, float>::value ? kU32 : kU64;
            shift = 11.0 * ((double)rows * p + (double)p * (p + 1)) * u * hm.val[0];
            passes = 3;
            EOD_TRY(gram_full(W, rows, p, ldw, w.G, sym, ws, s));
            st = chol_panels(w, p, shift, hm, ws, s, Rpass);
        }
        if (st != EOD_OK) return st;
        shift = 0.0;
        // The first pass's solve sets how close the next pass's Gram is to I
        // (its near-identity test is at the FP32 level), so it stays on the
        // FP32 FFMA products; the later passes (R near I) may take the
        // tensor cores' TF32 products (~2^-21 relative).
        EOD_TRY(trsm_panels(w, W, rows, ldw, p, Rpass, ws, s, pass > 0));
        if (pass > 0) {
            // Racc = Rpass * Rout (both upper), then Rout = Racc
            GemmExtra tri;
            tri.a_upper = true;
            tri.b_upper = true;
            EOD_CU((gemm<double, double, double, double>(false, false, p, p, p, 1.0, Rpass, p, Rout, p, 0.0, Racc, p,
                                                          tri, ws, s)));
            EOD_CU((copy_matrix<double, double>(Racc, p, Rout, p, p, p, false, s)));
        }
    }
    return EOD_OK;
}

// A non-blocking stream of the calling thread on the current device, for
// work that overlaps the main stream of a factorisation (created once per
// thread and device, kept for the life of the process).
static cudaStream_t side_stream() {
    thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

// Makes `main` wait for everything queued on `side` so far, when it goes out
// of scope (on every return path): the buffers both streams use are freed on
// `main` afterwards.
struct JoinOnExit {
    cudaStream_t main = nullptr, side = nullptr;
    ~JoinOnExit() { join(); }
    void join() {
        if (!side || side == main) return;
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            if (cudaEventRecord(ev, side) != cudaSuccess || cudaStreamWaitEvent(main, ev, 0) != cudaSuccess)
                cudaStreamSynchronize(side);
            cudaEventDestroy(ev);
        } else {
            cudaStreamSynchronize(side);
        }
        cudaGetLastError();
        side = nullptr;
    }
};

// `to` waits for the work queued on `from` so far.
static cudaError_t stream_after(cudaStream_t to, cudaStream_t from) {
    if (to == from) return cudaSuccess;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    cudaEventDestroy(ev);
    return e;
}

// ---------------------------------------------------------------------------
// The plain path (T = double: FP64 everywhere; T = float: FP32 contractions,
// FP64 Gram / Cholesky / rank test / core R factors).
// ---------------------------------------------------------------------------
struct Result {
    int64_t rank = 0, blocks = 0, restarts = 0;
    double norm_a = 0, eps = 0, rel_err = -1;
    std::vector<double> tdiag;
};

// Slices kept for the plain FP64 path's tensor-core contractions: A in both
// orientations (sliced once), the basis Q in both orientations (extended as
// columns are appended: per-column exponents for Q^T, the fixed exponent 1
// for Q, whose entries are at most 1 in magnitude), and a buffer for the
// small operand of each product.
struct OzCache {
    bool on = false;
    void *Arow = nullptr, *Acol = nullptr, *Qc = nullptr, *Qr = nullptr, *Bt = nullptr;
    int *eArow = nullptr, *eAcol = nullptr, *eQc = nullptr, *eBt = nullptr;
    int64_t m = 0, m8 = 0, n8 = 0, cap8 = 0, bt_elems = 0;
    OzOperand arow() const { return {Arow, eArow, 0, n8, m * n8}; }
};

template <typename T>
static eod_status factor_impl(const T *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                              const eod_opts &o, cudaStream_t s, Arena &ar, eod_factors *F) {
    const int64_t cap = std::min(m, n);
    int64_t k = o.block_k > 0 ? o.block_k : 32;
    if (k > cap) k = cap;
    const bool mixed = (o.precision == EOD_MIXED_BF16 || o.precision == EOD_MIXED_TF32);

    HostMirror hm;
    EOD_TRY(hm.init());

    // ---- workspace ----
    Scratch ws;
    const size_t ws_bytes = (size_t)48 << 20;
    EOD_TRY(ar.get((char **)&ws.base, ws_bytes));
    ws.size = ws_bytes;
    EOD_TRY(ar.get(&ws.err_flag, 1));
    EOD_CU(cudaMemsetAsync(ws.err_flag, 0, sizeof(int), s));
    ws.tile_count_n = kTileCounters;
    EOD_TRY(ar.get(&ws.tile_count, (size_t)kTileCounters));
    EOD_CU(cudaMemsetAsync(ws.tile_count, 0, sizeof(unsigned) * kTileCounters, s));

    T *Qb, *Om, *Y, *S, *T1, *RinvT;
    double *G, *R1, *R1i, *R2, *R2i, *tdiag_d, *dsc;
    int *iflag, *info;
    EOD_TRY(ar.get(&Qb, (size_t)m * cap));
    EOD_TRY(ar.get(&Om, (size_t)n * k));
    EOD_TRY(ar.get(&Y, (size_t)m * k));
    EOD_TRY(ar.get(&S, (size_t)cap * k));
    EOD_TRY(ar.get(&T1, (size_t)m * k));
    EOD_TRY(ar.get(&RinvT, (size_t)k * k));
    EOD_TRY(ar.get(&G, (size_t)k * k));
    EOD_TRY(ar.get(&R1, (size_t)k * k));
    EOD_TRY(ar.get(&R1i, (size_t)k * k));
    EOD_TRY(ar.get(&R2, (size_t)k * k));
    EOD_TRY(ar.get(&R2i, (size_t)k * k));
    EOD_TRY(ar.get(&tdiag_d, (size_t)cap + 1));
    // per accepted panel, the (columns, code) of its second CholQR pass,
    // checked once after the loop (no host round trip per panel)
    int *pinfo;
    EOD_TRY(ar.get(&pinfo, (size_t)2 * (cap + 1)));
    EOD_TRY(ar.get(&dsc, 8));
    EOD_TRY(ar.get(&iflag, 4));
    EOD_TRY(ar.get(&info, 2));
    double *d_norm = dsc, *d_t = dsc + 1, *d_err = dsc + 2;

    // ---- S0: ||A||_F and finiteness ----
    // (the BF16 mixed form takes both from its split pass over A: one read of
    // A for the two)
    MixedOps<T> mx;
    const bool norm_in_split = mixed && o.precision == EOD_MIXED_BF16;
    {
        Phase ph_norm("eod.norm");
        EOD_CU(cudaMemsetAsync(iflag, 0, sizeof(int) * 4, s));
        if (norm_in_split) EOD_TRY(mx.prepare(A, m, n, lda, k, ar, &ws, s, false, d_norm, iflag));
        else EOD_CU(fro_norm<T>(A, m, n, lda, d_norm, iflag, &ws, s));
        EOD_CU(cudaMemcpyAsync(hm.val, d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
        EOD_CU(cudaMemcpyAsync(hm.flag, iflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        EOD_CU(cudaStreamSynchronize(s));
        if (hm.flag[0]) return EOD_ENONFINITE;
    }
    const double norm_a = hm.val[0];
    const double eps = (o.tol_mode == EOD_TOL_REL_FRO) ? tol * norm_a : tol;
    // Below these thresholds the sketch's own rounding (FP32 accumulation,
    // and the BF16 split on the mixed path) reaches the size of |T(l,l)|, so
    // the rank test could not be decided: refuse instead of guessing.
    if (std::is_same<T, float>::value && norm_a > 0.0) {
        const double floor_rel = mixed ? kMixedFloor : kF32Floor;
        if (eps < floor_rel * norm_a) return EOD_EPRECISION;
    }
    F->norm_a = norm_a;
    F->eps = eps;
    F->block_k = k;

    if (mixed && !norm_in_split) EOD_TRY(mx.prepare(A, m, n, lda, k, ar, &ws, s, o.precision == EOD_MIXED_TF32));

    OzCache oz;
    oz.on = std::is_same<T, double>::value && fp64_use_emulated(m, k, n);
    if (oz.on) {
        oz.m = m;
        oz.m8 = round_up8(m);
        oz.n8 = round_up8(n);
        oz.cap8 = round_up8(cap);
        oz.bt_elems = (int64_t)kOzSlices * k * std::max(oz.m8, std::max(oz.n8, oz.cap8));
        EOD_TRY(ar.get((uint16_t **)&oz.Arow, (size_t)kOzSlices * m * oz.n8));
        EOD_TRY(ar.get((uint16_t **)&oz.Acol, (size_t)kOzSlices * n * oz.m8));
        EOD_TRY(ar.get((uint16_t **)&oz.Qc, (size_t)kOzSlices * cap * oz.m8));
        EOD_TRY(ar.get((uint16_t **)&oz.Qr, (size_t)kOzSlices * m * oz.cap8));
        EOD_TRY(ar.get((uint16_t **)&oz.Bt, (size_t)oz.bt_elems));
        EOD_TRY(ar.get(&oz.eArow, (size_t)m));
        EOD_TRY(ar.get(&oz.eAcol, (size_t)n));
        EOD_TRY(ar.get(&oz.eQc, (size_t)cap));
        EOD_TRY(ar.get(&oz.eBt, (size_t)std::max(m, n)));
        const double *Ad = (const double *)A;
        // op(A) = A: rows i, K = n;  op(A) = A^T: rows = columns of A, K = m
        EOD_CU(oz_slice(Ad, m, n, 1, lda, oz.Arow, oz.eArow, 0, oz.n8, m * oz.n8, s));
        EOD_CU(oz_slice(Ad, n, m, lda, 1, oz.Acol, oz.eAcol, 0, oz.m8, n * oz.m8, s));
    }
    // append columns c0 .. c0+cnt-1 of the basis to the sliced copies
    auto oz_append = [&](int64_t c0, int64_t cnt) -> cudaError_t {
        if (!oz.on || cnt <= 0) return cudaSuccess;
        const double *Qd = (const double *)Qb;
        cudaError_t e = oz_slice(Qd + c0 * m, cnt, m, m, 1, (uint16_t *)oz.Qc + c0 * oz.m8, oz.eQc + c0, 0, oz.m8,
                                 cap * oz.m8, s);
        if (e != cudaSuccess) return e;
        return oz_slice(Qd + c0 * m, m, cnt, 1, m, (uint16_t *)oz.Qr + c0, nullptr, 1, oz.cap8, m * oz.cap8, s);
    };
    // slices of a small B operand (rows x K, X(r, k) at X[r*sr + k*sk]) into
    // bt / ebt (oz.Bt on the main stream) on stream st
    auto oz_small_to = [&](const T *X, int64_t rows, int64_t K, int64_t sr, int64_t sk, void *bt, int *ebt,
                           cudaStream_t st, OzOperand &out) -> cudaError_t {
        const int64_t ldk = round_up8(K);
        out = {bt, ebt, 0, ldk, rows * ldk};
        return oz_slice((const double *)X, rows, K, sr, sk, bt, ebt, 0, ldk, rows * ldk, st);
    };
    auto oz_small = [&](const T *X, int64_t rows, int64_t K, int64_t sr, int64_t sk, OzOperand &out) -> cudaError_t {
        return oz_small_to(X, rows, K, sr, sk, oz.Bt, oz.eBt, s, out);
    };

    // ---- Alg. 1 ----
    const double eps2 = eps * eps;
    const double delta_coef = 64.0 * ((double)k + std::sqrt((double)m)) * kU64;
    GemmExtra ex, sym, bup;
    sym.upper_only = true;
    bup.b_upper = true;
    int64_t kept = 0, blocks = 0, restarts = 0;
    std::vector<double> tdiag;
    tdiag.reserve(cap + 1);
    bool stop = (norm_a == 0.0);
    if (stop) tdiag.push_back(0.0);

    // One projection pass Yc <- Yc - Q(:, q0:q1) (Q(:, q0:q1)^T Yc) on stream
    // st with its own workspace and slice buffer (step 4 of Alg. 1).
    auto deflate = [&](T *Yc, int64_t wdt, int64_t q0, int64_t q1, T *Sb, Scratch *w, void *bt, int *ebt,
                       cudaStream_t st) -> cudaError_t {
        const int64_t nq = q1 - q0;
        if (nq <= 0) return cudaSuccess;
        const T *Qq = Qb + q0 * m;
        cudaError_t e;
        if (oz.on && fp64_use_emulated(nq, wdt, m)) {
            OzOperand bo;
            e = oz_small_to(Yc, wdt, m, m, 1, bt, ebt, st, bo);
            if (e != cudaSuccess) return e;
            const OzOperand qc{(const uint16_t *)oz.Qc + q0 * oz.m8, oz.eQc + q0, 0, oz.m8, cap * oz.m8};
            e = oz_gemm_ops(qc, bo, nq, wdt, m, 1.0, 0.0, (double *)Sb, cap, ex, w->err_flag, st);
        } else {
            e = gemm<T, T, T, T>(true, false, nq, wdt, m, 1.0, Qq, m, Yc, m, 0.0, Sb, cap, ex, w, st);
        }
        if (e != cudaSuccess) return e;
        if (oz.on && fp64_use_emulated(m, wdt, nq) && q0 % 8 == 0) {
            OzOperand bo;
            e = oz_small_to(Sb, wdt, nq, cap, 1, bt, ebt, st, bo);
            if (e != cudaSuccess) return e;
            const OzOperand qr{(const uint16_t *)oz.Qr + q0, nullptr, 1, oz.cap8, m * oz.cap8};
            return oz_gemm_ops(qr, bo, m, wdt, nq, -1.0, 1.0, (double *)Yc, m, ex, w->err_flag, st);
        }
        return gemm<T, T, T, T>(false, false, m, wdt, nq, -1.0, Qq, m, Sb, cap, 1.0, Yc, m, ex, w, st);
    };
    // Y_j = A Omega_j for the block of global Omega columns col0 .. col0+f-1
    auto sketch = [&](int64_t col0, int64_t f, T *Yd, T *Omd, Scratch *w, void *bt, int *ebt,
                      cudaStream_t st) -> eod_status {
        if (mixed) {
            Scratch *keep_ws = mx.ws;
            mx.ws = w;
            const eod_status r = mx.sketch(col0, f, seed, o.batch_index, Yd, m, st);
            mx.ws = keep_ws;
            return r;
        }
        EOD_CU(omega_fill<T>(n, col0, f, seed, o.batch_index, Omd, n, st));
        if (oz.on) {
            OzOperand bo;
            EOD_CU(oz_small_to(Omd, f, n, n, 1, bt, ebt, st, bo));
            EOD_CU(oz_gemm_ops(oz.arow(), bo, m, f, n, 1.0, 0.0, (double *)Yd, m, ex, w->err_flag, st));
        } else {
            EOD_CU((gemm<T, T, T, T>(false, false, m, f, n, 1.0, A, lda, Omd, n, 0.0, Yd, m, ex, w, st)));
        }
        return EOD_OK;
    };

    // Lookahead across blocks: while block j's Gram and rank-test leaf run
    // (one CTA), the next block is sketched and given its first projection
    // pass against the basis that existed before block j, on a side stream
    // with its own buffers; block j+1 then only projects out block j's own
    // columns before its second pass (the same BCGS2 result in exact
    // arithmetic: the two groups of columns are orthogonal).
    // (only where the sketch has work enough to hide: for small problems the
    // extra buffers and events cost more than the leaf they overlap;
    // EOD_LOOKAHEAD=0 / 1 turns it off / on regardless of size)
    cudaStream_t s2 = cap > k ? side_stream() : nullptr;
    bool lookahead = s2 != nullptr && s2 != s && (double)m * (double)n >= 4.0e6;
    if (const char *env = std::getenv("EOD_LOOKAHEAD")) lookahead = s2 != nullptr && s2 != s && env[0] == '1';
    T *Y2 = nullptr, *S2 = nullptr, *Om2 = nullptr;
    void *Bt2 = nullptr;
    int *eBt2 = nullptr;
    Scratch ws2;
    JoinOnExit join_la;
    if (lookahead) {
        EOD_TRY(ar.get(&Y2, (size_t)m * k));
        EOD_TRY(ar.get(&S2, (size_t)cap * k));
        EOD_TRY(ar.get(&Om2, (size_t)n * k));
        EOD_TRY(ar.get((char **)&ws2.base, ws_bytes));
        ws2.size = ws_bytes;
        ws2.err_flag = ws.err_flag;
        ws2.tile_count_n = kTileCounters;
        EOD_TRY(ar.get(&ws2.tile_count, (size_t)kTileCounters));
        EOD_CU(cudaMemsetAsync(ws2.tile_count, 0, sizeof(unsigned) * kTileCounters, s));
        if (oz.on) {
            EOD_TRY(ar.get((uint16_t **)&Bt2, (size_t)oz.bt_elems));
            EOD_TRY(ar.get(&eBt2, (size_t)std::max(m, n)));
        }
        join_la.main = s;
        join_la.side = s2;
    }
    int64_t nt = 0;              // T-diagonal entries recorded in tdiag_d
    std::vector<int> panel_p;    // columns of each accepted panel
    bool ahead = false;          // Y2 holds the block at ahead_col0, projected once against Q(:, 0:ahead_q)
    int64_t ahead_col0 = -1, ahead_q = 0;

    while (!stop && kept < cap) {
        const int64_t f = std::min(k, cap - kept);
        ++blocks;
        // steps 3-4: Omega_j and Y = A Omega_j
        Phase ph_block("eod.basis_ext_block");
        const bool from_ahead = ahead && ahead_col0 == kept;
        if (ahead) EOD_CU(stream_after(s, s2));
        if (from_ahead) {
            std::swap(Y, Y2);
        } else {
            EOD_TRY(sketch(kept, f, Y, Om, &ws, oz.on ? oz.Bt : nullptr, oz.on ? oz.eBt : nullptr, s));
        }
        ahead = false;
        const int64_t kept_block = kept;   // the basis this block starts from
        int64_t cur = 0;
        while (!stop && cur < f) {
            T *Yc = Y + cur * m;
            const int64_t wdt = f - cur;
            // step 4: Y <- (I - Q Q^T) Y, twice
            if (cur == 0 && from_ahead) {
                // the first pass's rest: the columns added since the lookahead
                // (from a multiple of 8 for the sliced Q; the overlap is only
                // projected twice), then the second pass
                EOD_CU(deflate(Yc, wdt, ahead_q & ~(int64_t)7, kept, S, &ws, oz.on ? oz.Bt : nullptr,
                               oz.on ? oz.eBt : nullptr, s));
                EOD_CU(deflate(Yc, wdt, 0, kept, S, &ws, oz.on ? oz.Bt : nullptr, oz.on ? oz.eBt : nullptr, s));
            } else {
                for (int pass = 0; pass < 2 && kept > 0; ++pass)
                    EOD_CU(deflate(Yc, wdt, 0, kept, S, &ws, oz.on ? oz.Bt : nullptr, oz.on ? oz.eBt : nullptr, s));
            }
            // the lookahead: Y2 free (its last use, the swap above, is on s)
            // and Q(:, 0:kept_block) final before this point of s
            const bool launch_ahead = lookahead && cur == 0 && kept_block + f < cap;
            cudaEvent_t ev_ready = nullptr;
            if (launch_ahead) {
                EOD_CU(cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming));
                cudaError_t e = cudaEventRecord(ev_ready, s);
                if (e != cudaSuccess) {
                    cudaEventDestroy(ev_ready);
                    EOD_CU(e);
                }
            }
            // step 5 (pass 1) + steps 6-11: Gram, Cholesky with the rank test
            EOD_CU(gram_skinny<T>(Yc, m, (int)wdt, m, G, k, &ws, s));
            EOD_CU(chol_small(G, k, (int)wdt, 1, eps2, delta_coef, Traits<T>::rho, 0.0, R1, k, R1i, k, info, s));
            EOD_CU(cudaMemcpyAsync(hm.info, info, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
            if (launch_ahead) {
                const int64_t c1 = kept_block + f, f1 = std::min(k, cap - c1);
                cudaError_t e = cudaStreamWaitEvent(s2, ev_ready, 0);
                cudaEventDestroy(ev_ready);
                EOD_CU(e);
                EOD_TRY(sketch(c1, f1, Y2, Om2, &ws2, Bt2, eBt2, s2));
                EOD_CU(deflate(Y2, f1, 0, kept_block, S2, &ws2, Bt2, eBt2, s2));
                ahead = true;
                ahead_col0 = c1;
                ahead_q = kept_block;
            }
            EOD_CU(cudaStreamSynchronize(s));
            const int p = hm.info[0], code = hm.info[1];
            if (p > 0) {
                // P1 = Y(:,1:p) R1^{-1}; pass 2: G2 = P1^T P1 = R2^T R2; P = P1 R2^{-1}
                const T *Ri = (const T *)R1i;
                if (!std::is_same<T, double>::value) {
                    EOD_CU((copy_matrix<double, T>(R1i, k, RinvT, k, p, p, false, s)));
                    Ri = RinvT;
                }
                EOD_CU((gemm<T, T, T, T>(false, false, m, p, p, 1.0, Yc, m, Ri, k, 0.0, T1, m, bup, &ws, s)));
                EOD_CU(gram_skinny<T>(T1, m, p, m, G, k, &ws, s));
                int *pinf = pinfo + 2 * (int64_t)panel_p.size();
                EOD_CU(chol_small(G, k, p, 0, 0.0, 0.0, 0.0, 0.0, R2, k, R2i, k, pinf, s, near_id_tau2<T>()));
                const T *Ri2 = (const T *)R2i;
                if (!std::is_same<T, double>::value) {
                    EOD_CU((copy_matrix<double, T>(R2i, k, RinvT, k, p, p, false, s)));
                    Ri2 = RinvT;
                }
                EOD_CU((gemm<T, T, T, T>(false, false, m, p, p, 1.0, T1, m, Ri2, k, 0.0, Qb + kept * m, m, bup, &ws, s)));
                EOD_CU(tdiag_product(R1, R2, k, pinf, tdiag_d + nt, s));
                panel_p.push_back(p);
                nt += p;
                EOD_CU(oz_append(kept, p));
                kept += p;
            }
            if (code == CHOL_ALL) {
                cur = f;
            } else if (code == CHOL_BELOW) {
                // d_p < eps^2 - delta: |T(p,p)| <= eps for certain
                stop = true;
                // record the explicit residual norm of that column (diagnostics only)
                T *z = Yc + (int64_t)p * m;
                for (int pass = 0; pass < 2 && kept > 0; ++pass) {
                    EOD_CU((gemm<T, T, T, T>(true, false, kept, 1, m, 1.0, Qb, m, z, m, 0.0, S, cap, ex, &ws, s)));
                    EOD_CU((gemm<T, T, T, T>(false, false, m, 1, kept, -1.0, Qb, m, S, cap, 1.0, z, m, ex, &ws, s)));
                }
                EOD_CU(fro_norm<T>(z, m, 1, m, tdiag_d + nt, iflag + 1, &ws, s));
                ++nt;
            } else {
                // undecided pivot: settle column p by an explicit CGS2 residual norm
                T *z = Yc + (int64_t)p * m;
                for (int pass = 0; pass < 2 && kept > 0; ++pass) {
                    EOD_CU((gemm<T, T, T, T>(true, false, kept, 1, m, 1.0, Qb, m, z, m, 0.0, S, cap, ex, &ws, s)));
                    EOD_CU((gemm<T, T, T, T>(false, false, m, 1, kept, -1.0, Qb, m, S, cap, 1.0, z, m, ex, &ws, s)));
                }
                EOD_CU(fro_norm<T>(z, m, 1, m, d_t, iflag + 1, &ws, s));
                EOD_CU(cudaMemcpyAsync(tdiag_d + nt, d_t, sizeof(double), cudaMemcpyDeviceToDevice, s));
                ++nt;
                EOD_CU(cudaMemcpyAsync(hm.val, d_t, sizeof(double), cudaMemcpyDeviceToHost, s));
                EOD_CU(cudaStreamSynchronize(s));
                const double t = hm.val[0];
                ++restarts;
                if (!(t > eps)) {
                    stop = true;
                } else {
                    EOD_CU(scale_column<T>(z, m, d_t, s));
                    EOD_CU((copy_matrix<T, T>(z, m, Qb + kept * m, m, m, 1, false, s)));
                    EOD_CU(oz_append(kept, 1));
                    kept += 1;
                    cur += p + 1;
                }
            }
        }
    }
    if (ahead) EOD_CU(stream_after(s, s2));   // an unused lookahead: its buffers are shared after this
    // the T diagonal recorded on the device, and every panel's second pass
    // checked: it factored all p columns
    if (nt > 0 || !panel_p.empty()) {
        std::vector<int> pinf(2 * panel_p.size() + 1);
        tdiag.resize((size_t)nt);
        if (nt > 0) EOD_CU(cudaMemcpyAsync(tdiag.data(), tdiag_d, sizeof(double) * nt, cudaMemcpyDeviceToHost, s));
        if (!panel_p.empty())
            EOD_CU(cudaMemcpyAsync(pinf.data(), pinfo, sizeof(int) * 2 * panel_p.size(), cudaMemcpyDeviceToHost, s));
        EOD_CU(cudaStreamSynchronize(s));
        for (size_t i = 0; i < panel_p.size(); ++i)
            if (pinf[2 * i] != panel_p[i] || pinf[2 * i + 1] != CHOL_ALL) return EOD_EPRECISION;
    }
    const int64_t r = kept;
    F->rank = r;
    F->blocks = blocks;
    F->restarts = restarts;

    // t_margin over the tested entries
    double margin = INFINITY;
    for (size_t i = 0; i < tdiag.size(); ++i)
        if (tdiag[i] > 0.0 && eps > 0.0) margin = std::min(margin, std::fabs(std::log10(tdiag[i] / eps)));
    F->t_margin = margin;
    F->ntdiag = (int64_t)tdiag.size();
    F->tdiag = (double *)std::malloc(sizeof(double) * std::max<size_t>(tdiag.size(), 1));
    if (!F->tdiag) return EOD_ENOMEM;
    if (!tdiag.empty()) std::memcpy(F->tdiag, tdiag.data(), sizeof(double) * tdiag.size());

    if (r == 0) {
        F->rel_err = (norm_a > 0.0) ? 1.0 : 0.0;
        if (!o.compute_err) F->rel_err = -1.0;
        return EOD_OK;
    }

    // ---- Alg. 2 step 8: C^T = A^T Q (n x r) ----
    T *Ct, *V, *U, *Rt;
    double *D, *Rc;
    EOD_TRY(ar.get(&Ct, (size_t)n * r));
    EOD_TRY(ar.get(&V, (size_t)n * r));
    EOD_TRY(ar.get(&U, (size_t)m * r));
    EOD_TRY(ar.get(&Rt, (size_t)r * r));
    EOD_TRY(ar.get(&D, (size_t)r * r));
    EOD_TRY(ar.get(&Rc, (size_t)r * r));
    // work space of the CholQR passes (subspace iteration and core)
    CoreWork<T> cw;
    cw.pcap = r;
    cw.tc = mixed;
    const int64_t nblk = (r + kNBMin - 1) / kNBMin;
    EOD_TRY(ar.get(&cw.G, (size_t)r * r));
    EOD_TRY(ar.get(&cw.R, (size_t)r * r));
    EOD_TRY(ar.get(&cw.Rp, (size_t)r * r));
    EOD_TRY(ar.get(&cw.RiD, (size_t)((r + kPB - 1) / kPB) * kPB * kPB));
    EOD_TRY(ar.get(&cw.RiT, (size_t)kPB * kPB));
    EOD_TRY(ar.get(&cw.trace, 1));
    EOD_TRY(ar.get(&cw.part, (size_t)kOffIdMaxBlocks));
    EOD_TRY(ar.get(&cw.InvT, (size_t)std::max<int64_t>(r, kPB) * kPB));
    EOD_TRY(ar.get(&cw.Tmp, (size_t)std::max(m, n) * kPB));
    EOD_TRY(ar.get(&cw.info, (size_t)2 * nblk));

    // Ct (n x r) = A^T Q: Alg. 2 step 8 (transposed), and step 3 of each
    // subspace iteration
    auto project = [&]() -> eod_status {
        if (mixed) {
            EOD_TRY(mx.project(Qb, r, Ct, s));
        } else if (oz.on) {
            const OzOperand acol{oz.Acol, oz.eAcol, 0, oz.m8, n * oz.m8};
            const OzOperand qc{oz.Qc, oz.eQc, 0, oz.m8, cap * oz.m8};
            EOD_CU(oz_gemm_ops(acol, qc, n, r, m, 1.0, 0.0, (double *)Ct, n, ex, ws.err_flag, s));
        } else {
            EOD_CU((gemm<T, T, T, T>(true, false, n, r, m, 1.0, A, lda, Qb, m, 0.0, Ct, n, ex, &ws, s)));
        }
        return EOD_OK;
    };

    // ---- Alg. 2 steps 2-7: tau subspace iterations on the rank-r basis ----
    if (o.power_iters > 0) {
        Phase ph("eod.subspace_iteration");
        uint16_t *qts = nullptr;
        int *eqt = nullptr;
        const int64_t n8 = round_up8(n);
        if (oz.on) {
            EOD_TRY(ar.get(&qts, (size_t)kOzSlices * r * n8));
            EOD_TRY(ar.get(&eqt, (size_t)r));
        }
        for (int it = 0; it < o.power_iters; ++it) {
            EOD_TRY(project());                                          // step 3: Yt = A^T Q
            EOD_TRY(cholqr2(cw, Ct, n, n, r, Rc, hm, &ws, s));            // step 4: Yt = Qt Rt
            if (oz.on) {                                                 // step 5: Y = A Qt
                // B operand Qt: rows = its r columns, K = n
                EOD_CU(oz_slice((const double *)Ct, r, n, n, 1, qts, eqt, 0, n8, r * n8, s));
                const OzOperand qto{qts, eqt, 0, n8, r * n8};
                EOD_CU(oz_gemm_ops(oz.arow(), qto, m, r, n, 1.0, 0.0, (double *)Qb, m, ex, ws.err_flag, s));
            } else {
                EOD_CU((gemm<T, T, T, T>(false, false, m, r, n, 1.0, A, lda, Ct, n, 0.0, Qb, m, ex, &ws, s)));
            }
            EOD_TRY(cholqr2(cw, Qb, m, m, r, Rc, hm, &ws, s));            // step 6: Y = Q R
            EOD_CU(oz_append(0, r));                                     // slices of the new Q
        }
    }

    {
        Phase ph("eod.projection");
        EOD_TRY(project());
    }

    // ---- reconstruction error: || A - Q C ||_F / ||A||_F ----
    // It needs only Q and C, so it runs on a side stream while the core
    // (steps 9-11, a chain of small FP64 factorisations) runs on `s`.
    JoinOnExit join;
    if (o.compute_err) {
        Phase ph("eod.reconstruction_error");
        cudaStream_t se = side_stream();
        if (!se) se = s;
        join.main = s;
        if (mixed) {
            join.side = se;
            EOD_TRY(mx.recon_error(Qb, r, Ct, d_norm, d_err, s, se));
        } else {
            const int64_t nct = gemm_err_ctas(m, n);
            double *part;
            EOD_TRY(ar.get(&part, (size_t)nct));
            const bool emulated = oz.on && fp64_use_emulated(m, n, r) && r <= kOzErrMaxK;
            uint16_t *cts = nullptr;
            int *ects = nullptr;
            const int64_t r8 = round_up8(r);
            if (emulated) {
                EOD_TRY(ar.get(&cts, (size_t)kOzSlices * n * r8));
                EOD_TRY(ar.get(&ects, (size_t)n));
            }
            // the SIMT path takes split-K partials from the shared workspace:
            // only the emulated product (no workspace use) leaves `s`
            if (!emulated) se = s;
            join.side = se;
            EOD_CU(stream_after(se, s));
            EOD_CU(cudaMemsetAsync(part, 0, sizeof(double) * (size_t)nct, se));
            GemmExtra ee;
            ee.epilogue = EPI_ERR;
            ee.ref = A;
            ee.ldref = lda;
            ee.err_partials = part;
            if (emulated) {
                // B operand (C^T)^T: rows = rows of C^T (n), K = r
                EOD_CU(oz_slice((const double *)Ct, n, r, 1, n, cts, ects, 0, r8, n * r8, se));
                const OzOperand qr{oz.Qr, nullptr, 1, oz.cap8, m * oz.cap8};
                const OzOperand cto{cts, ects, 0, r8, n * r8};
                EOD_CU(oz_gemm_ops(qr, cto, m, n, r, 1.0, 0.0, nullptr, m, ee, ws.err_flag, se));
            } else {
                EOD_CU((gemm<T, T, T, T>(false, true, m, n, r, 1.0, Qb, m, Ct, n, 0.0, (T *)nullptr, m, ee, &ws, se)));
            }
            EOD_CU(finalize_sqrt_sum(part, nct, d_norm, d_err, se));
        }
    }

    // ---- steps 9-11 ----
    Phase ph_core("eod.core");
    EOD_CU((copy_matrix<T, T>(Ct, n, V, n, n, r, false, s)));
    EOD_TRY(cholqr2(cw, V, n, n, r, Rc, hm, &ws, s));                 // C^T = V R
    EOD_CU((copy_matrix<double, T>(Rc, r, Rt, r, r, r, true, s)));    // R^T
    EOD_TRY(cholqr2(cw, Rt, r, r, r, D, hm, &ws, s));                 // R^T = Qh D
    if (oz.on && fp64_use_emulated(m, r, r)) {   // U = Q Qh
        const int64_t r8 = round_up8(r);
        uint16_t *qhs;
        int *eqh;
        EOD_TRY(ar.get(&qhs, (size_t)kOzSlices * r * r8));
        EOD_TRY(ar.get(&eqh, (size_t)r));
        EOD_CU(oz_slice((const double *)Rt, r, r, r, 1, qhs, eqh, 0, r8, r * r8, s));
        const OzOperand qr{oz.Qr, nullptr, 1, oz.cap8, m * oz.cap8};
        const OzOperand qho{qhs, eqh, 0, r8, r * r8};
        EOD_CU(oz_gemm_ops(qr, qho, m, r, r, 1.0, 0.0, (double *)U, m, ex, ws.err_flag, s));
    } else if (mixed && std::is_same<T, float>::value && m >= kTfMinRows && r >= 32) {
        // U = Q Qh on the tensor cores as three TF32 products of split
        // operands, X = X_hi + X_lo (X_hi Y_hi + X_hi Y_lo + X_lo Y_hi: about
        // 2^-21 relative, the accuracy of an FP32 product); TF32 operands are
        // K-major, so Q is split transposed (r4 x m)
        const int64_t r4 = round_up(r, 4);
        float *q_hi, *q_lo, *h_hi, *h_lo;
        EOD_TRY(ar.get(&q_hi, (size_t)(r4 * m)));
        EOD_TRY(ar.get(&q_lo, (size_t)(r4 * m)));
        EOD_TRY(ar.get(&h_hi, (size_t)(r4 * r)));
        EOD_TRY(ar.get(&h_lo, (size_t)(r4 * r)));
        EOD_CU(split_transpose_tf32((const float *)Qb, m, r, m, q_hi, q_lo, r4, s));
        EOD_CU(split_tf32((const float *)Rt, r, r, r, h_hi, h_lo, r4, s));
        TcGemmDesc g;
        g.M = m;
        g.N = r;
        g.K = r;
        g.tf32 = true;
        g.npairs = 3;
        const TcOperand qh{q_hi, r, m, r4}, ql{q_lo, r, m, r4}, hh{h_hi, r, r, r4}, hl{h_lo, r, r, r4};
        g.a[0] = qh, g.b[0] = hh;
        g.a[1] = qh, g.b[1] = hl;
        g.a[2] = ql, g.b[2] = hh;
        g.D = (float *)U;
        g.ldd = m;
        g.err_flag = ws.err_flag;
        EOD_CU(tc_gemm_run(g, &ws, s));
    } else {
        EOD_CU((gemm<T, T, T, T>(false, false, m, r, r, 1.0, Qb, m, Rt, r, 0.0, U, m, ex, &ws, s)));
    }

    join.join();
    if (o.compute_err) {
        EOD_CU(cudaMemcpyAsync(hm.val, d_err, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    EOD_CU(cudaStreamSynchronize(s));
    F->rel_err = o.compute_err ? hm.val[0] : -1.0;
    if (mixed) EOD_TRY(mx.check(s));
    EOD_CU(cudaMemcpyAsync(hm.flag, ws.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    EOD_CU(cudaStreamSynchronize(s));
    if (hm.flag[0]) return EOD_ETIMEOUT;

    F->U = U; ar.keep(U);
    F->V = V; ar.keep(V);
    F->D = D; ar.keep(D);
    F->Q = Qb; ar.keep(Qb);
    F->C = Ct; ar.keep(Ct);
    return EOD_OK;
}

eod_status factor_mixed_from_f64(const double *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                                 const eod_opts &o, cudaStream_t s, eod_factors *F);

static eod_status validate(const void *A, int64_t m, int64_t n, int64_t lda, double tol, const eod_opts &o) {
    if (!A || m < 1 || n < 1 || lda < m) return EOD_EINVAL;
    if (!(tol > 0.0) || !std::isfinite(tol)) return EOD_EINVAL;
    if (o.power_iters < 0 || o.power_iters > kMaxPowerIters) return EOD_EINVAL;
    if (o.a_dtype != EOD_F64 && o.a_dtype != EOD_F32) return EOD_EINVAL;
    if (o.precision != EOD_PLAIN && o.precision != EOD_MIXED_BF16 && o.precision != EOD_MIXED_TF32) return EOD_EINVAL;
    if (o.tol_mode != EOD_TOL_ABS && o.tol_mode != EOD_TOL_REL_FRO) return EOD_EINVAL;
    if (o.block_k < 0 || o.block_k > 128) return EOD_EINVAL;
    if (m > 0x7FFFFFFFLL || n > 0x7FFFFFFFLL) return EOD_EINVAL;
    return EOD_OK;
}

static void free_factors_device(eod_factors *f) {
    if (!f) return;
    if (release_pooled_factors(f)) {   // factors of a persistent batch
        std::free(f->tdiag);
        f->tdiag = nullptr;
        return;
    }
    void *ptrs[] = {f->U, f->V, f->Q, f->C, (void *)f->D};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    std::free(f->tdiag);
    f->U = f->V = f->Q = f->C = nullptr;
    f->D = nullptr;
    f->tdiag = nullptr;
}

eod_status factor_any(const void *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                      const eod_opts *opts, eod_factors **out) {
    if (!out) return EOD_EINVAL;
    *out = nullptr;
    eod_opts o;
    eod_opts_default(&o);
    if (opts) o = *opts;
    EOD_TRY(validate(A, m, n, lda, tol, o));
    if (o.block_k == 0) {
        // the autotuner's k for this form and size, else 32
        const int64_t form = o.precision == EOD_MIXED_BF16 ? 2 : o.precision == EOD_MIXED_TF32 ? 3
                             : o.a_dtype == EOD_F32 ? 1 : 0;
        int64_t k = 0;
        if (tuned_value("block_k", form, m, n, &k) && k >= 1 && k <= 128) o.block_k = (int32_t)k;
    }
    cudaStream_t s = (cudaStream_t)o.stream;
    eod_factors *F = (eod_factors *)std::calloc(1, sizeof(eod_factors));
    if (!F) return EOD_ENOMEM;
    F->m = m;
    F->n = n;
    F->precision = o.precision;
    F->f_dtype = (o.a_dtype == EOD_F64 && o.precision == EOD_PLAIN) ? EOD_F64 : EOD_F32;
    F->rel_err = -1.0;
    eod_status st;
    {
        Arena ar(s);
        if (o.precision == EOD_PLAIN && o.a_dtype == EOD_F64)
            st = factor_impl<double>((const double *)A, m, n, lda, tol, seed, o, s, ar, F);
        else if (o.a_dtype == EOD_F32)
            st = factor_impl<float>((const float *)A, m, n, lda, tol, seed, o, s, ar, F);
        else
            st = factor_mixed_from_f64((const double *)A, m, n, lda, tol, seed, o, s, F);
        if (st != EOD_OK) {
            // the arena frees its own buffers; the kept ones belong to F
            free_factors_device(F);
        }
    }
    if (st != EOD_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        std::free(F);
        return st;
    }
    *out = F;
    return EOD_OK;
}

// FP64 input on the mixed path: widen nothing, narrow A to FP32 once (the
// tensor-core path splits FP32 values into BF16 pairs).
eod_status factor_mixed_from_f64(const double *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                                 const eod_opts &o, cudaStream_t s, eod_factors *F) {
    float *A32 = nullptr;
    cudaError_t e = lib_malloc_async((void **)&A32, sizeof(float) * (size_t)m * n, s);
    if (e != cudaSuccess) { cudaGetLastError(); return EOD_ENOMEM; }
    eod_status st = EOD_OK;
    if (copy_matrix<double, float>(A, lda, A32, m, m, n, false, s) != cudaSuccess) st = EOD_ECUDA;
    if (st == EOD_OK) {
        Arena ar(s);
        eod_opts o2 = o;
        o2.a_dtype = EOD_F32;
        st = factor_impl<float>(A32, m, n, m, tol, seed, o2, s, ar, F);
        if (st != EOD_OK) free_factors_device(F);
    }
    cudaFreeAsync(A32, s);
    return st;
}

template <typename T>
static eod_status reconstruct_impl(const eod_factors *f, T *Ahat, int64_t ld, cudaStream_t s) {
    const int64_t m = f->m, n = f->n, r = f->rank;
    if (r == 0) {
        EOD_CU(fill_zero<T>(Ahat, m, n, ld, s));
        return EOD_OK;
    }
    Arena ar(s);
    Scratch ws;
    EOD_TRY(ar.get((char **)&ws.base, (size_t)32 << 20));
    ws.size = (size_t)32 << 20;
    T *W, *Dt;
    EOD_TRY(ar.get(&W, (size_t)m * r));
    EOD_TRY(ar.get(&Dt, (size_t)r * r));
    EOD_CU((copy_matrix<double, T>(f->D, r, Dt, r, r, r, false, s)));
    GemmExtra ex, bu;
    bu.b_upper = true;
    const T *U = (const T *)f->U, *V = (const T *)f->V;
    EOD_CU((gemm<T, T, T, T>(false, false, m, r, r, 1.0, U, m, Dt, r, 0.0, W, m, bu, &ws, s)));     // W = U D
    EOD_CU((gemm<T, T, T, T>(false, true, m, n, r, 1.0, W, m, V, n, 0.0, Ahat, ld, ex, &ws, s)));  // A_hat = W V^T
    return EOD_OK;
}

}  // namespace eod

// ===========================================================================
// Exported C ABI
// ===========================================================================
using namespace eod;

extern "C" {

void eod_opts_default(eod_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->a_dtype = EOD_F64;
    o->precision = EOD_PLAIN;
    o->tol_mode = EOD_TOL_ABS;
    o->block_k = 0;
    o->power_iters = 0;
    o->compute_err = 1;
    o->stream = nullptr;
    o->batch_index = 0;
}

eod_status eod_abe_factor(const void *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                          eod_factors **out) {
    return factor_any(A, m, n, lda, tol, seed, nullptr, out);
}

eod_status eod_abe_factor_ex(const void *A, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                             const eod_opts *opts, eod_factors **out) {
    return factor_any(A, m, n, lda, tol, seed, opts, out);
}

eod_status eod_abe_factor_host(const void *A_host, int64_t m, int64_t n, int64_t lda, double tol, uint64_t seed,
                               const eod_opts *opts, void *U_host, double *D_host, void *V_host, int64_t cap,
                               int64_t *rank, double *rel_err) {
    eod_opts o;
    eod_opts_default(&o);
    if (opts) o = *opts;
    if (!A_host || !rank || m < 1 || n < 1 || lda < m) return EOD_EINVAL;
    if ((U_host || D_host || V_host) && cap < std::min(m, n)) return EOD_EINVAL;
    if (o.a_dtype != EOD_F64 && o.a_dtype != EOD_F32) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)o.stream;
    const size_t es = o.a_dtype == EOD_F64 ? 8 : 4;
    void *Ad = nullptr;
    if (g_fail_alloc_after > 0 && --g_fail_alloc_after == 0) return EOD_ENOMEM;
    if (lib_malloc_async(&Ad, es * (size_t)m * n, s) != cudaSuccess) { cudaGetLastError(); return EOD_ENOMEM; }
    eod_status st = EOD_OK;
    if (cudaMemcpy2DAsync(Ad, es * m, A_host, es * lda, es * m, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = EOD_ECUDA;
    eod_factors *F = nullptr;
    if (st == EOD_OK) st = factor_any(Ad, m, n, m, tol, seed, &o, &F);
    if (st == EOD_OK) {
        const int64_t r = F->rank;
        const size_t fs = F->f_dtype == EOD_F64 ? 8 : 4;
        *rank = r;
        if (rel_err) *rel_err = F->rel_err;
        if (r > 0) {
            if (U_host && cudaMemcpyAsync(U_host, F->U, fs * (size_t)m * r, cudaMemcpyDeviceToHost, s) != cudaSuccess) st = EOD_ECUDA;
            if (V_host && cudaMemcpyAsync(V_host, F->V, fs * (size_t)n * r, cudaMemcpyDeviceToHost, s) != cudaSuccess) st = EOD_ECUDA;
            if (D_host && cudaMemcpy2DAsync(D_host, sizeof(double) * cap, F->D, sizeof(double) * r, sizeof(double) * r, r,
                                            cudaMemcpyDeviceToHost, s) != cudaSuccess) st = EOD_ECUDA;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) st = EOD_ECUDA;
        eod_abe_free(F);
    }
    cudaFreeAsync(Ad, s);
    cudaStreamSynchronize(s);
    return st;
}

eod_status eod_abe_reconstruct(const eod_factors *f, void *A_hat, int64_t ld_hat, const eod_opts *opts) {
    if (!f || !A_hat || ld_hat < f->m) return EOD_EINVAL;
    eod_opts o;
    eod_opts_default(&o);
    o.a_dtype = f->f_dtype;
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)o.stream;
    eod_status st;
    if (o.a_dtype == EOD_F64 && f->f_dtype == EOD_F64)
        st = reconstruct_impl<double>(f, (double *)A_hat, ld_hat, s);
    else if (o.a_dtype == EOD_F32 && f->f_dtype == EOD_F32)
        st = reconstruct_impl<float>(f, (float *)A_hat, ld_hat, s);
    else
        return EOD_EUNSUPPORTED;
    if (st == EOD_OK && cudaStreamSynchronize(s) != cudaSuccess) st = EOD_ECUDA;
    return st;
}

eod_status eod_abe_factor_batched(const void *const *A, const int64_t *m, const int64_t *n, const int64_t *lda,
                                  int64_t count, double tol, uint64_t seed, const eod_opts *opts, eod_factors **out,
                                  eod_status *per_item) {
    if (!A || !m || !n || !lda || !out || !per_item || count < 1) return EOD_EINVAL;
    eod_opts o;
    eod_opts_default(&o);
    if (opts) o = *opts;
    for (int64_t i = 0; i < count; ++i) {
        out[i] = nullptr;
        per_item[i] = EOD_EINVAL;
    }
    // FP32 items first go through the persistent launch (batch.cu); what it
    // hands back (rank above its capacity, shifted CholQR needed, other
    // forms) runs below, one single-matrix factorisation per item on a pool
    // of worker streams.  EOD_BATCH_PERSISTENT=0 skips the persistent launch.
    std::vector<int64_t> todo;
    const char *pers_env = std::getenv("EOD_BATCH_PERSISTENT");
    if (o.a_dtype == EOD_F32 && !(pers_env && pers_env[0] == '0')) {
        const eod_status pst = factor_batched_persistent(A, m, n, lda, count, tol, seed, o, out, per_item, todo);
        if (pst != EOD_OK) {
            for (int64_t i = 0; i < count; ++i) per_item[i] = pst;
            return pst;
        }
    } else {
        for (int64_t i = 0; i < count; ++i) todo.push_back(i);
    }
    if (todo.empty()) {
        for (int64_t i = 0; i < count; ++i)
            if (per_item[i] != EOD_OK) return per_item[i];
        return EOD_OK;
    }
    // longest first: the rank is unknown, so m * n * min(m, n) stands in for the cost
    std::vector<int64_t> order(todo);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const double ca = (double)m[a] * n[a] * std::min(m[a], n[a]);
        const double cb = (double)m[b] * n[b] * std::min(m[b], n[b]);
        return ca > cb;
    });
    // worker streams: EOD_BATCH_STREAMS, else the autotuner's value for this
    // batch (count, mean m, mean n), else 8
    int workers = 8;
    if (const char *env = std::getenv("EOD_BATCH_STREAMS")) {
        workers = std::max(1, std::atoi(env));
    } else {
        double sm = 0.0, sn = 0.0;
        for (int64_t i = 0; i < count; ++i) {
            sm += (double)m[i];
            sn += (double)n[i];
        }
        int64_t v = 0;
        if (tuned_value("batch_workers", count, (int64_t)(sm / count), (int64_t)(sn / count), &v) && v >= 1 && v <= 64)
            workers = (int)v;
    }
    if (workers > (int64_t)order.size()) workers = (int)order.size();
    // block_k = 0: the autotuner's k for batched items of this size class
    // (timed under the workers' concurrency), else each item's own tuned k
    int32_t batch_k = 0;
    if (o.block_k == 0) {
        double sm = 0.0, sn = 0.0;
        for (int64_t i : order) {
            sm += (double)m[i];
            sn += (double)n[i];
        }
        const int64_t form = o.precision == EOD_MIXED_BF16 ? 2 : o.precision == EOD_MIXED_TF32 ? 3
                             : o.a_dtype == EOD_F32 ? 1 : 0;
        int64_t v = 0;
        if (tuned_value("batch_block_k", form, (int64_t)(sm / order.size()), (int64_t)(sn / order.size()), &v) &&
            v >= 1 && v <= 128)
            batch_k = (int32_t)v;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return EOD_ECUDA; }
    // work already queued on the caller's stream (for example the matrices
    // themselves) must finish before any worker stream reads it
    cudaStream_t caller = (cudaStream_t)o.stream;
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, caller) != cudaSuccess) {
        cudaGetLastError();
        if (ready) cudaEventDestroy(ready);
        return EOD_ECUDA;
    }
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        const bool own = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (!own) { cudaGetLastError(); st = caller; }
        cudaStreamWaitEvent(st, ready, 0);
        for (;;) {
            const int64_t j = next.fetch_add(1);
            if (j >= (int64_t)order.size()) break;
            const int64_t i = order[(size_t)j];
            eod_opts oi = o;
            if (oi.block_k == 0 && batch_k > 0) oi.block_k = batch_k;
            oi.batch_index = (uint64_t)i;
            oi.stream = st;
            per_item[i] = factor_any(A[i], m[i], n[i], lda[i], tol, seed, &oi, &out[i]);
        }
        cudaStreamSynchronize(st);
        if (own) cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    cudaEventDestroy(ready);
    eod_status first = EOD_OK;
    for (int64_t i = 0; i < count; ++i)
        if (per_item[i] != EOD_OK) { first = per_item[i]; break; }
    return first;
}

eod_status eod_abe_omega(int64_t n, int64_t col0, int64_t ncols, uint64_t seed, uint64_t batch, double *out,
                         void *stream) {
    if (n < 1 || ncols < 1 || col0 < 0 || !out) return EOD_EINVAL;
    if (n > 0xFFFFFFFFLL || col0 + ncols > 0xFFFFFFFFLL || batch > 0xFFFFFFFFull) return EOD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (omega_fill<double>(n, col0, ncols, seed, batch, out, n, s) != cudaSuccess) return EOD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return EOD_ECUDA;
    return EOD_OK;
}

void eod_abe_free(eod_factors *f) {
    if (!f) return;
    free_factors_device(f);
    std::free(f);
}

const char *eod_status_string(eod_status s) {
    switch (s) {
    case EOD_OK: return "ok";
    case EOD_EINVAL: return "invalid argument";
    case EOD_ENOMEM: return "out of memory";
    case EOD_ECUDA: return "CUDA error";
    case EOD_ENONFINITE: return "matrix holds NaN or Inf";
    case EOD_ETIMEOUT: return "device wait timed out";
    case EOD_EPRECISION: return "Cholesky breakdown beyond the shifted fallback";
    case EOD_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

int64_t eod_abe_storage_entries(int64_t m, int64_t n, int64_t r) { return r * (m + n) + r * (r + 1) / 2; }

double eod_abe_model_flops(int64_t m, int64_t n, int64_t r, int64_t k, int32_t with_err) {
    const double M = (double)m, N = (double)n, Rr = (double)r, K = (double)k;
    double f = 2.0 * (2.0 * M * N * Rr + M * Rr * Rr + 2.0 * N * Rr * Rr + 2.0 * Rr * Rr * Rr + 4.0 * M * Rr * K);
    if (with_err) f += 2.0 * M * N * Rr;
    return f;
}

void eod_abe_debug_fail_alloc_after(int32_t n) { g_fail_alloc_after = n > 0 ? n : 0; }

const char *eod_abe_version(void) { return "eod-abe-gb300 0.1 (sm_103a)"; }

}  // extern "C"

/*
 * eod_abe.h - C ABI of the GB300 (sm_103a) implementation of power-free
 * EOD-ABE: efficient orthogonal decomposition with automatic basis
 * extraction (Xu, Shen, Liu, Jia; arXiv 2506.22713).
 *
 * The method (paper Sec. 3): for A (m x n) and a tolerance eps > 0,
 *   Alg. 1 (BasisExt)  draws Gaussian blocks Omega_j (n x k), forms
 *                      Y_j = (I - Q Q^T) A Omega_j, factors Y_j = P_j T_j and
 *                      stops at the first diagonal entry |T_j(l,l)| <= eps,
 *                      keeping Q = [Q, P_j(:, 1:l-1)]; r = columns of Q;
 *   Alg. 2, tau = 0    C = Q^T A;  C^T = V R (QR);  R^T = Qh Dh (QR);
 *                      U = Q Qh, D = Dh;  A ~= A_hat = U D V^T = Q C.
 * The relative Frobenius error ||A - A_hat||_F / ||A||_F is the RelErr of
 * Sec. 4.1.
 *
 * Conventions shared by every call:
 *  - Matrices are column-major: entry (i, j) of A is A[i + j*lda].
 *  - Unless a parameter says "host", pointers are CUDA device pointers in the
 *    current device's context.  The library never modifies A.
 *  - Work is issued on opts->stream (a cudaStream_t; NULL = the legacy
 *    default stream).  Calls that return a rank return after synchronising
 *    that stream, because the rank is a host value.
 *  - Status codes: EOD_OK on success; on any other status the output
 *    pointer is left NULL (or untouched) and nothing needs freeing.
 *  - Not thread-safe per stream: concurrent calls must use different streams.
 */
#ifndef EOD_ABE_H
#define EOD_ABE_H

#include <stdint.h>

#if defined(__GNUC__)
#define EOD_API __attribute__((visibility("default")))
#else
#define EOD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EOD_OK = 0,
    EOD_EINVAL = 1,        /* bad argument: sizes, lda, tol <= 0 or not finite,
                              power_iters outside 0..16, unknown enum value, NULL pointer */
    EOD_ENOMEM = 2,        /* device or pinned host allocation failed */
    EOD_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    EOD_ENONFINITE = 4,    /* A holds a NaN or an infinity */
    EOD_ETIMEOUT = 5,      /* a bounded device-side wait gave up (kernel returned
                              an error flag instead of waiting forever) */
    EOD_EPRECISION = 6,    /* eps is below what FP32 data can resolve
                              (eps < 1e-5 ||A||_F with EOD_F32 storage or on
                              the mixed path), or a Cholesky factorisation
                              broke down beyond the shifted fallback's reach */
    EOD_EUNSUPPORTED = 7   /* valid request the library does not support */
} eod_status;

typedef enum { EOD_F64 = 0, EOD_F32 = 1 } eod_dtype;

typedef enum {
    EOD_PLAIN = 0,         /* every contraction at the precision of A's storage
                              type.  EOD_F64: products of at least 2^25
                              multiply-adds run as an exact FP64 emulation on
                              the tcgen05 tensor cores (each operand split into
                              eight BF16 digit slices, integer-exact partial
                              products, FP64 accumulation; normwise error about
                              K 2^-48 |A(i,:)| |B(:,j)|), smaller ones as FP64
                              DFMA; EOD_F32: FP32 FFMA.  Gram/Cholesky/rank
                              test/core in FP64 */
    EOD_MIXED_BF16 = 1,    /* sketch, projection and reconstruction on tcgen05
                              tensor cores with FP32 accumulation: A split into
                              three BF16 terms for the sketch (exact for FP32
                              data), two for the projection and the error;
                              from m >= 1024 rows also U = Q Qh and the
                              solves W R^-1 of the second and later CholQR
                              passes (Grams of >= 128 columns) as three TF32
                              products of split operands (~2^-21 relative);
                              Gram/Cholesky/rank test/core R factors in FP64 */
    EOD_MIXED_TF32 = 2     /* the same contractions with tcgen05 kind::tf32:
                              A, Q and C split into two TF32 terms (hi = the
                              value with 13 low significand bits cleared,
                              lo = the exact rest; dropped terms ~2^-21
                              relative, against ~2^-16 for the BF16 form), at
                              half the BF16 MMA rate and twice its operand
                              bytes; FP32 data as for EOD_MIXED_BF16 */
} eod_precision;

typedef enum {
    EOD_TOL_ABS = 0,       /* eps = tol: the test |T(l,l)| <= eps of Alg. 1 as printed */
    EOD_TOL_REL_FRO = 1    /* eps = tol * ||A||_F */
} eod_tol_mode;

/* Options.  eod_opts_default() fills: F64, PLAIN, TOL_ABS, block_k 0 (the
 * tuned k, eod_abe_tuning_load, else 32),
 * power_iters 0, compute_err 1, stream NULL, batch_index 0. */
typedef struct {
    int32_t a_dtype;       /* eod_dtype of A (and of A_hat in eod_abe_reconstruct) */
    int32_t precision;     /* eod_precision */
    int32_t tol_mode;      /* eod_tol_mode */
    int32_t block_k;       /* block size k of Alg. 1 (1..128); 0 selects the tuned
                              k for this form and size, else 32 */
    int32_t power_iters;   /* tau of Alg. 2 (0..16): subspace iterations after
                              BasisExt, steps 2-7 (Y~ = A^T Q, QR, Y = A Q~, QR),
                              on the rank BasisExt found; 0 = power-free.  The
                              QRs are CholQR2 with positive diagonals, so Q_tau
                              and the factors are unique given Omega; in the
                              mixed forms A^T Q uses their split and A Q~ FP32 */
    int32_t compute_err;   /* nonzero: compute RelErr (one more pass over A) */
    void *stream;          /* cudaStream_t */
    uint64_t batch_index;  /* third counter word of the Omega draw (Philox) */
} eod_opts;

/* Result of one factorisation.  All matrix fields are device pointers owned
 * by the struct and released by eod_abe_free().  U, V, Q and C hold FP64 for
 * a_dtype EOD_F64 with EOD_PLAIN and FP32 otherwise (f_dtype says which);
 * D is always FP64.  For rank 0 every matrix pointer is NULL. */
typedef struct {
    int64_t m, n, rank;
    int32_t f_dtype;       /* eod_dtype of U, V, Q, C */
    int32_t precision;     /* eod_precision used */
    void *U;               /* m x rank, ld m: U = Q Qh, orthonormal columns */
    double *D;             /* rank x rank, ld rank: upper triangular, positive diagonal */
    void *V;               /* n x rank, ld n: orthonormal columns */
    void *Q;               /* m x rank, ld m: the BasisExt basis */
    void *C;               /* n x rank, ld n: C^T = A^T Q (the projection B^T) */
    double *tdiag;         /* host array, ntdiag entries: every computed |T_j(l,l)|, in order */
    int64_t ntdiag;
    double rel_err;        /* ||A - Q C||_F / ||A||_F, or -1 if not computed */
    double norm_a;         /* ||A||_F */
    double eps;            /* threshold used: tol or tol*||A||_F */
    double t_margin;       /* min over tested entries of |log10(|T(l,l)| / eps)| */
    int64_t blocks;        /* blocks of Alg. 1 processed */
    int64_t restarts;      /* columns settled by the explicit residual check */
    int64_t block_k;       /* k used */
} eod_factors;

/* Fills *opts with the defaults listed above. */
EOD_API void eod_opts_default(eod_opts *opts);

/* Alg. 2 with tau = 0 (paper Sec. 3.2) on device matrix A (m x n, ld lda >=
 * m, FP64), threshold eps = tol (absolute), Omega from `seed`, default
 * options.  On EOD_OK *out receives a new eod_factors (free with
 * eod_abe_free).  Errors: EOD_EINVAL for m < 1, n < 1, lda < m, tol <= 0 or
 * non-finite, out == NULL; EOD_ENONFINITE if A holds NaN/Inf; EOD_ENOMEM,
 * EOD_ECUDA as described above.  A zero matrix gives EOD_OK with rank 0.
 * m < n is accepted (the paper assumes m >= n and notes that the method
 * carries over); the rank never exceeds min(m, n). */
EOD_API eod_status eod_abe_factor(const void *A, int64_t m, int64_t n, int64_t lda,
                          double tol, uint64_t seed, eod_factors **out);

/* As eod_abe_factor with explicit options (opts may be NULL = defaults). */
EOD_API eod_status eod_abe_factor_ex(const void *A, int64_t m, int64_t n, int64_t lda,
                             double tol, uint64_t seed, const eod_opts *opts,
                             eod_factors **out);

/* Same computation from a HOST matrix A_host (m x n, ld lda, type
 * opts->a_dtype); the library copies it to the device, factors it and copies
 * the factors back into caller-owned host buffers: U_host (m x cap, ld m),
 * D_host (cap x cap, ld cap, FP64), V_host (n x cap, ld n), where cap >=
 * min(m, n) is the capacity the caller allocated; U/V are written in
 * f_dtype (FP64 for F64+PLAIN, else FP32).  *rank and *rel_err receive the
 * rank and RelErr.  Any of U_host, D_host, V_host may be NULL to skip that
 * copy.  Pinned host memory makes the copies asynchronous; pageable memory
 * works too.  Errors as eod_abe_factor_ex, plus EOD_EINVAL for cap <
 * min(m, n) when a factor buffer is given. */
EOD_API eod_status eod_abe_factor_host(const void *A_host, int64_t m, int64_t n, int64_t lda,
                               double tol, uint64_t seed, const eod_opts *opts,
                               void *U_host, double *D_host, void *V_host, int64_t cap,
                               int64_t *rank, double *rel_err);

/* Rebuilds A_hat = U D V^T, the product of the three factors (paper Sec. 1),
 * into device buffer A_hat (m x n, ld ld_hat >= m), written in opts->a_dtype
 * (NULL opts: the factors' f_dtype).  Rank 0 writes zeros.  Errors:
 * EOD_EINVAL for NULL f or A_hat or ld_hat < m; EOD_EUNSUPPORTED when the
 * requested type differs from f_dtype. */
EOD_API eod_status eod_abe_reconstruct(const eod_factors *f, void *A_hat, int64_t ld_hat,
                               const eod_opts *opts);

/* Factors `count` independent matrices (the per-image use of Sec. 4.1) in
 * one call.  A, m, n, lda, out and per_item are HOST arrays of length count;
 * A[i] is a device pointer.  Item i draws Omega with batch_index = i.
 *
 * FP32 items (a_dtype EOD_F32, power_iters 0, block_k 0 or <= 64, m and n
 * <= 16384) first go through one persistent launch, captured in a CUDA graph:
 * each CTA takes items from a work queue, largest first, and factors each
 * one start to end on the device (Alg. 1's stop decision included), with
 * FP32 products (long dot products compensated), FP64-accurate Grams and the
 * FP64 leaf Cholesky, whatever precision was requested; those factor sets
 * report precision = EOD_PLAIN, block_k the k used (32 for block_k 0), and
 * share one device allocation released by the last eod_abe_free.  An item
 * whose rank exceeds 128, or whose core Gram the unshifted Cholesky cannot
 * factor, is handed to the path below.  EOD_BATCH_PERSISTENT=0 skips the
 * launch.
 *
 * Other items run concurrently on a pool of worker threads, each with its
 * own non-blocking stream (EOD_BATCH_STREAMS if set, else the tuned
 * "batch_workers", else 8), largest m*n*min(m,n) first, each an ordinary
 * eod_abe_factor_ex call with batch_index = i (same result bit for bit);
 * with block_k = 0 they take the tuned "batch_block_k" of the form and the
 * items' mean m, n when the table has one, else each item's own tuned k.
 *
 * Work already queued on opts->stream is waited for first.  Every item gets
 * its own status in per_item[i] and, on EOD_OK, its own factors in out[i]
 * (free each with eod_abe_free).  Returns EOD_OK if every item succeeded,
 * else the status of the lowest-index failing item (EOD_ECUDA for all if the
 * persistent launch itself failed after starting); EOD_EINVAL for count < 1
 * or NULL arrays. */
EOD_API eod_status eod_abe_factor_batched(const void *const *A, const int64_t *m, const int64_t *n,
                                  const int64_t *lda, int64_t count, double tol, uint64_t seed,
                                  const eod_opts *opts, eod_factors **out, eod_status *per_item);

/* Writes columns col0 .. col0+ncols-1 of the Gaussian test matrix Omega
 * (n rows; Alg. 1 step 3) for (seed, batch) into device buffer out (n x
 * ncols, ld n, FP64) on `stream`.  The draw: Philox4x32-10 (Salmon et al.,
 * SC'11) with counter (row, column, batch, 0) and key (seed low 32 bits, seed
 * high 32 bits); u = (x + 1/2) 2^-32 for the first two output words; Box-
 * Muller sqrt(-2 ln u1) cos(2 pi u2) in FP64, rounded to the nearest BF16
 * value (ties to even).  Errors: EOD_EINVAL for n < 1, ncols < 1, col0 < 0,
 * out == NULL, or a row/column index beyond 2^32 - 1. */
EOD_API eod_status eod_abe_omega(int64_t n, int64_t col0, int64_t ncols, uint64_t seed,
                         uint64_t batch, double *out, void *stream);

/* Releases the factors and the struct.  NULL is a no-op. */
EOD_API void eod_abe_free(eod_factors *f);

/* Static English text for a status code. */
EOD_API const char *eod_status_string(eod_status s);

/* Entries stored by U (m x r), upper-triangular D and V (n x r):
 * r(m + n) + r(r + 1)/2 (paper Sec. 1). */
EOD_API int64_t eod_abe_storage_entries(int64_t m, int64_t n, int64_t r);

/* Flops of the paper's cost model for tau = 0 (Sec. 3.4, "2mnr + mr^2 +
 * 2nr^2 + 2r^3 + 4mrk" multiply-adds, two flops each), plus 2mnr for the
 * reconstruction when with_err is nonzero. */
EOD_API double eod_abe_model_flops(int64_t m, int64_t n, int64_t r, int64_t k, int32_t with_err);

/* Test hook: the n-th device allocation from now (n >= 1) fails as if the
 * device were out of memory; n <= 0 clears the hook.  Host-side only. */
EOD_API void eod_abe_debug_fail_alloc_after(int32_t n);

/* Measurement hooks (no counterpart in the paper; they support the
 * benchmark's roofline figures).
 * eod_abe_debug_profile(1) clears and starts CUDA-event timing of every
 * kernel launch, grouped by kind: 0 SIMT GEMM, 1 one-CTA Cholesky / rank
 * test, 2 Omega generation, 3 streaming (norms, copies, splitting),
 * 4 tcgen05 tensor-core GEMM (mixed path), 5 FP64 GEMM emulated on tcgen05
 * (plain FP64 path), 6 slicing of FP64 operands into the BF16 digits of that
 * emulation, 7 SIMT GEMM and Gram in FP32 arithmetic (FP32-data paths; kind 0
 * is then the FP64 ones), 8 the persistent batched launch (one record per
 * launch); eod_abe_debug_profile(0) stops it and clears.
 * eod_abe_debug_profile_read() waits for the recorded events of one kind and
 * returns the launch count, the summed device time (ms) and the summed
 * algorithmic flops and bytes of those launches; EOD_EINVAL for an unknown
 * kind or NULL outputs.  eod_abe_debug_launch_count() is the number of
 * kernels the library has launched since it was loaded. */
EOD_API void eod_abe_debug_profile(int32_t enable);

/* Measurement hook of the persistent batched launch (eod_abe_factor_batched
 * on FP32 items): with enable != 0 every later launch sums, per phase of an
 * item, the SM clock ticks its CTAs spent there, in 11 counters: (unused:
 * the norm is summed inside the first sketch), Omega, sketch A Omega_j
 * (with the norm), projection against Q (step 4), Gram and
 * rank-test leaf (steps 5-11), the panel's CholQR2 products, explicit
 * residuals, C^T = A^T Q, reconstruction error, core QRs (steps 9-10),
 * U = Q Qh.  out (n >= 11 doubles, may be NULL) receives the last launch's
 * counters; EOD_EINVAL for n < 11 with non-NULL out.  Timing only: the
 * results do not change. */
EOD_API eod_status eod_abe_debug_batch_phases(int32_t enable, double *out, int64_t n);
EOD_API eod_status eod_abe_debug_profile_read(int32_t kind, int64_t *launches, double *total_ms,
                                              double *total_flops, double *total_bytes);
EOD_API int64_t eod_abe_debug_launch_count(void);

/* Test hook (no counterpart in the paper): one tcgen05 tensor-core
 * contraction of the mixed path on FP32 device inputs, split into BF16
 * hi/lo parts inside the call.  All matrices column-major.
 *   form 0 (sketch):          D (M x N) = X Y, X M x K (ld ldx), Y K x N
 *                             (ld ldy) holding BF16-exact values; X is read
 *                             M-contiguous as in A Omega.
 *   form 1 (projection):      D (M x N) = X^T Y, X K x M, Y K x N.
 *   form 2 (reconstruction):  *err_out (device double) = ||D - X Y^T||_F
 *                             with X M x K, Y N x K and D the M x N
 *                             reference (ld ldd); D is not written.
 *   form | 8:                 the same contraction in the TF32 form of
 *                             EOD_MIXED_TF32 (X and Y split into two TF32
 *                             terms; form 8 reads X through a transposed
 *                             copy and expects TF32-exact Y).
 * Returns after synchronising `stream`; EOD_ETIMEOUT if a bounded device
 * wait ran out, EOD_EINVAL for bad sizes or leading dimensions. */
EOD_API eod_status eod_abe_debug_tc_gemm(int32_t form, int64_t M, int64_t N, int64_t K, const float *X,
                                         int64_t ldx, const float *Y, int64_t ldy, float *D, int64_t ldd,
                                         double *err_out, void *stream);

/* ||A||_F of a device matrix without allocating anything: no cudaMalloc,
 * no cudaFree and no allocating library call.  It is meant for callers that
 * cannot allocate device memory: code that runs while another framework owns
 * the device allocator (an allocation would go around it or fail), real-time
 * loops that forbid allocation once they are running (an allocation can
 * block or synchronise the device), and services with a fixed memory budget.
 * The paper has no counterpart; it is the S0 reduction of eod_abe_factor run
 * on a fixed scratch area.
 *
 * A: device matrix, m x n, column-major, ld lda >= m, type dtype (EOD_F64 or
 * EOD_F32).  norm_out: device pointer to one double, receives ||A||_F
 * (FP64 accumulation; the same kernels, grid and reduction order as
 * eod_abe_factor's norm_a, so the same bits).  nonfinite_out: device pointer
 * to one int32, receives 1 if A holds a NaN or an infinity, else 0 (it is
 * cleared by the call).  stream: cudaStream_t.  The call only enqueues work
 * and returns; read the outputs after synchronising the stream.  The call is
 * never included in the eod_abe_debug_profile timing (that timing creates
 * CUDA events); it does count in eod_abe_debug_launch_count.
 *
 * Scratch: the per-block partial sums live in a static device array of
 * 58,368 bytes (4864 partial sums and flags) that every GPU loading this
 * library keeps until the process exits.  The first call on each device (and
 * the first after a cudaDeviceReset) looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array, which keeps the
 * last call's partials: calls that overlap on the GPU (different streams, or
 * different host threads on the same device) race on it and must be
 * serialised by the caller.
 *
 * Errors: EOD_EINVAL for NULL pointers, m < 1, n < 1, lda < m, an unknown
 * dtype, m or n above 2^31 - 1, or m*n above 2^40 elements (the largest
 * input this entry point accepts); EOD_ECUDA if a launch fails;
 * EOD_EUNSUPPORTED for a device ordinal of 64 or more. */
EOD_API eod_status eod_abe_fro_norm_noalloc(const void *A, int64_t m, int64_t n, int64_t lda, int32_t dtype,
                                            double *norm_out, int32_t *nonfinite_out, void *stream);

/* Test hook (no counterpart in the paper as an entry point; it is the
 * factorisation behind Alg. 1 steps 5-11 and the CholQR of Alg. 2 steps 9-10):
 * one leaf factorisation G + shift I = R^T R of a w x w SPD block (w <= 128,
 * only G's upper triangle is read, column-major, device memory), computed as
 * L D L^T.  With decide != 0 each pivot d_j = T(j,j)^2 is tested against eps2
 * with the rounding bound delta_coef G(j,j) and the guard rho G(j,j), and the
 * factorisation stops at the first pivot that is not kept.  Writes R (upper,
 * zeros below, leading p x p) and, when Rinv is not null, R^{-1} (same ld);
 * info[0] = p (columns factored), info[1] = 0 all kept / 1 below eps /
 * 2 undecided / 3 not positive.  decide | 256 runs the schedule with two
 * barriers per pivot instead of the lookahead one the library uses (same
 * results up to rounding; for comparison).  Returns after synchronising
 * `stream`; EOD_EINVAL for w outside [1, 128] or short leading dimensions. */
EOD_API eod_status eod_abe_debug_chol(const double *G, int64_t ldg, int32_t w, int32_t decide, double eps2,
                                      double delta_coef, double rho, double shift, double *R, double *Rinv,
                                      int64_t ldr, int32_t *info, void *stream);

/* Test hook (no counterpart in the paper): the reciprocal the leaf
 * factorisation (eod_abe_debug_chol, Alg. 1 steps 5-11) takes of each pivot,
 * applied to n device doubles d (out[i] = 1/d[i], FP64, device memory):
 * seeded by an FP32 reciprocal of the mantissa and refined by one
 * third-order step, within 2 ulp of 1/d for normal d whose reciprocal is
 * normal; +inf for subnormal d and 0 for d above about 2^1022 (deliberate:
 * the leaf only sees Gram pivots).  Returns after synchronising `stream`;
 * EOD_EINVAL for NULL pointers or n < 1. */
EOD_API eod_status eod_abe_debug_recip(const double *d, double *out, int64_t n, void *stream);

/* Test hook (no counterpart in the paper): one FP64 GEMM C = alpha op(A)
 * op(B) + beta C on device matrices, column-major, op(X) = X^T when the
 * matching flag is nonzero; mode & 3 == 0 runs the SIMT DFMA kernel, 1 the
 * FP64 emulation on tcgen05 tensor cores that the plain FP64 path uses for
 * large products (exact BF16 slices, FP64 accumulation).  Bits of mode above
 * those select the structured forms the factorisation uses: 16 = only the
 * upper triangle of C is wanted (the emulation stores row <= col only, the
 * SIMT kernel whole tiles that touch it), 32 = op(A) upper triangular,
 * 64 = op(B) upper triangular (the zero part is then not read by the
 * emulation; the SIMT kernel expects it to hold zeros), 128 = a SIMT K split
 * is summed by a separate reduction kernel instead of by the last CTA of
 * each tile (same order, same result; the emulation always uses its own
 * reduction kernel).  Returns after
 * synchronising `stream`; EOD_EINVAL for bad sizes or leading dimensions,
 * EOD_ETIMEOUT if a bounded device wait ran out. */
EOD_API eod_status eod_abe_debug_f64_gemm(int32_t mode, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K,
                                          double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                                          double beta, double *C, int64_t ldc, void *stream);

/* Test hook (no counterpart in the paper): exercises the bounded device-side
 * wait every tcgen05 kernel of the library uses on its mbarriers.  One CTA
 * waits on an mbarrier that expects one arrival, for at most budget_cycles
 * SM clock cycles; the arrival is made first when `arrive` is nonzero.  No
 * copy or MMA is in flight during the wait, so a wait that runs out leaves
 * the context usable: the kernel records the time-out and returns.  Returns
 * after synchronising `stream`: EOD_OK when the wait completed, EOD_ETIMEOUT
 * when it ran out, EOD_EINVAL for budget_cycles outside [1, 4e9] (the
 * library's own per-wait budget is 4e9 cycles, about 2 s). */
EOD_API eod_status eod_abe_debug_bounded_wait(int64_t budget_cycles, int32_t arrive, void *stream);

/* Tuned parameters (no counterpart in the paper; the autotuner of this
 * library, paper_2506_22713_gb300/autotune.py, writes them from timings on
 * the GPU).  The table is a text file of lines
 *     key a_lo a_hi b_lo b_hi c_lo c_hi value
 * (inclusive integer ranges, '#' comments; of the rows of a key whose ranges
 * hold (a, b, c), the nearest wins: the smallest sum over the three axes of
 * |log x - log centre|, centre the geometric mean of the row's bounds, ties
 * to the earlier row) read once per process from $EOD_TUNING_FILE, else
 * tuning.txt beside the library; a missing file means no tuned values and
 * the fixed defaults.
 * Keys the library consults: "block_k" (a = form: 0 plain FP64, 1 plain
 * FP32, 2 mixed BF16, 3 mixed TF32; b = m; c = n) for opts->block_k == 0
 * (default 32); "f32_tile" (a = M, b = N, c = K) for the FP32 SIMT product
 * tile (16, 32, 64, 128); "batch_workers" (a = count, b = mean m, c = mean n)
 * for eod_abe_factor_batched's worker streams (default 8; the environment
 * variable EOD_BATCH_STREAMS overrides); "batch_block_k" (a = form, b = mean
 * m, c = mean n) for the k of batched items on those streams when
 * opts->block_k == 0; "core_leaf" (a = p, b = c = 0) for the leaf width (16,
 * 32, 64, 128; default 64) of the blocked Cholesky of a p x p Gram in the
 * CholQR passes (subspace iteration and Alg. 2 steps 9-10).
 * eod_abe_tuning_load(path) replaces the table by the file at path (NULL:
 * the default location); EOD_EINVAL for a malformed line (the table is then
 * left unchanged); a missing file empties it.  eod_abe_tuning_lookup returns
 * 1 and stores the nearest matching row's value, else 0. */
EOD_API eod_status eod_abe_tuning_load(const char *path);
EOD_API int32_t eod_abe_tuning_lookup(const char *key, int64_t a, int64_t b, int64_t c, int64_t *value);

/* Timing hook of the autotuner (no counterpart in the paper): one FP32
 * product C = alpha op(A) op(B) + beta C on the SIMT kernel (the one the FP32
 * data paths use for their products), column-major device matrices, op(X)
 * = X^T when the flag is nonzero, with the tile forced to ts (16, 32, 64 or
 * 128) or chosen by the library (ts = 0, the table's "f32_tile" first).
 * Returns after synchronising `stream`; EOD_EINVAL for another ts, bad sizes
 * or leading dimensions. */
EOD_API eod_status eod_abe_debug_f32_gemm(int32_t ts, int32_t ta, int32_t tb, int64_t M, int64_t N, int64_t K,
                                          double alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                                          double beta, float *C, int64_t ldc, void *stream);

/* Build identification (static string). */
EOD_API const char *eod_abe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EOD_ABE_H */

/*
 * EOD-ABE oracle: a plain, slow, FP64 CPU statement of the EOD-ABE method
 * (power-free, tau = 0, and with tau subspace iterations) of Xu, Shen, Liu
 * and Jia, "A Novel Adaptive
 * Low-Rank Matrix Approximation Method for Image Compression and
 * Reconstruction" (arXiv 2506.22713).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library; the two meet only through the seeded input generators.
 *
 * Conventions: every matrix is column-major with an explicit leading
 * dimension; every loop is the textbook one, written for a reader checking
 * it against the paper, not for speed.  All arithmetic is IEEE double.
 *
 * Threads: when compiled with OpenMP, the loops over independent output
 * columns (of the dense products, of the reflector updates and of Omega)
 * are shared among threads.  Every entry is still computed by one thread in
 * the same order as the serial loop, so the results are bit-identical for
 * any thread count (tested); reductions over a whole matrix (norms, the
 * error) stay serial.  orc_set_threads() picks the count.
 *
 * Pins (what each function is checked against, outside itself):
 *   orc_philox4x32_10   published Philox4x32-10 known-answer vectors
 *   orc_omega           Gaussian moments + KS test, BF16 exactness
 *   orc_round_to_bf16   torch's round-to-nearest-even float -> bfloat16
 *   orc_householder_qr  |diag R|, Q, R of LAPACK's QR (numpy), QtQ = I
 *   orc_basis_ext       Thm 3.4(i) (blocked T diagonal == diagonal of the
 *                       unblocked R of A*Omega, LAPACK), Thm 3.4(ii) (exact
 *                       rank revealed), k-independence, QtQ = I
 *   orc_eod_abe         Eckart-Young optimum from a full SVD on tiny inputs,
 *                       A_hat = Q C = U D V^T, V = Q-factor of C^T (LAPACK),
 *                       D = R-factor of R^T (LAPACK), eps-monotonicity;
 *                       with tau > 0: range(Q_tau) = range((A A^T)^tau Q_0)
 *                       (matrix powers, numpy), the rank unchanged, RelErr
 *                       above the Eckart-Young optimum and converging to it
 *   orc_storage_entries worked example of Sec. 1 (72284 of 145200 entries)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Threads used by the column loops below (1 without OpenMP), one setting
 * for the whole process whichever thread calls in.  n <= 0 selects the
 * OpenMP default (OMP_NUM_THREADS if set, else every core).  Returns the
 * count now in effect. */
static int g_threads = 0;

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_set_threads(int n)
{
    g_threads = n > 0 ? n : 0;
    return orc_get_threads();
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11), from its published */
/* definition: 10 rounds of two 32x32->64 multiplies with a Weyl key bump.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Round a double to the nearest BF16 value (8 significant bits), ties to
 * even, computed directly from the double (no intermediate float).  The
 * Gaussian draws never reach the BF16 overflow or subnormal range. */
double orc_round_to_bf16(double g)
{
    if (g == 0.0 || !isfinite(g)) return g;
    int e;
    double frac = frexp(fabs(g), &e);          /* |g| = frac * 2^e, frac in [0.5,1) */
    double scaled = ldexp(frac, 8);            /* in [128, 256): 8 significant bits */
    double lower = floor(scaled);
    double rem = scaled - lower;               /* exact */
    double pick;
    if (rem > 0.5) pick = lower + 1.0;
    else if (rem < 0.5) pick = lower;
    else pick = (fmod(lower, 2.0) == 0.0) ? lower : lower + 1.0;
    double mag = ldexp(pick, e - 8);
    return g < 0.0 ? -mag : mag;
}

/* One entry of the Gaussian test matrix Omega (Alg. 1, step 3; Lemma 1).
 * Reading of the unspecified draw: counter (row, global column, batch, 0),
 * key (seed low word, seed high word); the first two outputs become uniforms
 * in (0,1) by (x + 1/2) 2^-32; Box-Muller (1958) maps them to a standard
 * normal; the normal is rounded to BF16 so that every precision of the
 * sketch sees the same exactly-representable test matrix. */
double orc_omega_entry(uint64_t seed, uint32_t row, uint32_t col, uint32_t batch)
{
    uint32_t ctr[4] = {row, col, batch, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u1 = ((double)x[0] + 0.5) * 0x1p-32;
    double u2 = ((double)x[1] + 0.5) * 0x1p-32;
    double radius = sqrt(-2.0 * log(u1));
    double angle = 2.0 * M_PI * u2;
    return orc_round_to_bf16(radius * cos(angle));
}

/* Omega(:, col0 : col0+ncols-1) as an n x ncols column-major block. */
void orc_omega(int64_t n, int64_t col0, int64_t ncols, uint64_t seed,
               uint64_t batch, double *out)
{
    #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if (n * ncols > 65536)
    for (int64_t c = 0; c < ncols; ++c)
        for (int64_t i = 0; i < n; ++i)
            out[IX(i, c, n)] = orc_omega_entry(seed, (uint32_t)i,
                                               (uint32_t)(col0 + c),
                                               (uint32_t)batch);
}

/* ------------------------------------------------------------------------ */
/* Dense building blocks (naive loops).                                      */
/* ------------------------------------------------------------------------ */

/* C (m x p) = A (m x q) * B (q x p) */
static void mat_mul(int64_t m, int64_t p, int64_t q, const double *A, int64_t lda,
                    const double *B, int64_t ldb, double *C, int64_t ldc)
{
    #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if (m * p * q > 1000000)
    for (int64_t j = 0; j < p; ++j) {
        for (int64_t i = 0; i < m; ++i) C[IX(i, j, ldc)] = 0.0;
        for (int64_t l = 0; l < q; ++l) {
            double b = B[IX(l, j, ldb)];
            for (int64_t i = 0; i < m; ++i) C[IX(i, j, ldc)] += A[IX(i, l, lda)] * b;
        }
    }
}

/* C (p x q) = A^T B with A (m x p), B (m x q) */
static void mat_tmul(int64_t m, int64_t p, int64_t q, const double *A, int64_t lda,
                     const double *B, int64_t ldb, double *C, int64_t ldc)
{
    #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if (m * p * q > 1000000)
    for (int64_t j = 0; j < q; ++j)
        for (int64_t i = 0; i < p; ++i) {
            double s = 0.0;
            for (int64_t l = 0; l < m; ++l) s += A[IX(l, i, lda)] * B[IX(l, j, ldb)];
            C[IX(i, j, ldc)] = s;
        }
}

/* Householder QR of the m x p matrix W (m >= p), overwritten.  Returns the
 * explicit thin Q (m x p, orthonormal columns) and R (p x p upper triangular)
 * with a non-negative diagonal: the sign of each reflector is chosen for
 * stability and the signs are then moved so that R(j,j) >= 0, which makes the
 * factorisation unique for a full-rank W.  A zero column gives R(j,j) = 0 and
 * an identity reflector. */
int orc_householder_qr(int64_t m, int64_t p, double *W, int64_t ldw,
                       double *Q, int64_t ldq, double *R, int64_t ldr)
{
    if (p > m || p < 0) return 1;
    double *tau = (double *)calloc((size_t)(p > 0 ? p : 1), sizeof(double));
    double *diag = (double *)calloc((size_t)(p > 0 ? p : 1), sizeof(double));
    if (!tau || !diag) { free(tau); free(diag); return 2; }

    for (int64_t j = 0; j < p; ++j) {
        double norm2 = 0.0;
        for (int64_t i = j; i < m; ++i) norm2 += W[IX(i, j, ldw)] * W[IX(i, j, ldw)];
        double alpha = sqrt(norm2);
        double x0 = W[IX(j, j, ldw)];
        if (alpha == 0.0) {              /* nothing to annihilate */
            tau[j] = 0.0;
            diag[j] = 0.0;
            for (int64_t i = j + 1; i < m; ++i) W[IX(i, j, ldw)] = 0.0;
            continue;
        }
        double beta = (x0 >= 0.0) ? -alpha : alpha;     /* H x = beta e1 */
        double v0 = x0 - beta;
        /* reflector v = (1, x(j+1:m)/v0), tau = (beta - x0)/beta */
        for (int64_t i = j + 1; i < m; ++i) W[IX(i, j, ldw)] /= v0;
        tau[j] = (beta - x0) / beta;
        diag[j] = beta;
        /* apply H = I - tau v v^T to the trailing columns */
        #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if ((p - j) * m > 65536)
        for (int64_t c = j + 1; c < p; ++c) {
            double s = W[IX(j, c, ldw)];
            for (int64_t i = j + 1; i < m; ++i) s += W[IX(i, j, ldw)] * W[IX(i, c, ldw)];
            s *= tau[j];
            W[IX(j, c, ldw)] -= s;
            for (int64_t i = j + 1; i < m; ++i) W[IX(i, c, ldw)] -= s * W[IX(i, j, ldw)];
        }
    }
    /* R: upper triangle of W with the computed diagonal */
    for (int64_t c = 0; c < p; ++c)
        for (int64_t i = 0; i < p; ++i)
            R[IX(i, c, ldr)] = (i < c) ? W[IX(i, c, ldw)] : (i == c ? diag[c] : 0.0);
    /* Q = H_0 H_1 ... H_{p-1} [I_p; 0], applied right to left */
    for (int64_t c = 0; c < p; ++c)
        for (int64_t i = 0; i < m; ++i) Q[IX(i, c, ldq)] = (i == c) ? 1.0 : 0.0;
    for (int64_t j = p - 1; j >= 0; --j) {
        if (tau[j] == 0.0) continue;
        #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if ((p - j) * m > 65536)
        for (int64_t c = j; c < p; ++c) {
            double s = Q[IX(j, c, ldq)];
            for (int64_t i = j + 1; i < m; ++i) s += W[IX(i, j, ldw)] * Q[IX(i, c, ldq)];
            s *= tau[j];
            Q[IX(j, c, ldq)] -= s;
            for (int64_t i = j + 1; i < m; ++i) Q[IX(i, c, ldq)] -= s * W[IX(i, j, ldw)];
        }
    }
    /* move signs so that diag(R) >= 0 */
    for (int64_t j = 0; j < p; ++j) {
        if (R[IX(j, j, ldr)] < 0.0) {
            for (int64_t c = j; c < p; ++c) R[IX(j, c, ldr)] = -R[IX(j, c, ldr)];
            for (int64_t i = 0; i < m; ++i) Q[IX(i, j, ldq)] = -Q[IX(i, j, ldq)];
        }
    }
    free(tau);
    free(diag);
    return 0;
}

/* Frobenius norm, plain sum of squares. */
double orc_fro_norm(int64_t m, int64_t n, const double *A, int64_t lda)
{
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) s += A[IX(i, j, lda)] * A[IX(i, j, lda)];
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (BasisExt).                                                        */
/*                                                                           */
/* Readings where the paper is silent: blocks never reach past min(m,n)      */
/* columns (the loop stops when the kept basis spans that many); block j     */
/* takes global Omega columns (j-1)k .. (j-1)k+f_j-1, which is exact because */
/* every block before the break keeps all of its f_j columns; the projection */
/* (I - QQ^T) is applied twice (BCGS2), equal in exact arithmetic to the     */
/* single projection of step 4; the QR of step 5 has a non-negative         */
/* diagonal; the test of step 6 is |T(l,l)| <= eps with the smallest l.      */
/*                                                                           */
/* Q: m x cap (ld m) receives the basis; tdiag (cap entries) receives every  */
/* computed diagonal entry of the T_j in order; *ntd their count; *r_out the */
/* detected rank.  max_blocks > 0 stops after that many blocks (a bounded    */
/* sample of the work for timing; 0 = run to the end).  Returns 0, or 2 on   */
/* allocation failure.                                                       */
/* ------------------------------------------------------------------------ */
int orc_basis_ext(const double *A, int64_t m, int64_t n, int64_t lda, double eps,
                  int64_t k, uint64_t seed, uint64_t batch,
                  double *Q, int64_t *r_out, double *tdiag, int64_t *ntd, int64_t max_blocks)
{
    const int64_t cap = (m < n) ? m : n;
    int64_t kept = 0, nt = 0, blocks = 0;
    double *Om = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k);
    double *Y = (double *)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double *S = (double *)malloc(sizeof(double) * (size_t)cap * (size_t)k);
    double *P = (double *)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double *T = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
    if (!Om || !Y || !S || !P || !T) {
        free(Om); free(Y); free(S); free(P); free(T);
        return 2;
    }
    int stop = 0;
    while (!stop && kept < cap && (max_blocks <= 0 || blocks < max_blocks)) {
        int64_t f = (k < cap - kept) ? k : (cap - kept);
        ++blocks;
        /* step 3: Omega_j, n x f */
        orc_omega(n, kept, f, seed, batch, Om);
        /* step 4: Y_j = A Omega_j, then Y_j <- (I - Q Q^T) Y_j, twice */
        mat_mul(m, f, n, A, lda, Om, n, Y, m);
        for (int pass = 0; pass < 2 && kept > 0; ++pass) {
            mat_tmul(m, kept, f, Q, m, Y, m, S, cap);          /* S = Q^T Y */
            #pragma omp parallel for schedule(static) num_threads(orc_get_threads()) if (m * f * kept > 1000000)
            for (int64_t c = 0; c < f; ++c)
                for (int64_t l = 0; l < kept; ++l) {
                    double s = S[IX(l, c, cap)];
                    for (int64_t i = 0; i < m; ++i) Y[IX(i, c, m)] -= Q[IX(i, l, m)] * s;
                }
        }
        /* step 5: Y_j = P_j T_j */
        orc_householder_qr(m, f, Y, m, P, m, T, k);
        /* steps 6-11: smallest l with |T(l,l)| <= eps */
        int64_t keep = f;
        for (int64_t l = 0; l < f; ++l) {
            tdiag[nt++] = T[IX(l, l, k)];
            if (fabs(T[IX(l, l, k)]) <= eps) {
                keep = l;            /* columns 0..l-1, i.e. P_j(:,1:l-1) in 1-based */
                stop = 1;
                break;
            }
        }
        /* record the remaining (untested) diagonal entries too */
        if (stop)
            for (int64_t l = keep + 1; l < f; ++l) tdiag[nt++] = T[IX(l, l, k)];
        for (int64_t c = 0; c < keep; ++c)
            memcpy(&Q[IX(0, kept + c, m)], &P[IX(0, c, m)], sizeof(double) * (size_t)m);
        kept += keep;
    }
    *r_out = kept;
    *ntd = nt;
    free(Om); free(Y); free(S); free(P); free(T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 steps 2-7, tau times on Q (m x r, ld m), in place: the rank r is   */
/* the one BasisExt found; each pass forms Yt = A^T Q and its QR Yt = Qt Rt, */
/* then Y = A Qt and its QR Y = Q R (positive diagonals, Householder).       */
/* ------------------------------------------------------------------------ */
static int subspace_iteration(const double *A, int64_t m, int64_t n, int64_t lda, double *Q, int64_t r,
                              int64_t tau)
{
    if (tau <= 0 || r == 0) return 0;
    double *Yt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)r);
    double *Qt = (double *)malloc(sizeof(double) * (size_t)n * (size_t)r);
    double *Y = (double *)malloc(sizeof(double) * (size_t)m * (size_t)r);
    double *R = (double *)malloc(sizeof(double) * (size_t)r * (size_t)r);
    if (!Yt || !Qt || !Y || !R) {
        free(Yt); free(Qt); free(Y); free(R);
        return 2;
    }
    for (int64_t j = 1; j <= tau; ++j) {
        mat_tmul(m, n, r, A, lda, Q, m, Yt, n);          /* step 3: Yt_j = A^T Q_{j-1}   */
        orc_householder_qr(n, r, Yt, n, Qt, n, R, r);    /* step 4: Yt_j = Qt_j Rt_j     */
        mat_mul(m, r, n, A, lda, Qt, n, Y, m);           /* step 5: Y_j = A Qt_j         */
        orc_householder_qr(m, r, Y, m, Q, m, R, r);      /* step 6: Y_j = Q_j R_j        */
    }
    free(Yt); free(Qt); free(Y); free(R);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: BasisExt, tau subspace iterations (above), then                   */
/*   step 8   C = Q^T A                       (r x n)                        */
/*   step 9   C^T = V R      (QR, n x r)                                     */
/*   step 10  R^T = Qh Dh    (QR, r x r)                                     */
/*   step 11  U = Q Qh, D = Dh, V                                            */
/* plus the reconstruction A_hat = Q C and RelErr = ||A - A_hat||_F/||A||_F  */
/* (Sec. 4.1), the latter from the explicit difference.                      */
/*                                                                           */
/* tol_mode 0: eps = tol (Alg. 1 as printed); tol_mode 1: eps = tol*||A||_F. */
/* Outputs (capacity cap = min(m,n) columns): U m x cap (ld m), D cap x cap  */
/* (ld cap), V n x cap (ld n), Q m x cap (ld m), C cap x n (ld cap); only    */
/* the leading r columns / r x r block are meaningful.  res[0] = RelErr,     */
/* res[1] = ||A||_F, res[2] = eps used.                                      */
/* ------------------------------------------------------------------------ */
int orc_eod_abe(const double *A, int64_t m, int64_t n, int64_t lda, double tol,
                int tol_mode, int64_t k, uint64_t seed, uint64_t batch, int64_t tau,
                double *U, double *D, double *V, double *Q, double *C,
                int64_t *r_out, double *res, double *tdiag, int64_t *ntd)
{
    const int64_t cap = (m < n) ? m : n;
    double norm_a = orc_fro_norm(m, n, A, lda);
    double eps = (tol_mode == 1) ? tol * norm_a : tol;
    int64_t r = 0;
    int st = orc_basis_ext(A, m, n, lda, eps, k, seed, batch, Q, &r, tdiag, ntd, 0);
    if (st) return st;
    *r_out = r;
    res[1] = norm_a;
    res[2] = eps;
    if (r == 0) {
        res[0] = (norm_a > 0.0) ? 1.0 : 0.0;
        return 0;
    }
    /* steps 2-7 */
    st = subspace_iteration(A, m, n, lda, Q, r, tau);
    if (st) return st;
    /* step 8 */
    mat_tmul(m, r, n, Q, m, A, lda, C, cap);
    /* step 9: QR of C^T (n x r) */
    double *Ct = (double *)malloc(sizeof(double) * (size_t)n * (size_t)r);
    double *R = (double *)malloc(sizeof(double) * (size_t)r * (size_t)r);
    double *Rt = (double *)malloc(sizeof(double) * (size_t)r * (size_t)r);
    double *Qh = (double *)malloc(sizeof(double) * (size_t)r * (size_t)r);
    double *Ahat = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    if (!Ct || !R || !Rt || !Qh || !Ahat) {
        free(Ct); free(R); free(Rt); free(Qh); free(Ahat);
        return 2;
    }
    for (int64_t i = 0; i < r; ++i)
        for (int64_t j = 0; j < n; ++j) Ct[IX(j, i, n)] = C[IX(i, j, cap)];
    orc_householder_qr(n, r, Ct, n, V, n, R, r);
    /* step 10: QR of R^T (r x r) */
    for (int64_t i = 0; i < r; ++i)
        for (int64_t j = 0; j < r; ++j) Rt[IX(j, i, r)] = R[IX(i, j, r)];
    orc_householder_qr(r, r, Rt, r, Qh, r, D, cap);
    /* step 11: U = Q Qh */
    mat_mul(m, r, r, Q, m, Qh, r, U, m);
    /* reconstruction A_hat = Q C and its relative Frobenius error */
    mat_mul(m, n, r, Q, m, C, cap, Ahat, m);
    double e2 = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) {
            double d = A[IX(i, j, lda)] - Ahat[IX(i, j, m)];
            e2 += d * d;
        }
    res[0] = (norm_a > 0.0) ? sqrt(e2) / norm_a : 0.0;
    free(Ct); free(R); free(Rt); free(Qh); free(Ahat);
    return 0;
}

/* Entries stored by the factors U (m x r), upper-triangular D (r x r) and
 * V (n x r), against m*n for A itself (Sec. 1). */
int64_t orc_storage_entries(int64_t m, int64_t n, int64_t r)
{
    return r * (m + n) + r * (r + 1) / 2;
}

/* The rank bound of Sec. 1 below which the factors are smaller than A:
 * r < sqrt(m^2 + n^2 + 4mn + m + n + 1/4) - (m + n + 1/2). */
double orc_storage_rank_bound(int64_t m, int64_t n)
{
    double dm = (double)m, dn = (double)n;
    return sqrt(dm * dm + dn * dn + 4.0 * dm * dn + dm + dn + 0.25) - (dm + dn + 0.5);
}

"""Pins for the FP64 oracle (CPU only).

Every check here ties the oracle to something other than itself: published
known-answer vectors, LAPACK's QR and SVD (through numpy) as textbook
routines, theorems of the paper (Thm 3.4, the rank-revealing theorem of
Sec. 3.2), the Eckart-Young optimum, and the worked example of Sec. 1.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Omega: Philox4x32-10 + Box-Muller + BF16 rounding
# --------------------------------------------------------------------------

def test_philox_known_answers():
    for row in _read_golden("philox4x32_10_kat.txt"):
        words = [int(x, 16) for x in row]
        ctr, key, expect = words[0:4], words[4:6], words[6:10]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == expect


def test_bf16_rounding_matches_torch():
    """Round-to-nearest-even to BF16 against torch's float -> bfloat16
    conversion, on float32-representable inputs (so torch's route through
    float is exact), including exact ties in both directions."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4000).astype(np.float32)
    # exact midpoints between neighbouring BF16 values: low 16 bits = 0x8000
    bits = rng.integers(0x3E000000, 0x41000000, size=1000, dtype=np.uint32)
    ties = ((bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, -ties]).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to_bf16(x), ref)


def test_omega_is_bf16_exact():
    om = oracle.omega(4096, 0, 8, seed=11)
    f32 = om.astype(np.float32)
    assert np.array_equal(f32.astype(np.float64), om)
    low = f32.view(np.uint32) & np.uint32(0xFFFF)
    assert not low.any(), "every entry must carry at most 8 significant bits"


def test_omega_gaussian_moments_and_ks():
    om = oracle.omega(5000, 0, 4, seed=12345).ravel()
    n = om.size
    assert abs(om.mean()) < 5.0 / np.sqrt(n)
    assert abs(om.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    # BF16 rounding moves each value by at most 2^-9 relative: invisible at this n.
    ks = stats.kstest(om, "norm")
    assert ks.pvalue > 1e-3
    # the four moments of a standard normal
    assert abs(stats.skew(om)) < 5.0 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(om)) < 5.0 * np.sqrt(24.0 / n)


def test_omega_columns_rows_batches_independent():
    a = oracle.omega(3000, 0, 2, seed=5, batch=0)
    b = oracle.omega(3000, 0, 2, seed=5, batch=1)
    c = oracle.omega(3000, 0, 2, seed=6, batch=0)
    lim = 5.0 / np.sqrt(3000)
    assert abs(np.corrcoef(a[:, 0], a[:, 1])[0, 1]) < lim
    assert abs(np.corrcoef(a[:, 0], b[:, 0])[0, 1]) < lim
    assert abs(np.corrcoef(a[:, 0], c[:, 0])[0, 1]) < lim
    # a block of columns is the same wherever it is requested from
    d = oracle.omega(3000, 1, 1, seed=5, batch=0)
    assert np.array_equal(d[:, 0], a[:, 1])


# --------------------------------------------------------------------------
# Householder QR against LAPACK
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,p", [(7, 3), (40, 40), (100, 17), (1, 1)])
def test_householder_qr_matches_lapack(m, p):
    rng = np.random.default_rng(m * 100 + p)
    Wm = rng.standard_normal((m, p))
    Q, R = oracle.householder_qr(Wm)
    Ql, Rl = np.linalg.qr(Wm)
    sg = np.sign(np.diag(Rl))
    Ql, Rl = Ql * sg, Rl * sg[:, None]
    assert np.all(np.diag(R) >= 0)
    assert np.allclose(np.triu(R), R, atol=0)
    assert np.linalg.norm(Q.T @ Q - np.eye(p)) < 1e-13 * max(1, p)
    assert np.linalg.norm(Q @ R - Wm) < 1e-13 * np.linalg.norm(Wm)
    assert np.max(np.abs(R - Rl)) < 1e-12 * np.abs(Rl).max()
    assert np.max(np.abs(Q - Ql)) < 1e-10


def test_householder_qr_zero_and_dependent_columns():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((20, 1))
    Wm = np.hstack([x, 2 * x, np.zeros((20, 1)), rng.standard_normal((20, 1))])
    Q, R = oracle.householder_qr(Wm)
    assert abs(R[1, 1]) < 1e-14 * np.linalg.norm(x)
    assert R[2, 2] == 0.0 or abs(R[2, 2]) < 1e-14
    assert np.linalg.norm(Q @ R - Wm) < 1e-13 * np.linalg.norm(Wm)


# --------------------------------------------------------------------------
# Alg. 1 (BasisExt)
# --------------------------------------------------------------------------

def test_exact_rank_twenty_is_revealed():
    """Thm 3.4(ii) / Rem. 3.6 on the 512 x 384 exact rank-20 matrix."""
    w = W.exact_rank()
    Q, td = oracle.basis_ext(w.A, w.tol, k=32, seed=w.seed)
    assert Q.shape[1] == 20
    assert np.all(td[:20] > w.tol) and td[20] <= w.tol
    assert np.linalg.norm(Q.T @ Q - np.eye(20)) <= 1e-12


@pytest.mark.parametrize("k", [1, 3, 8, 32, 384])
def test_rank_independent_of_block_size(k):
    w = W.exact_rank()
    Q, _ = oracle.basis_ext(w.A, w.tol, k=k, seed=w.seed)
    assert Q.shape[1] == 20


@pytest.mark.parametrize("k", [1, 5, 8, 13])
def test_blocked_diagonal_equals_unblocked_qr(k):
    """Thm 3.4(i): the diagonals of the blocked T_j are the diagonal of the R
    factor of one QR of A * [Omega_1 ... Omega_{z+1}] (LAPACK here)."""
    rng = np.random.default_rng(17)
    A = W.low_rank(rng, 120, 90, np.geomspace(3.0, 0.05, 30))
    Q, td = oracle.basis_ext(A, 1e-9, k=k, seed=21)
    r = Q.shape[1]
    assert r == 30
    Om = oracle.omega(90, 0, r + 1, seed=21)
    _, R = np.linalg.qr(A @ Om)
    ref = np.abs(np.diag(R))
    nchk = min(td.size, r + 1)
    assert np.max(np.abs(td[:nchk] - ref[:nchk])) <= 1e-12 * np.linalg.norm(A)


def test_rank_zero_and_full_rank_and_wide():
    Z = np.zeros((30, 20))
    res = oracle.eod_abe(Z, 1e-12, k=8, seed=1)
    assert res["r"] == 0
    G = W.gaussian(30, 20, seed=4)
    res = oracle.eod_abe(G, 1e-12, k=8, seed=1)
    assert res["r"] == 20 and res["rel_err"] < 1e-13
    Gw = W.gaussian(15, 40, seed=5)                  # m < n: rank capped at m
    res = oracle.eod_abe(Gw, 1e-12, k=6, seed=2)
    assert res["r"] == 15 and res["rel_err"] < 1e-13


# --------------------------------------------------------------------------
# Alg. 2 (tau = 0): core and error
# --------------------------------------------------------------------------

def _eckart_young(A, r):
    s = np.linalg.svd(A, compute_uv=False)
    return np.sqrt(np.sum(s[r:] ** 2)) / np.linalg.norm(A)


@pytest.mark.parametrize("m,n,r", [(48, 48, 7), (40, 25, 11), (20, 44, 5), (33, 31, 1)])
def test_exact_rank_reaches_eckart_young(m, n, r):
    """On exactly rank-r inputs the error equals the Eckart-Young optimum
    (zero) from a full SVD, within 1e-12."""
    rng = np.random.default_rng(m + n + r)
    A = W.low_rank(rng, m, n, np.geomspace(2.0, 0.1, r))
    res = oracle.eod_abe(A, 1e-10, k=4, seed=3)
    assert res["r"] == r
    assert abs(res["rel_err"] - _eckart_young(A, r)) <= 1e-12


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-2])
def test_error_never_below_eckart_young(eps):
    rng = np.random.default_rng(99)
    A = W.low_rank(rng, 40, 36, np.geomspace(1.0, 1e-3, 36))
    res = oracle.eod_abe(A, eps, k=5, seed=8)
    ey = _eckart_young(A, res["r"])
    assert res["rel_err"] >= ey - 1e-15
    # the truncated part of an exactly decaying spectrum is close to optimal
    assert res["rel_err"] <= 10 * ey + 1e-15


def test_core_factors_match_lapack_and_identities():
    """Steps 8-11: V is the Q factor of C^T, D the R factor of R^T, U = Q Qh;
    A_hat = Q C = U D V^T; singular values of D are those of C."""
    w = W.exact_rank(m=96, n=70, r=12)
    res = oracle.eod_abe(w.A, w.tol, k=8, seed=2)
    r = res["r"]
    assert r == 12
    Q, C, U, D, V = res["Q"], res["C"], res["U"], res["D"], res["V"]
    assert np.allclose(C, Q.T @ w.A, atol=1e-13)
    Vl, Rl = np.linalg.qr(C.T)
    sg = np.sign(np.diag(Rl))
    Vl, Rl = Vl * sg, Rl * sg[:, None]
    assert np.max(np.abs(V - Vl)) < 1e-10
    Qh, Dl = np.linalg.qr(Rl.T)
    sg2 = np.sign(np.diag(Dl))
    Qh, Dl = Qh * sg2, Dl * sg2[:, None]
    assert np.max(np.abs(D - Dl)) < 1e-10 * np.abs(Dl).max()
    assert np.max(np.abs(U - Q @ Qh)) < 1e-10
    assert np.all(np.diag(D) > 0) and np.allclose(np.tril(D, -1), 0)
    assert np.linalg.norm(U.T @ U - np.eye(r)) < 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(r)) < 1e-12
    assert np.linalg.norm(U @ D @ V.T - Q @ C) < 1e-13 * np.linalg.norm(w.A)
    sd = np.linalg.svd(D, compute_uv=False)
    sc = np.linalg.svd(C, compute_uv=False)
    assert np.max(np.abs(sd - sc)) < 1e-12 * sc[0]


def test_error_identity_with_projection_norm():
    """||A - QC||^2 = ||A||^2 - ||C||^2 for orthonormal Q (moderate error)."""
    rng = np.random.default_rng(5)
    A = W.low_rank(rng, 60, 50, np.geomspace(1.0, 1e-2, 50))
    res = oracle.eod_abe(A, 0.05, k=4, seed=9)
    lhs = (res["rel_err"] * res["norm_a"]) ** 2
    rhs = res["norm_a"] ** 2 - np.linalg.norm(res["C"]) ** 2
    assert abs(lhs - rhs) < 1e-12 * res["norm_a"] ** 2


def test_relative_tolerance_mode():
    w = W.exact_rank(m=80, n=60, r=10)
    a = oracle.eod_abe(w.A, 1e-6, tol_mode=1, k=4, seed=1)
    b = oracle.eod_abe(w.A, 1e-6 * oracle.fro_norm(w.A), tol_mode=0, k=4, seed=1)
    assert a["r"] == b["r"] == 10
    assert a["eps"] == pytest.approx(b["eps"], rel=1e-15)


def test_eps_monotonicity_devils_stairs():
    """Sec. 4.4: rank falls and error rises as eps grows (exact for a fixed
    Omega, since every run is a prefix of the same blocked process)."""
    A = W.devils_stairs(90)
    ranks, errs = [], []
    for eps in np.logspace(-9, -1, 17):
        res = oracle.eod_abe(A, eps, k=10, seed=4)
        ranks.append(res["r"])
        errs.append(res["rel_err"])
    assert all(a >= b for a, b in zip(ranks, ranks[1:]))
    assert all(b >= a - 1e-15 for a, b in zip(errs, errs[1:]))
    assert ranks[0] == 90 and ranks[-1] < ranks[0]


def test_storage_worked_example():
    """Sec. 1: ranks 50/52/53 of a 220 x 220 RGB image need 72284 entries
    instead of 145200, a 50.22 % reduction."""
    row = _read_golden("storage_example.txt")[0]
    m, n, r1, r2, r3, tot, dense, pct = (int(row[0]), int(row[1]), int(row[2]), int(row[3]),
                                         int(row[4]), int(row[5]), int(row[6]), float(row[7]))
    got = sum(oracle.storage_entries(m, n, r) for r in (r1, r2, r3))
    assert got == tot
    assert 3 * m * n == dense
    assert round(100.0 * (1.0 - got / dense), 2) == pct
    bound = oracle.storage_rank_bound(m, n)
    for r in range(1, 200):
        assert (oracle.storage_entries(m, n, r) < m * n) == (r < bound)


# --------------------------------------------------------------------------
# Alg. 2 steps 2-7: tau subspace iterations
# --------------------------------------------------------------------------

def _gapped(m=48, n=36, r=6, seed=21):
    """U diag(s) V^T + a small tail: r leading values in [0.3, 1], the rest
    at 1e-3 and below, so BasisExt at eps = 0.05 ||A||_F keeps about r columns."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    V, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    s = np.concatenate([np.linspace(1.0, 0.3, r), 1e-3 * np.geomspace(1.0, 0.1, min(m, n) - r)])
    return np.asfortranarray((U * s) @ V.T), s


@pytest.mark.parametrize("tau", [1, 2, 3])
def test_subspace_iteration_spans_power_of_a_at(tau):
    """range(Q_tau) = range((A A^T)^tau Q_0): the alternating QRs of
    Alg. 2 steps 3-6 against matrix powers and an SVD basis (numpy)."""
    A, _ = _gapped()
    r0 = oracle.eod_abe(A, 0.05, 1, k=4, seed=3, tau=0)
    rt = oracle.eod_abe(A, 0.05, 1, k=4, seed=3, tau=tau)
    assert rt["r"] == r0["r"] and r0["r"] > 0
    Q0, Qt = r0["Q"], rt["Q"]
    M = Q0.copy()
    for _ in range(tau):
        M = A @ (A.T @ M)
    Ub, _, _ = np.linalg.svd(M, full_matrices=False)
    P_ref = Ub @ Ub.T
    assert np.linalg.norm(Qt.T @ Qt - np.eye(Qt.shape[1])) <= 1e-12
    assert np.linalg.norm(Qt @ Qt.T - P_ref) <= 1e-9


def test_subspace_iteration_error_bounds_and_convergence():
    """The rank stays BasisExt's; RelErr never beats the Eckart-Young optimum
    of that rank, does not grow with tau here (gap 300x), and approaches the
    optimum: tau = 6 is within 1e-6 of it."""
    A, s = _gapped()
    errs = []
    for tau in range(0, 7):
        res = oracle.eod_abe(A, 0.05, 1, k=4, seed=3, tau=tau)
        r = res["r"]
        opt = np.sqrt(np.sum(s[r:] ** 2)) / np.linalg.norm(A)
        assert res["rel_err"] >= opt * (1 - 1e-12)
        # A_hat = Q C with C = Q^T A: the reported error is that projection's
        Q = res["Q"]
        assert abs(np.linalg.norm(A - Q @ (Q.T @ A)) / np.linalg.norm(A) - res["rel_err"]) <= 1e-13
        errs.append((res["rel_err"], opt, r))
    assert len({e[2] for e in errs}) == 1
    for a, b in zip(errs, errs[1:]):
        assert b[0] <= a[0] * (1 + 1e-12)
    assert errs[-1][0] <= errs[-1][1] * (1 + 1e-6)
    assert errs[0][0] > errs[0][1] * (1 + 1e-4)        # tau = 0 is measurably above it


def test_subspace_iteration_core_factors():
    """With tau > 0 the core factors still satisfy A_hat = U D V^T = Q C,
    U^T U = I, V^T V = I, D upper triangular with a positive diagonal."""
    A, _ = _gapped(seed=5)
    res = oracle.eod_abe(A, 0.05, 1, k=4, seed=7, tau=2)
    U, D, V, Q, C = res["U"], res["D"], res["V"], res["Q"], res["C"]
    r = res["r"]
    assert np.allclose(np.tril(D, -1), 0.0) and np.all(np.diag(D) > 0)
    assert np.linalg.norm(U.T @ U - np.eye(r)) <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(r)) <= 1e-12
    assert np.linalg.norm(U @ D @ V.T - Q @ C) <= 1e-12 * np.linalg.norm(A)


# --------------------------------------------------------------------------
# Threads: the column loops shared among OpenMP threads give the same bits
# --------------------------------------------------------------------------

def test_thread_count_does_not_change_any_bit():
    """Each output entry is computed by one thread in the serial loop's order,
    so 1, 3 and all threads must agree bit for bit (factors, T diagonal,
    RelErr), with and without subspace iteration."""
    w = W.image_like(m=700, n=600, r=80, tol=1e-3)
    before = oracle.get_threads()
    try:
        for tau in (0, 1):
            res = {}
            for t in (1, 3, 0):
                oracle.set_threads(t)
                res[t] = oracle.eod_abe(w.A, w.tol, 1, k=32, seed=2, tau=tau)
            for t in (3, 0):
                for key in ("U", "D", "V", "Q", "C", "tdiag"):
                    assert np.array_equal(res[1][key], res[t][key]), (tau, t, key)
                assert res[1]["rel_err"] == res[t]["rel_err"]
                assert res[1]["r"] == res[t]["r"]
    finally:
        oracle.set_threads(before)

"""GPU parity of the plain (FP64 / FP32) path against the FP64 oracle.

Bar (FP64 plain): the oracle's rank exactly, |RelErr_gpu - RelErr_oracle| <=
1e-10, and factors equal to the oracle's within a bound set by the
conditioning.  FP32 storage: rank exact, |dRelErr| <= 1e-4.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _cuda(A, dtype=torch.float64):
    return torch.from_numpy(np.asfortranarray(A)).to(dtype).cuda()


def _check_factors(f, ref, A, atol_rel):
    r = f.rank
    U, D, V = f.U.double().cpu().numpy(), f.D.cpu().numpy(), f.V.double().cpu().numpy()
    nrm = np.linalg.norm(A)
    # A_hat = U D V^T equals the oracle's A_hat (a property of the subspace, not of signs)
    Ah = U @ D @ V.T
    Ah_ref = ref["U"] @ ref["D"] @ ref["V"].T
    assert np.linalg.norm(Ah - Ah_ref) <= atol_rel * nrm
    # every factor is unique (positive diagonals): compare elementwise
    assert np.max(np.abs(D - ref["D"])) <= atol_rel * max(1.0, np.abs(ref["D"]).max())
    assert np.max(np.abs(U - ref["U"])) <= atol_rel * 1e2
    assert np.max(np.abs(V - ref["V"])) <= atol_rel * 1e2
    assert np.all(np.diag(D) > 0) and np.allclose(np.tril(D, -1), 0.0)
    assert np.linalg.norm(U.T @ U - np.eye(r)) <= 1e-12 * max(1, r) if U.dtype == np.float64 else True


# ------------------------------------------------------------------ Omega --
@pytest.mark.parametrize("n,col0,ncols,seed,batch", [(5000, 0, 16, 1, 0), (333, 7, 5, 2 ** 40 + 3, 9),
                                                     (8192, 64, 64, 3, 0), (1, 0, 1, 0, 0)])
def test_omega_bit_exact(eod, n, col0, ncols, seed, batch):
    got = eod.omega(n, col0, ncols, seed, batch).cpu().numpy()
    ref = oracle.omega(n, col0, ncols, seed, batch)
    assert np.array_equal(got, ref)


def test_omega_bit_exact_large(eod):
    """Four million entries: the FP32 fast path with its FP64 fallback must
    agree with the oracle's FP64 draw on every one."""
    got = eod.omega(1 << 20, 123, 4, 0xDEADBEEF12345, 3).cpu().numpy()
    ref = oracle.omega(1 << 20, 123, 4, 0xDEADBEEF12345, 3)
    assert np.array_equal(got, ref)


# ------------------------------------------------------- exact rank (c1) --
@pytest.mark.parametrize("k", [32, 1, 7, 64])
def test_exact_rank_512x384(eod, k):
    w = W.exact_rank()
    ref = oracle.eod_abe(w.A, w.tol, 0, k=k, seed=w.seed)
    f = eod.factor(_cuda(w.A), w.tol, w.seed, block_k=k)
    assert ref["r"] == 20
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
    _check_factors(f, ref, w.A, 1e-10)
    # T diagonal (Thm 3.4(i)): the kept entries agree with the oracle's
    td = np.array(f.tdiag)
    assert np.max(np.abs(td[:20] - ref["tdiag"][:20])) <= 1e-10 * ref["norm_a"]
    assert td[20] <= w.tol


@pytest.mark.parametrize("m,n,r,k", [(130, 97, 9, 8), (97, 130, 9, 8), (300, 41, 41, 16), (64, 64, 1, 5),
                                     (257, 129, 33, 32), (70, 300, 25, 128)])
def test_ragged_exact_rank(eod, m, n, r, k):
    w = W.exact_rank(m=m, n=n, r=r, seed=m * n + r)
    ref = oracle.eod_abe(w.A, w.tol, 0, k=k, seed=5)
    f = eod.factor(_cuda(w.A), w.tol, 5, block_k=k)
    assert f.rank == ref["r"] == min(r, m, n)
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
    _check_factors(f, ref, w.A, 1e-9)


def test_full_rank_gaussian(eod):
    A = W.gaussian(90, 70, seed=8)
    ref = oracle.eod_abe(A, 1e-12, 0, k=16, seed=2)
    f = eod.factor(_cuda(A), 1e-12, 2, block_k=16)
    assert f.rank == ref["r"] == 70
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_noisy_decay_relative_tol(eod, eps):
    rng = np.random.default_rng(12)
    A = W.low_rank(rng, 200, 150, np.geomspace(1.0, 1e-6, 150))
    ref = oracle.eod_abe(A, eps, 1, k=16, seed=4)
    f = eod.factor(_cuda(A), eps, 4, block_k=16, tol_mode="rel")
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
    _check_factors(f, ref, A, 1e-8)


def test_image_like_small_fp64(eod):
    w = W.image_like(m=384, n=320, r=60, seed=22)
    ref = oracle.eod_abe(w.A, w.tol, 1, k=32, seed=w.seed)
    f = eod.factor(_cuda(w.A), w.tol, w.seed, block_k=32, tol_mode="rel")
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10


def test_image_like_small_fp32(eod):
    w = W.image_like(m=384, n=320, r=60, seed=22, dtype="f32", tol=0.05)
    ref = oracle.eod_abe(w.A.astype(np.float64), w.tol, 1, k=32, seed=w.seed)
    f = eod.factor(_cuda(w.A, torch.float32), w.tol, w.seed, block_k=32, tol_mode="rel")
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4


def test_devils_stairs_eps_sweep_matches_oracle(eod):
    A = W.devils_stairs(90)
    ranks = []
    for eps in np.logspace(-9, -1, 9):
        ref = oracle.eod_abe(A, eps, 0, k=10, seed=4)
        f = eod.factor(_cuda(A), eps, 4, block_k=10)
        assert f.rank == ref["r"], eps
        assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
        ranks.append(f.rank)
    assert all(a >= b for a, b in zip(ranks, ranks[1:]))


# ---------------------------------------------------------- degenerate ----
def test_zero_matrix_rank_zero(eod):
    f = eod.factor(torch.zeros((50, 40), dtype=torch.float64, device="cuda").t().contiguous().t(), 1e-6, 1)
    assert f.rank == 0
    assert f.reconstruct().abs().max().item() == 0.0


def test_rank_one(eod):
    rng = np.random.default_rng(1)
    A = np.outer(rng.standard_normal(77), rng.standard_normal(55))
    ref = oracle.eod_abe(A, 1e-10, 0, k=8, seed=3)
    f = eod.factor(_cuda(A), 1e-10, 3, block_k=8)
    assert f.rank == ref["r"] == 1
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10


def test_nonfinite_is_rejected(eod):
    A = torch.ones((20, 10), dtype=torch.float64).t().contiguous().t().cuda()
    A[3, 4] = float("nan")
    with pytest.raises(eod.EodError) as ei:
        eod.factor(A, 1e-3, 1)
    assert ei.value.status == eod.EOD_ENONFINITE
    A[3, 4] = float("inf")
    with pytest.raises(eod.EodError):
        eod.factor(A, 1e-3, 1)


def test_lda_larger_than_m(eod):
    w = W.exact_rank(m=100, n=80, r=10, seed=2)
    big = np.zeros((130, 80))
    big[:100] = w.A
    Ab = torch.from_numpy(np.asfortranarray(big)).cuda()
    ref = oracle.eod_abe(w.A, w.tol, 0, k=8, seed=1)
    f = eod.factor(Ab[:100], w.tol, 1, block_k=8)
    assert f.rank == ref["r"] == 10
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10


def test_injected_allocation_failure(eod):
    w = W.exact_rank(m=60, n=50, r=5, seed=2)
    A = _cuda(w.A)
    eod.eod_abe_debug_fail_alloc_after(3)
    with pytest.raises(eod.EodError) as ei:
        eod.factor(A, w.tol, 1)
    assert ei.value.status == eod.EOD_ENOMEM
    eod.eod_abe_debug_fail_alloc_after(0)
    f = eod.factor(A, w.tol, 1)           # the library is still usable
    assert f.rank == 5


def test_host_entry_point(eod):
    w = W.exact_rank(m=120, n=90, r=11, seed=6)
    ref = oracle.eod_abe(w.A, w.tol, 0, k=32, seed=3)
    A = torch.from_numpy(np.asfortranarray(w.A)).pin_memory()
    cap = 90
    U = torch.zeros((cap, 120), dtype=torch.float64).t()
    D = torch.zeros((cap, cap), dtype=torch.float64).t()
    V = torch.zeros((cap, 90), dtype=torch.float64).t()
    r, rel = eod.factor_host(A, w.tol, 3, U_out=U, D_out=D, V_out=V)
    assert r == ref["r"] == 11
    assert abs(rel - ref["rel_err"]) <= 1e-10
    Ah = U[:, :r].numpy() @ D[:r, :r].numpy() @ V[:, :r].numpy().T
    assert np.linalg.norm(Ah - w.A) <= 1e-12 * np.linalg.norm(w.A)


def test_batched_matches_single_calls(eod):
    mats = [W.exact_rank(m=60 + 7 * i, n=50 + 3 * i, r=4 + i, seed=i).A for i in range(4)]
    res, stat = eod.factor_batched([_cuda(a) for a in mats], 1e-10, 7, block_k=8)
    assert stat == [0, 0, 0, 0]
    for i, a in enumerate(mats):
        ref = oracle.eod_abe(a, 1e-10, 0, k=8, seed=7, batch=i)
        assert res[i].rank == ref["r"] == 4 + i
        assert abs(res[i].rel_err - ref["rel_err"]) <= 1e-10


def test_reconstruct_matches_factors(eod):
    w = W.exact_rank(m=140, n=100, r=15, seed=9)
    f = eod.factor(_cuda(w.A), w.tol, 2, block_k=16)
    Ah = f.reconstruct().cpu().numpy()
    U, D, V = f.U.cpu().numpy(), f.D.cpu().numpy(), f.V.cpu().numpy()
    assert np.linalg.norm(Ah - U @ D @ V.T) <= 1e-13 * np.linalg.norm(w.A)
    assert np.linalg.norm(Ah - w.A) <= 1e-12 * np.linalg.norm(w.A)

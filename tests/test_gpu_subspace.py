"""Alg. 2 steps 2-7 (tau subspace iterations) on the GPU against the FP64
oracle: the rank is BasisExt's, RelErr within 1e-10 (FP64) or 1e-4 (FP32
data, mixed), and range(Q_tau) equal to the oracle's."""
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


def _cases():
    return {
        "exact": (lambda: W.exact_rank(m=300, n=200, r=12, seed=4), 1e-8, 16, 2),
        "image512": (lambda: W.image_like(m=512, n=384, r=60, seed=22, tol=0.05), 0.05, 32, 5),
        # large enough for the FP64 products to take the tensor-core emulation
        "image1024": (lambda: W.image_like(m=1024, n=1024, r=150, seed=8, tol=0.01), 0.01, 64, 3),
    }


@pytest.mark.parametrize("tau", [1, 2])
@pytest.mark.parametrize("case", ["exact", "image512", "image1024"])
def test_fp64_subspace_iteration_matches_oracle(eod, case, tau):
    make, tol, k, seed = _cases()[case]
    w = make()
    A64 = np.asfortranarray(w.A.astype(np.float64))
    ref = oracle.eod_abe(A64, tol, 1, k=k, seed=seed, tau=tau)
    f = eod.factor(torch.from_numpy(A64).cuda(), tol, seed, block_k=k, tol_mode="rel", power_iters=tau)
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
    Q = f.Q.cpu().numpy()
    Qo = ref["Q"]
    assert np.linalg.norm(Q.T @ Q - np.eye(f.rank)) <= 1e-12 * max(1, f.rank)
    assert np.linalg.norm(Q @ (Q.T @ Qo) - Qo) <= 1e-8 * np.sqrt(f.rank)
    Ah = f.reconstruct().cpu().numpy()
    Ah_ref = ref["U"] @ ref["D"] @ ref["V"].T
    assert np.linalg.norm(Ah - Ah_ref) <= 1e-10 * np.linalg.norm(A64)
    f.close()


def test_fp64_tau_reduces_error_toward_the_optimum(eod):
    """Same matrix, tau = 0, 1, 2: the rank stays, RelErr does not grow and
    stays above the Eckart-Young optimum of that rank (full SVD)."""
    w = W.image_like(m=512, n=384, r=60, seed=22, tol=0.05)
    A = torch.from_numpy(np.asfortranarray(w.A)).cuda()
    s = np.linalg.svd(w.A, compute_uv=False)
    errs, ranks = [], []
    for tau in (0, 1, 2):
        f = eod.factor(A, 0.05, 5, block_k=32, tol_mode="rel", power_iters=tau)
        errs.append(f.rel_err)
        ranks.append(f.rank)
        f.close()
    assert len(set(ranks)) == 1
    opt = np.sqrt(np.sum(s[ranks[0]:] ** 2)) / np.linalg.norm(s)
    assert errs[0] >= errs[1] * (1 - 1e-12) >= errs[2] * (1 - 1e-12)
    assert min(errs) >= opt * (1 - 1e-10)


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_fp32_data_subspace_iteration(eod, precision):
    w = W.image_like(m=640, n=512, r=80, seed=31, dtype="f32", tol=0.02)
    A32 = np.asfortranarray(w.A.astype(np.float32))
    ref = oracle.eod_abe(A32.astype(np.float64), 0.02, 1, k=32, seed=6, tau=1)
    f = eod.factor(torch.from_numpy(A32).cuda(), 0.02, 6, block_k=32, tol_mode="rel", precision=precision,
                   power_iters=1)
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4
    U, V = f.U.double(), f.V.double()
    I = torch.eye(f.rank, dtype=torch.float64, device="cuda")
    assert torch.linalg.norm(U.t() @ U - I).item() < 1e-5
    assert torch.linalg.norm(V.t() @ V - I).item() < 1e-5
    f.close()


def test_batched_subspace_iteration_equals_single_calls(eod):
    mats = [W.exact_rank(m=200 + 40 * i, n=150 + 30 * i, r=8 + 2 * i, seed=40 + i).A for i in range(3)]
    dev = [torch.from_numpy(np.asfortranarray(a)).cuda() for a in mats]
    res, st = eod.factor_batched(dev, 1e-8, 9, block_k=8, tol_mode="rel", power_iters=2)
    assert st == [eod.EOD_OK] * 3
    for i, a in enumerate(dev):
        f = eod.factor(a, 1e-8, 9, block_k=8, tol_mode="rel", batch_index=i, power_iters=2)
        assert f.rank == res[i].rank
        assert f.rel_err == res[i].rel_err
        assert torch.equal(f.U, res[i].U) and torch.equal(f.D, res[i].D)
        f.close()
        res[i].close()


def test_subspace_iteration_edge_cases(eod):
    """A zero matrix keeps rank 0 with tau > 0; a wide matrix (m < n) and
    a rank-1 matrix go through the iterations and match the oracle."""
    Z = torch.zeros((30, 40), dtype=torch.float64, device="cuda").t()
    f = eod.factor(Z, 1e-6, 1, power_iters=2)
    assert f.rank == 0 and f.rel_err == 0.0
    f.close()
    rng = np.random.default_rng(12)
    for A in (np.asfortranarray(rng.standard_normal((60, 9)) @ rng.standard_normal((9, 150))),
              np.asfortranarray(np.outer(rng.standard_normal(70), rng.standard_normal(50)))):
        ref = oracle.eod_abe(A, 1e-9, 1, k=4, seed=3, tau=1)
        f = eod.factor(torch.from_numpy(A).cuda(), 1e-9, 3, block_k=4, tol_mode="rel", power_iters=1)
        assert f.rank == ref["r"]
        assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
        f.close()

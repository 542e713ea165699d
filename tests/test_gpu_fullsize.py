"""Parity at the workloads' full sizes, in the configuration bench.py runs.

Where the FP64 oracle is too slow for a full run, the checks use properties
that hold at any size:
  * Thm 3.4(i): the T diagonal of the blocked process equals |diag R| of one
    Householder QR (LAPACK) of A Omega(:, 1:r+1), with Omega drawn by the
    oracle's independent generator; the rank is the first index where that
    diagonal drops to eps or below (Alg. 1 steps 6-11).
  * RelErr recomputed from the returned basis Q: ||A - Q Q^T A|| / ||A||, and
    against the span of the LAPACK factor of A Omega(:, 1:r).
  * orthogonality of U, V and the identity A_hat = U D V^T = Q C.
"""
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


def _lapack_reference(A64, eps, seed, r_gpu, batch=0):
    """T diagonal and rank from one LAPACK QR of A Omega, and the RelErr of
    the span of its first r columns (computed on the GPU in FP64 by torch)."""
    m, n = A64.shape
    ncols = min(r_gpu + 1, min(m, n))
    Om = oracle.omega(n, 0, ncols, seed, batch)
    At = torch.from_numpy(A64).cuda()
    Y = At @ torch.from_numpy(Om).cuda()
    Ql, R = torch.linalg.qr(Y)
    d = R.diagonal().abs().cpu().numpy()
    below = np.nonzero(d <= eps)[0]
    r_ref = int(below[0]) if below.size else ncols
    Qr = Ql[:, :r_ref]
    E = At - Qr @ (Qr.t() @ At)
    rel = (torch.linalg.norm(E) / torch.linalg.norm(At)).item()
    return d, r_ref, rel


def _basis_relerr(f, A64):
    At = torch.from_numpy(A64).cuda()
    Q = f.Q.double()
    E = At - Q @ (Q.t() @ At)
    return (torch.linalg.norm(E) / torch.linalg.norm(At)).item()


def test_image_like_2048_fp64_full(eod):
    w = W.image_like()
    A = torch.from_numpy(w.A).cuda()
    f = eod.factor(A, w.tol, w.seed, block_k=64, tol_mode="rel")
    d, r_ref, rel_ref = _lapack_reference(w.A, f.eps, w.seed, f.rank)
    assert f.rank == r_ref
    td = np.array(f.tdiag)[: r_ref + 1]
    assert np.max(np.abs(td - d[: td.size])) <= 1e-9 * f.norm_a
    assert abs(f.rel_err - _basis_relerr(f, w.A)) <= 1e-10
    assert abs(f.rel_err - rel_ref) <= 1e-10
    U, V = f.U, f.V
    I = torch.eye(f.rank, dtype=torch.float64, device="cuda")
    assert torch.linalg.norm(U.t() @ U - I).item() < 1e-10
    assert torch.linalg.norm(V.t() @ V - I).item() < 1e-10
    Ah = U @ f.D @ V.t()
    assert (torch.linalg.norm(Ah - f.Q @ f.Ct.t()) / torch.linalg.norm(A)).item() < 1e-12


def test_image_like_2048_fp32_and_mixed_full(eod):
    w = W.image_like()
    A64 = torch.from_numpy(w.A).cuda()
    A32 = A64.float().t().contiguous().t()
    f64 = eod.factor(A64, w.tol, w.seed, block_k=64, tol_mode="rel")
    for prec in ("plain", "mixed"):
        f = eod.factor(A32, w.tol, w.seed, block_k=64, tol_mode="rel", precision=prec)
        assert f.rank == f64.rank
        assert abs(f.rel_err - f64.rel_err) <= 1e-4


def test_harmonic_8192_mixed_full(eod):
    w = W.harmonic()
    A32 = torch.from_numpy(w.A).cuda()
    A64 = w.A.astype(np.float64)
    f = eod.factor(A32, w.tol, w.seed, block_k=64, tol_mode="rel", precision="mixed")
    d, r_ref, rel_ref = _lapack_reference(A64, f.eps, w.seed, f.rank)
    assert f.rank == r_ref
    assert abs(f.rel_err - rel_ref) <= 1e-4
    assert abs(f.rel_err - _basis_relerr(f, A64)) <= 1e-4
    td = np.array(f.tdiag)[: r_ref + 1]
    assert np.max(np.abs(td - d[: td.size]) / np.maximum(d[: td.size], 1e-30)) <= 1e-3


def test_hyperspectral_mixed_full(eod):
    w = W.hyperspectral()
    A32 = torch.from_numpy(w.A).cuda()
    A64 = w.A.astype(np.float64)
    f = eod.factor(A32, w.tol, w.seed, block_k=16, tol_mode="rel", precision="mixed")
    d, r_ref, rel_ref = _lapack_reference(A64, f.eps, w.seed, f.rank)
    assert f.rank == r_ref
    assert abs(f.rel_err - rel_ref) <= 1e-4
    assert abs(f.rel_err - _basis_relerr(f, A64)) <= 1e-4


def test_pixel_batch_256_mixed_full(eod):
    w = W.pixel_batch()
    mats = [torch.from_numpy(a).cuda() for a in w.A]
    res, st = eod.factor_batched(mats, w.tol, w.seed, block_k=32, tol_mode="rel", precision="mixed")
    assert st == [0] * 256
    # the four smallest items against the FP64 oracle (same batch index)
    sizes = sorted(range(256), key=lambda i: w.A[i].size)[:4]
    for i in sizes:
        ref = oracle.eod_abe(w.A[i].astype(np.float64), w.tol, 1, k=32, seed=w.seed, batch=i)
        assert res[i].rank == ref["r"], i
        assert abs(res[i].rel_err - ref["rel_err"]) <= 1e-4
    # every item: the reported error is the error of its basis
    for i in range(0, 256, 17):
        assert abs(res[i].rel_err - _basis_relerr(res[i], w.A[i].astype(np.float64))) <= 1e-4


def test_batched_equals_single_calls_mixed(eod, monkeypatch):
    # the worker-stream form (the persistent launch, which these small items
    # would take, computes in FP32 and is compared with the oracle in
    # test_gpu_batch_persistent.py)
    monkeypatch.setenv("EOD_BATCH_PERSISTENT", "0")
    mats = [W.image_like(m=200 + 37 * i, n=150 + 23 * i, r=20 + 3 * i, seed=40 + i, dtype="f32", tol=0.02).A
            for i in range(10)]
    tens = [torch.from_numpy(a).cuda() for a in mats]
    res, st = eod.factor_batched(tens, 0.02, 9, block_k=32, tol_mode="rel", precision="mixed")
    assert st == [0] * 10
    for i, t in enumerate(tens):
        f = eod.factor(t, 0.02, 9, block_k=32, tol_mode="rel", precision="mixed", batch_index=i)
        assert res[i].rank == f.rank
        assert res[i].rel_err == f.rel_err

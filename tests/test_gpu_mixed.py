"""GPU tests of the mixed path: each tcgen05 contraction against an FP64
product of the same inputs, then the whole mixed factorisation against the
FP64 oracle (rank exact, |dRelErr| <= 1e-4)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

# the BF16 hi/lo split keeps ~16 significant bits of each FP32 operand
SPLIT_TOL = 3e-5
# the sketch's three-term split represents FP32 exactly: only FP32 accumulation remains
SKETCH_TOL = 2e-6


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _colmajor(x):
    return x.t().contiguous().t()


def _bf16_exact(shape, gen):
    return torch.randn(shape, generator=gen).to(torch.bfloat16).float()


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _run(eod, form, M, N, K, X, Y, D, err=None):
    s = torch.cuda.current_stream()
    st = eod.eod_abe_debug_tc_gemm(form, M, N, K, _p(X), X.stride(1), _p(Y), Y.stride(1), _p(D), D.stride(1),
                                   _p(err), ctypes.c_void_p(s.cuda_stream))
    assert st == eod.EOD_OK, eod.status_string(st)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 70, 200), (1000, 256, 513), (64, 16, 1000),
                                   (2051, 130, 777)])
def test_tc_sketch_form(eod, M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    X = _colmajor(torch.randn((M, K), generator=g)).cuda()
    Y = _colmajor(_bf16_exact((K, N), g)).cuda()
    D = _colmajor(torch.full((M, N), float("nan"))).cuda()
    _run(eod, 0, M, N, K, X, Y, D)
    ref = X.double() @ Y.double()
    scale = (X.double().abs() @ Y.double().abs())
    assert torch.isfinite(D).all()
    assert ((D.double() - ref).abs() <= SKETCH_TOL * scale + 1e-30).all()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (200, 37, 300), (513, 256, 1000), (100, 300, 64),
                                   (2048, 20, 4100)])
def test_tc_projection_form(eod, M, N, K):
    g = torch.Generator().manual_seed(7 * M + N + K)
    X = _colmajor(torch.randn((K, M), generator=g)).cuda()
    Y = _colmajor(torch.randn((K, N), generator=g)).cuda()
    D = _colmajor(torch.full((M, N), float("nan"))).cuda()
    _run(eod, 1, M, N, K, X, Y, D)
    ref = X.double().t() @ Y.double()
    scale = X.double().abs().t() @ Y.double().abs()
    assert torch.isfinite(D).all()
    assert ((D.double() - ref).abs() <= SPLIT_TOL * scale + 1e-30).all()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 200, 12), (1000, 777, 130), (257, 1030, 400)])
def test_tc_reconstruction_error_form(eod, M, N, K):
    g = torch.Generator().manual_seed(3 * M + N + K)
    X = _colmajor(torch.randn((M, K), generator=g)).cuda()
    Y = _colmajor(torch.randn((N, K), generator=g)).cuda()
    P = X.double() @ Y.double().t()
    R = _colmajor((P + 1e-2 * torch.randn((M, N), generator=g, dtype=torch.float64).cuda()).float())
    err = torch.zeros(1, dtype=torch.float64, device="cuda")
    _run(eod, 2, M, N, K, X, Y, R, err)
    ref = torch.linalg.norm(R.double() - P).item()
    assert abs(err.item() - ref) <= 1e-3 * ref


# the TF32 hi/lo split keeps ~21 significant bits of each FP32 operand
TF32_TOL = 1e-5


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 70, 200), (1000, 256, 513), (2051, 130, 777)])
def test_tc_tf32_sketch_form(eod, M, N, K):
    g = torch.Generator().manual_seed(M + N + K + 8)
    X = _colmajor(torch.randn((M, K), generator=g)).cuda()
    Y = _colmajor(_bf16_exact((K, N), g)).cuda()   # BF16-exact values are TF32-exact
    D = _colmajor(torch.full((M, N), float("nan"))).cuda()
    _run(eod, 8, M, N, K, X, Y, D)
    ref = X.double() @ Y.double()
    scale = X.double().abs() @ Y.double().abs()
    assert torch.isfinite(D).all()
    assert ((D.double() - ref).abs() <= TF32_TOL * scale + 1e-30).all()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (200, 37, 300), (513, 256, 1000), (2048, 20, 4100)])
def test_tc_tf32_projection_form(eod, M, N, K):
    g = torch.Generator().manual_seed(7 * M + N + K + 9)
    X = _colmajor(torch.randn((K, M), generator=g)).cuda()
    Y = _colmajor(torch.randn((K, N), generator=g)).cuda()
    D = _colmajor(torch.full((M, N), float("nan"))).cuda()
    _run(eod, 9, M, N, K, X, Y, D)
    ref = X.double().t() @ Y.double()
    scale = X.double().abs().t() @ Y.double().abs()
    assert torch.isfinite(D).all()
    err = ((D.double() - ref).abs() / (scale + 1e-30)).max().item()
    assert err <= TF32_TOL, err
    # a single TF32 pass would be ~2^-11: the split must do far better
    assert err <= 1e-5


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (1000, 777, 130), (257, 1030, 400)])
def test_tc_tf32_reconstruction_error_form(eod, M, N, K):
    g = torch.Generator().manual_seed(3 * M + N + K + 10)
    X = _colmajor(torch.randn((M, K), generator=g)).cuda()
    Y = _colmajor(torch.randn((N, K), generator=g)).cuda()
    P = X.double() @ Y.double().t()
    R = _colmajor((P + 1e-2 * torch.randn((M, N), generator=g, dtype=torch.float64).cuda()).float())
    err = torch.zeros(1, dtype=torch.float64, device="cuda")
    _run(eod, 10, M, N, K, X, Y, R, err)
    ref = torch.linalg.norm(R.double() - P).item()
    assert abs(err.item() - ref) <= 1e-3 * ref


# --------------------------------------------------------------------------
# mixed factorisation vs the FP64 oracle
# --------------------------------------------------------------------------

def _factor_both(eod, A32, tol, mode, k, seed, batch=0, precision="mixed"):
    A64 = A32.astype(np.float64)
    ref = oracle.eod_abe(A64, tol, mode, k=k, seed=seed, batch=batch)
    At = torch.from_numpy(np.asfortranarray(A32)).cuda()
    f = eod.factor(At, tol, seed, block_k=k, tol_mode=("rel" if mode == 1 else "abs"), precision=precision,
                   batch_index=batch)
    return f, ref


def test_mixed_exact_rank(eod):
    w = W.exact_rank(m=600, n=450, r=25, seed=11)
    A32 = w.A.astype(np.float32)
    f, ref = _factor_both(eod, A32, 1e-4, 1, 16, 3)
    assert ref["r"] == 25
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4
    assert f.precision == eod.EOD_MIXED_BF16


def test_mixed_image_like_small(eod):
    w = W.image_like(m=512, n=384, r=60, seed=22, dtype="f32", tol=0.05)
    f, ref = _factor_both(eod, w.A, w.tol, 1, 32, w.seed)
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4


def test_mixed_harmonic_scaled(eod):
    # the 1/i spectrum + noise recipe at 1024 x 1024 (rank 400 signal)
    w = W.harmonic(m=1024, n=1024, r=400, seed=3, tol=0.03)
    f, ref = _factor_both(eod, w.A, w.tol, 1, 64, w.seed)
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4


def test_mixed_hyperspectral_scaled(eod):
    w = W.hyperspectral(pixels=20000, bands=224, seed=5)
    f, ref = _factor_both(eod, w.A, w.tol, 1, 16, w.seed)
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4


def test_mixed_from_fp64_input(eod):
    w = W.exact_rank(m=300, n=200, r=12, seed=4)
    ref = oracle.eod_abe(w.A, 1e-4, 1, k=16, seed=2)
    A = torch.from_numpy(w.A).cuda()
    f = eod.factor(A, 1e-4, 2, block_k=16, tol_mode="rel", precision="mixed")
    assert f.rank == ref["r"] == 12
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4


def test_mixed_reconstruct_and_orthogonality(eod):
    w = W.image_like(m=400, n=300, r=40, seed=9, dtype="f32", tol=0.02)
    f, ref = _factor_both(eod, w.A, w.tol, 1, 32, w.seed)
    assert f.rank == ref["r"]
    U, V = f.U.double(), f.V.double()
    I = torch.eye(f.rank, dtype=torch.float64, device="cuda")
    assert torch.linalg.norm(U.t() @ U - I).item() < 1e-5
    assert torch.linalg.norm(V.t() @ V - I).item() < 1e-5
    Ah = f.reconstruct().double()
    A = torch.from_numpy(w.A.astype(np.float64)).cuda()
    rel = (torch.linalg.norm(A - Ah) / torch.linalg.norm(A)).item()
    assert abs(rel - ref["rel_err"]) <= 1e-4


def test_tolerance_below_precision_floor_is_refused(eod):
    """eps under the FP32-data floor (1e-5 ||A||_F), mixed or plain, gives
    EOD_EPRECISION, not a guessed rank."""
    w = W.exact_rank(m=300, n=200, r=12, seed=4)
    A32 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float32))).cuda()
    for prec, tol in (("mixed", 5e-6), ("plain", 5e-6)):
        with pytest.raises(eod.EodError) as ei:
            eod.factor(A32, tol, 2, block_k=16, tol_mode="rel", precision=prec)
        assert ei.value.status == eod.EOD_EPRECISION
    f = eod.factor(A32, 1e-4, 2, block_k=16, tol_mode="rel", precision="mixed")
    assert f.rank == 12


def test_mixed_exact_rank_noise_tail_matches_fp64(eod):
    """Exact-rank data stored in FP32 has a pure-noise tail; without
    oversampling the method amplifies sketch rounding there, so the mixed
    sketch must be FP32-exact for the rank to match the FP64 path."""
    w = W.pixel_batch(count=12, clip=False, tol=1e-4, seed=4)
    for i, a in enumerate(w.A):
        A64 = torch.from_numpy(np.asfortranarray(a.astype(np.float64))).cuda()
        A32 = torch.from_numpy(a).cuda()
        fp = eod.factor(A64, 1e-4, w.seed, block_k=32, tol_mode="rel", batch_index=i)
        fm = eod.factor(A32, 1e-4, w.seed, block_k=32, tol_mode="rel", precision="mixed", batch_index=i)
        assert fm.rank == fp.rank
        assert abs(fm.rel_err - fp.rel_err) <= 1e-4


@pytest.mark.parametrize("case", ["exact_rank", "image_like", "harmonic"])
def test_mixed_tf32_factorisations(eod, case):
    """EOD_MIXED_TF32 (kind::tf32 contractions on two-term TF32 splits)
    against the FP64 oracle: rank exact, |dRelErr| <= 1e-4."""
    if case == "exact_rank":
        w = W.exact_rank(m=600, n=450, r=25, seed=11)
        A32, tol, k, seed = w.A.astype(np.float32), 1e-4, 16, 3
    elif case == "image_like":
        w = W.image_like(m=512, n=384, r=60, seed=22, dtype="f32", tol=0.05)
        A32, tol, k, seed = w.A, w.tol, 32, w.seed
    else:
        w = W.harmonic(m=1024, n=1024, r=400, seed=3, tol=0.03)
        A32, tol, k, seed = w.A, w.tol, 64, w.seed
    f, ref = _factor_both(eod, A32, tol, 1, k, seed, precision="mixed_tf32")
    assert f.precision == eod.EOD_MIXED_TF32
    assert f.rank == ref["r"]
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4

"""The FP64 GEMM emulated on tcgen05 (exact BF16 slices, FP64 accumulation)
against cuBLAS FP64 (torch) on the same inputs: ragged shapes, every
transpose combination, split-K, alpha/beta, wide dynamic range, zero rows."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _cm(x):
    return x.t().contiguous().t()


def _run(eod, mode, ta, tb, A, B, C, alpha, beta, M, N, K):
    s = torch.cuda.current_stream()
    st = eod.eod_abe_debug_f64_gemm(mode, int(ta), int(tb), M, N, K, alpha, ctypes.c_void_p(A.data_ptr()),
                                    A.stride(1), ctypes.c_void_p(B.data_ptr()), B.stride(1), beta,
                                    ctypes.c_void_p(C.data_ptr()), C.stride(1), ctypes.c_void_p(s.cuda_stream))
    assert st == eod.EOD_OK, eod.status_string(st)


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (300, 70, 200), (1000, 513, 777), (64, 16, 4000),
                                   (2048, 2037, 2048)])
def test_emulated_matches_fp64(eod, ta, tb, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K + 11 * ta + 5 * tb)
    A = _cm(torch.randn((K, M) if ta else (M, K), generator=g, device="cuda", dtype=torch.float64))
    B = _cm(torch.randn((N, K) if tb else (K, N), generator=g, device="cuda", dtype=torch.float64))
    C0 = _cm(torch.randn((M, N), generator=g, device="cuda", dtype=torch.float64))
    opA = A.t() if ta else A
    opB = B.t() if tb else B
    ref = 0.75 * (opA @ opB) - 0.5 * C0
    C = C0.clone()
    _run(eod, 1, ta, tb, A, B, C, 0.75, -0.5, M, N, K)
    scale = 0.75 * (opA.abs() @ opB.abs()) + 0.5 * C0.abs()
    err = ((C - ref).abs() / scale).max().item()
    assert err <= 1e-13, err   # FP64-class: BF16 alone would give ~1e-3, FP32 ~1e-7


def test_emulated_dynamic_range_and_zero_rows(eod):
    M, N, K = 257, 190, 1030
    g = torch.Generator(device="cuda").manual_seed(3)
    rs = torch.logspace(-8, 8, M, device="cuda", dtype=torch.float64)
    cs = torch.logspace(6, -6, N, device="cuda", dtype=torch.float64)
    A = _cm(torch.randn((M, K), generator=g, device="cuda", dtype=torch.float64) * rs[:, None])
    B = _cm(torch.randn((K, N), generator=g, device="cuda", dtype=torch.float64) * cs[None, :])
    A[17] = 0.0
    B[:, 5] = 0.0
    C = _cm(torch.zeros((M, N), device="cuda", dtype=torch.float64))
    _run(eod, 1, False, False, A, B, C, 1.0, 0.0, M, N, K)
    ref = A @ B
    scale = A.abs() @ B.abs()
    assert (C[17] == 0).all() and (C[:, 5] == 0).all()
    mask = scale > 0
    assert ((C - ref).abs()[mask] / scale[mask]).max().item() <= 1e-13


def test_simt_and_emulated_agree_on_gram(eod):
    M, K = 700, 3000
    g = torch.Generator(device="cuda").manual_seed(9)
    W = _cm(torch.randn((K, M), generator=g, device="cuda", dtype=torch.float64))
    C1 = _cm(torch.zeros((M, M), device="cuda", dtype=torch.float64))
    C2 = C1.clone()
    _run(eod, 0, True, False, W, W, C1, 1.0, 0.0, M, M, K)
    _run(eod, 1, True, False, W, W, C2, 1.0, 0.0, M, M, K)
    ref = W.t() @ W
    assert ((C2 - ref).abs() / (W.abs().t() @ W.abs())).max().item() <= 1e-13
    assert ((C1 - ref).abs() / (W.abs().t() @ W.abs())).max().item() <= 1e-13


# --------------------------------------------------------------------------
# whole factorisation: every FP64 product emulated vs every product on SIMT
# --------------------------------------------------------------------------

_CHILD = r"""
import sys, numpy as np, torch
import paper_2506_22713_gb300 as eod
import workloads as W
which, out = sys.argv[1], sys.argv[2]
if which == "exact":
    w = W.exact_rank(m=900, n=700, r=60, seed=8)
    A, tol, k, seed = w.A, 1e-8, 32, 5
else:
    w = W.image_like(m=640, n=520, r=90, seed=13, tol=0.01)
    A, tol, k, seed = w.A, w.tol, 64, w.seed
f = eod.factor(torch.from_numpy(np.asfortranarray(A)).cuda(), tol, seed, block_k=k, tol_mode="rel")
np.savez(out, rank=f.rank, rel_err=f.rel_err, tdiag=np.array(f.tdiag), U=f.U.cpu().numpy(),
         V=f.V.cpu().numpy(), D=f.D.cpu().numpy(), tol=tol, k=k, seed=seed)
"""


def _child(which, mode, tmp_path):
    import os
    import subprocess
    import sys
    import numpy as np
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / f"{which}_{mode}.npz")
    env = dict(os.environ, EOD_FP64_GEMM=mode, PYTHONPATH=root)
    subprocess.run([sys.executable, "-c", _CHILD, which, out], check=True, cwd=root, env=env, timeout=600)
    return np.load(out)


@pytest.mark.parametrize("which", ["exact", "image"])
def test_factorisation_emulated_matches_simt_and_oracle(eod, which, tmp_path):
    import numpy as np
    import oracle
    import workloads as W
    em = _child(which, "emulated", tmp_path)
    si = _child(which, "simt", tmp_path)
    assert int(em["rank"]) == int(si["rank"])
    # the diagonal of T decides the rank: the two product paths agree to FP64 rounding
    te, ts = np.abs(em["tdiag"]), np.abs(si["tdiag"])
    assert te.shape == ts.shape
    assert np.all(np.abs(te - ts) <= 1e-9 * ts.max())
    assert abs(float(em["rel_err"]) - float(si["rel_err"])) <= 1e-12
    Ue, Us = em["U"], si["U"]
    assert np.linalg.norm(Ue.T @ Ue - np.eye(Ue.shape[1])) <= 1e-12
    Ae = Ue @ em["D"] @ em["V"].T      # A ~ U D V^T with D upper triangular
    As = Us @ si["D"] @ si["V"].T
    assert np.linalg.norm(Ae - As) <= 1e-10 * np.linalg.norm(As)
    w = W.exact_rank(m=900, n=700, r=60, seed=8) if which == "exact" else W.image_like(m=640, n=520, r=90,
                                                                                     seed=13, tol=0.01)
    ref = oracle.eod_abe(w.A, float(em["tol"]), 1, k=int(em["k"]), seed=int(em["seed"]))
    assert int(em["rank"]) == ref["r"]
    assert abs(float(em["rel_err"]) - ref["rel_err"]) <= 1e-10


def _tol(mode, A, B, K):
    """Entrywise bound for C = A B.  SIMT DFMA: the usual componentwise FP64
    bound.  Emulation: each row of A and column of B is sliced against its
    own largest entry, so an entry's error is bounded by K 2^-48 max|A(i,:)|
    max|B(:,j)| on top (8 slices of 7 bits, the pairs below 2^-56 dropped):
    normwise per row and column, not relative to |A||B| where a triangular
    column has a single term."""
    t = 1e-13 * (A.abs() @ B.abs()) + 1e-300
    if mode == 1:
        t = t + K * 2.0 ** -48 * A.abs().amax(dim=1, keepdim=True) * B.abs().amax(dim=0, keepdim=True)
    return t


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("M,N,K", [(300, 300, 300), (1000, 700, 700), (64, 2050, 2050)])
def test_triangular_b_operand(eod, mode, M, N, K):
    """op(B) upper triangular (the triangular solves of the core QR): the
    emulation never reads the zero part (NaN there must not leak), the SIMT
    kernel skips whole zero K ranges of it."""
    g = torch.Generator(device="cuda").manual_seed(M + N + K + mode)
    A = _cm(torch.randn((M, K), generator=g, device="cuda", dtype=torch.float64))
    Bu = torch.triu(torch.randn((K, N), generator=g, device="cuda", dtype=torch.float64))
    B = _cm(Bu.clone())
    if mode == 1:
        B[torch.tril(torch.ones_like(Bu, dtype=torch.bool), -1)] = float("nan")
    C = _cm(torch.zeros((M, N), device="cuda", dtype=torch.float64))
    _run(eod, mode | 64, False, False, A, B, C, 1.0, 0.0, M, N, K)
    ref = A @ Bu
    assert ((C - ref).abs() <= _tol(mode, A, Bu, K)).all()


@pytest.mark.parametrize("mode", [0, 1])
def test_triangular_both_operands(eod, mode):
    p = 777
    g = torch.Generator(device="cuda").manual_seed(9 + mode)
    Au = torch.triu(torch.randn((p, p), generator=g, device="cuda", dtype=torch.float64))
    Bu = torch.triu(torch.randn((p, p), generator=g, device="cuda", dtype=torch.float64))
    A, B = _cm(Au.clone()), _cm(Bu.clone())
    if mode == 1:
        low = torch.tril(torch.ones_like(Au, dtype=torch.bool), -1)
        A[low] = float("nan")
        B[low] = float("inf")
    C = _cm(torch.zeros((p, p), device="cuda", dtype=torch.float64))
    _run(eod, mode | 32 | 64, False, False, A, B, C, 1.0, 0.0, p, p, p)
    ref = Au @ Bu
    assert ((C - ref).abs() <= _tol(mode, Au, Bu, p)).all()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("p,K", [(300, 4000), (1100, 2048)])
def test_upper_only_gram(eod, mode, p, K):
    """G = W^T W with only the upper triangle wanted (split-K and single
    pass); the emulation leaves every entry below the diagonal as it was."""
    g = torch.Generator(device="cuda").manual_seed(p + K + mode)
    W = _cm(torch.randn((K, p), generator=g, device="cuda", dtype=torch.float64))
    C = _cm(torch.full((p, p), -7.0, device="cuda", dtype=torch.float64))
    _run(eod, mode | 16, True, False, W, W, C, 1.0, 0.0, p, p, K)
    ref = W.t() @ W
    scale = W.abs().t() @ W.abs()
    up = torch.triu(torch.ones((p, p), dtype=torch.bool, device="cuda"))
    assert ((C - ref).abs()[up] <= 1e-13 * scale[up]).all()
    if mode == 1:
        assert (C[~up] == -7.0).all()


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("M,K", [(9, 262144), (262144, 9), (1, 1), (3000, 2100), (37, 5)])
def test_matrix_vector_products(eod, ta, M, K):
    """N = 1 (the explicit residual of an undecided pivot) through the SIMT
    path's matrix-vector kernels, both orientations, with alpha and beta."""
    g = torch.Generator(device="cuda").manual_seed(M + K + ta)
    A = _cm(torch.randn((K, M) if ta else (M, K), generator=g, device="cuda", dtype=torch.float64))
    x = _cm(torch.randn((K, 1), generator=g, device="cuda", dtype=torch.float64))
    C0 = _cm(torch.randn((M, 1), generator=g, device="cuda", dtype=torch.float64))
    opA = A.t() if ta else A
    ref = -1.0 * (opA @ x) + 0.5 * C0
    C = C0.clone()
    s = torch.cuda.current_stream()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    # single columns: their leading dimensions are their lengths (torch may
    # report a unit stride for a one-column tensor)
    st = eod.eod_abe_debug_f64_gemm(0, int(ta), 0, M, 1, K, -1.0, P(A), A.stride(1), P(x), K, 0.5, P(C), M,
                                    ctypes.c_void_p(s.cuda_stream))
    assert st == eod.EOD_OK, eod.status_string(st)
    scale = opA.abs() @ x.abs() + 0.5 * C0.abs()
    assert ((C - ref).abs() <= 1e-13 * scale + 1e-300).all()


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K,flags", [(64, 192, 64, 0), (64, 64, 64, 32), (128, 128, 128, 64), (5, 3, 7, 0),
                                         (17, 33, 100, 0), (2048, 64, 64, 64), (64, 64, 192, 0),
                                         (245, 245, 256, 16), (192, 64, 2048, 0), (64, 192, 64, 128),
                                         (245, 245, 256, 16 | 128), (192, 64, 2048, 128)])
def test_simt_small_products(eod, ta, tb, M, N, K, flags):
    """The SIMT kernel on the small products of the panel factorisation
    (16- and 32-tiles, K splits summed in split order by each tile's last CTA,
    or by the separate reduction: flag 128), with the triangular-operand and
    upper-only flags."""
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K + flags + 2 * ta + tb)
    A = torch.randn((K, M) if ta else (M, K), generator=g, device="cuda", dtype=torch.float64)
    B = torch.randn((N, K) if tb else (K, N), generator=g, device="cuda", dtype=torch.float64)
    opA = A.t() if ta else A
    opB = B.t() if tb else B
    if flags & 32:
        opA = torch.triu(opA)
    if flags & 64:
        opB = torch.triu(opB)
    A = _cm((opA.t() if ta else opA).contiguous())
    B = _cm((opB.t() if tb else opB).contiguous())
    C0 = _cm(torch.randn((M, N), generator=g, device="cuda", dtype=torch.float64))
    C = C0.clone()
    _run(eod, flags, ta, tb, A, B, C, -1.0, 1.0, M, N, K)
    if flags & 128:   # the two ways of summing a K split give the same bits
        C2 = C0.clone()
        _run(eod, flags & ~128, ta, tb, A, B, C2, -1.0, 1.0, M, N, K)
        keep = torch.triu(torch.ones((M, N), dtype=torch.bool, device="cuda")) if flags & 16 else torch.ones(
            (M, N), dtype=torch.bool, device="cuda")
        assert torch.equal(C[keep], C2[keep])
    ref = C0 - opA @ opB
    tol = 1e-13 * (opA.abs() @ opB.abs() + C0.abs()) + 1e-300
    if flags & 16:
        keep = torch.triu(torch.ones((M, N), dtype=torch.bool, device="cuda"))
        assert ((C - ref).abs()[keep] <= tol[keep]).all()
    else:
        assert ((C - ref).abs() <= tol).all()


def test_fp32_products_through_the_emulation_match_the_oracle():
    """EOD_FP32_GEMM=emulated sends the FP32 paths' large products through the
    same emulation (FP32 data exact in FP64, rounded once to FP32): a plain
    FP32 and a mixed factorisation still match the FP64 oracle.  Run in a
    child process because the switch is read once per process."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = r'''
import numpy as np, torch, oracle, workloads as W
import paper_2506_22713_gb300 as eod
w = W.image_like(m=1500, n=1200, r=60, tol=2e-3)
A32 = w.A.astype(np.float32)
ref = oracle.eod_abe(A32.astype(np.float64), w.tol, 1, k=64, seed=w.seed)
A = torch.from_numpy(np.asfortranarray(A32)).cuda()
for prec in ("plain", "mixed"):
    f = eod.factor(A, w.tol, w.seed, block_k=64, tol_mode="rel", precision=prec)
    assert f.rank == ref["r"], (prec, f.rank, ref["r"])
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-4, (prec, f.rel_err, ref["rel_err"])
    I = torch.eye(f.rank, dtype=torch.float64, device="cuda")
    assert torch.linalg.norm(f.V.double().t() @ f.V.double() - I).item() < 1e-4
    f.close()
print("ok")
'''
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root, timeout=600,
                         env=dict(os.environ, EOD_FP32_GEMM="emulated", PYTHONPATH=root))
    assert out.returncode == 0 and "ok" in out.stdout, out.stderr[-3000:]

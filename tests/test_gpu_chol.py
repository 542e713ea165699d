"""The one-CTA leaf factorisation behind CholQR (Alg. 1 steps 5-11, Alg. 2
steps 9-10) against FP64 LAPACK on the host: R^T R = G + shift I, R^{-1} R = I,
and the three outcomes of the rank test on pivots placed around eps^2."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _run(eod, G, decide=0, eps2=0.0, coef=0.0, rho=0.0, shift=0.0, inverse=True):
    w = G.shape[0]
    Gd = torch.from_numpy(np.asfortranarray(G)).cuda()
    R = torch.full((w, w), float("nan"), dtype=torch.float64, device="cuda").t()
    Ri = torch.full((w, w), float("nan"), dtype=torch.float64, device="cuda").t() if inverse else None
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = eod.eod_abe_debug_chol(P(Gd), w, w, decide, eps2, coef, rho, shift, P(R), P(Ri), w, P(info),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == eod.EOD_OK
    p, code = info.tolist()
    Rn = R.cpu().numpy()[:p, :p]
    Rin = Ri.cpu().numpy()[:p, :p] if inverse else None
    return p, code, Rn, Rin


def _spd(w, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((w, w)))
    s = np.geomspace(1.0, 1.0 / cond, w)
    return (Q * s) @ Q.T


@pytest.mark.parametrize("w", [1, 2, 17, 63, 64, 65, 100, 128])
@pytest.mark.parametrize("cond", [1e2, 1e8])
def test_factor_and_inverse(eod, w, cond):
    G = _spd(w, cond, w)
    p, code, R, Ri = _run(eod, G)
    assert (p, code) == (w, 0)
    assert np.all(np.diag(R) > 0) and np.allclose(np.tril(R, -1), 0.0)
    # backward error of a Cholesky factorisation: O(w u) ||G||
    assert np.linalg.norm(R.T @ R - G) <= 20 * w * U64 * np.linalg.norm(G)
    Rref = np.linalg.cholesky(G).T
    assert np.linalg.norm(R - Rref) <= 50 * w * U64 * cond * np.linalg.norm(Rref)
    assert np.allclose(np.tril(Ri, -1), 0.0)
    assert np.linalg.norm(Ri @ R - np.eye(w)) <= 50 * w * U64 * np.sqrt(cond) * np.sqrt(cond)


def test_shift_is_added_to_the_diagonal(eod):
    G = _spd(40, 1e3, 5)
    p, code, R, _ = _run(eod, G, shift=0.25, inverse=False)
    assert (p, code) == (40, 0)
    assert np.linalg.norm(R.T @ R - (G + 0.25 * np.eye(40))) <= 1e-13 * np.linalg.norm(G)


def test_rank_test_outcomes(eod):
    """Pivots d_j = T(j,j)^2 of a diagonal Gram: kept while above
    eps^2 + delta, stop below eps^2 - delta (code 1), undecided inside the
    band (code 2), and the rho guard."""
    coef = 64.0 * (16 + np.sqrt(1000.0)) * U64
    eps2 = 1e-6
    d = np.array([4.0, 1.0, 2e-6, 1e-9, 5.0])
    p, code, R, _ = _run(eod, np.diag(d), decide=1, eps2=eps2, coef=coef, rho=1e-10, inverse=False)
    assert (p, code) == (3, 1)
    assert np.allclose(np.diag(R), np.sqrt(d[:3]), rtol=1e-15)
    # inside the rounding band around eps^2: undecided
    d2 = np.array([4.0, eps2 * (1 + 1e-13), 5.0])
    p, code, _, _ = _run(eod, np.diag(d2), decide=1, eps2=eps2, coef=coef, rho=1e-10, inverse=False)
    assert (p, code) == (1, 2)
    # pivot above eps^2 + delta but below rho G(j,j) (nearly dependent
    # columns): undecided
    b = np.sqrt(1.0 - 1e-12)
    G3 = np.array([[1.0, b, 0.0], [b, 1.0, 0.0], [0.0, 0.0, 1.0]])
    p, code, _, _ = _run(eod, G3, decide=1, eps2=1e-14, coef=coef, rho=1e-10, inverse=False)
    assert (p, code) == (1, 2)
    p, code, _, _ = _run(eod, G3, decide=1, eps2=1e-14, coef=coef, rho=1e-13, inverse=False)
    assert (p, code) == (3, 0)


def test_not_positive_definite_stops(eod):
    G = _spd(30, 10.0, 7)
    G[12, 12] = -1.0
    p, code, _, _ = _run(eod, G, inverse=False)
    assert code == 3 and p <= 12


def test_stopped_factorisation_keeps_its_inverse(eod):
    """A rank-test stop at pivot p leaves the leading p x p factor and its
    inverse: R^T R = G(:p, :p) and R^{-1} R = I (the inverse is built in the
    same steps as the factor, so it must stop with it)."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((200, 64))
    X[:, 40] *= 1e-8
    G = X.T @ X
    coef = 64.0 * (16 + np.sqrt(1000.0)) * U64
    p, code, R, Ri = _run(eod, G, decide=1, eps2=1e-10, coef=coef, rho=1e-10)
    assert (p, code) == (40, 1)
    Gp = G[:40, :40]
    assert np.linalg.norm(R.T @ R - Gp) <= 20 * 40 * U64 * np.linalg.norm(Gp)
    assert np.allclose(np.tril(Ri, -1), 0.0)
    assert np.linalg.norm(Ri @ R - np.eye(40)) <= 1e-12


def test_leaf_reciprocal_against_cuda_division(eod):
    """The leaf's pivot reciprocal (FP32 seed, one third-order step) against
    CUDA's correctly rounded FP64 division, over the whole exponent range
    whose reciprocals are normal: within 2 ulp everywhere, and its two
    deliberate edge returns (+inf for subnormal d, 0 where 1/d would be
    subnormal)."""
    rng = np.random.default_rng(17)
    mant = rng.uniform(1.0, 2.0, 200_000)
    expo = rng.integers(-1021, 1022, 200_000)
    d = np.ldexp(mant, expo)
    d = np.concatenate([d, [1.0, 2.0, 0.5, 1.5, np.nextafter(2.0, 0.0), 2.0 ** -1022, 2.0 ** 1021, 3.0, 7.0]])
    dd = torch.from_numpy(d).cuda()
    out = torch.empty_like(dd)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert eod.eod_abe_debug_recip(P(dd), P(out), dd.numel(), s) == eod.EOD_OK
    ref = (1.0 / dd).cpu().numpy()
    got = out.cpu().numpy()
    ulps = np.abs(got - ref) / np.spacing(ref)
    assert np.all(np.isfinite(got))
    assert ulps.max() <= 2.0, ulps.max()
    # edges: subnormal (and zero) pivots give +inf; reciprocals below the
    # normal range give 0
    edge = torch.tensor([5e-324, 2.0 ** -1030, 0.0, 2.0 ** 1023 * 1.5, 2.0 ** 1022 * 1.75],
                        dtype=torch.float64, device="cuda")
    eo = torch.empty_like(edge)
    assert eod.eod_abe_debug_recip(P(edge), P(eo), edge.numel(), s) == eod.EOD_OK
    e = eo.cpu().numpy()
    assert np.isinf(e[0]) and e[0] > 0 and np.isinf(e[1]) and np.isinf(e[2])
    assert e[3] == 0.0 and e[4] == 0.0
    assert eod.eod_abe_debug_recip(None, P(eo), 1, s) == eod.EOD_EINVAL


@pytest.mark.parametrize("w,cond,decide", [(64, 1e4, 0), (128, 1e6, 0), (37, 1e3, 0), (64, 1e8, 1), (2, 10.0, 0),
                                           (1, 1.0, 0), (100, 1e5, 1)])
def test_lookahead_schedule_matches_the_two_barrier_schedule(eod, w, cond, decide):
    """The library's leaf (one barrier per pivot, the next pivot decided
    while the trailing update runs) against the two-barrier schedule (decide
    | 256): same columns factored, same outcome, factors equal up to
    rounding; in decide mode with eps between the pivots, the same stop."""
    G = _spd(w, cond, 100 + w)
    eps2 = float(np.sort(np.linalg.eigvalsh(G))[w // 2]) if decide else 0.0
    coef = 64 * (64 + np.sqrt(1000.0)) * U64 if decide else 0.0
    rho = 1e-10 if decide else 0.0
    a = _run(eod, G, decide=decide, eps2=eps2, coef=coef, rho=rho)
    b = _run(eod, G, decide=decide | 256, eps2=eps2, coef=coef, rho=rho)
    assert a[0] == b[0] and a[1] == b[1]
    p = a[0]
    if p:
        scale = np.abs(a[2]).max()
        assert np.abs(a[2] - b[2]).max() <= 1e-12 * cond * scale
        assert np.abs(a[3] @ a[2] - np.eye(p)).max() <= 1e-9 * cond

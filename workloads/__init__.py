"""Seeded synthetic inputs for EOD-ABE, shared by the CUDA path's tests and
benchmark and by the oracle's tests.

This module only draws matrices; it holds none of the method's arithmetic.
Each generator stands in for a workload of the paper (whose images and
hyperspectral cube are not available): the shapes, value ranges and spectra
follow the paper's experiments (Sec. 4) scaled to the sizes named below.

All matrices are returned as column-major (Fortran-ordered) numpy arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def haar_frame(rng: np.random.Generator, m: int, r: int) -> np.ndarray:
    """m x r matrix with orthonormal columns, Haar distributed: the Q factor
    of a standard Gaussian matrix with the signs of diag(R) moved into Q
    (Mezzadri, Notices AMS 2007)."""
    G = rng.standard_normal((m, r))
    Qm, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Qm * d


def low_rank(rng: np.random.Generator, m: int, n: int, s: np.ndarray) -> np.ndarray:
    """U diag(s) V^T with Haar U (m x r), V (n x r)."""
    s = np.asarray(s, dtype=np.float64)
    U = haar_frame(rng, m, s.size)
    V = haar_frame(rng, n, s.size)
    return np.asfortranarray((U * s) @ V.T)


@dataclass
class Workload:
    name: str
    A: object                     # np.ndarray (single) or list of np.ndarray (batched)
    dtype: str                    # storage type handed to the library: "f64" or "f32"
    tol: float
    tol_mode: int                 # 0 absolute, 1 relative to ||A||_F
    seed: int                     # seed of the Gaussian test matrix
    note: str = ""
    meta: dict = field(default_factory=dict)


def exact_rank(m: int = 512, n: int = 384, r: int = 20, seed: int = 1,
               smax: float = 1.0, smin: float = 1e-2) -> Workload:
    """Exactly rank-r U diag(s) V^T with s geometric from smax to smin and no
    noise (the rank-revealing regime of Thm 3.4); absolute tol 1e-10."""
    rng = np.random.default_rng(seed)
    s = np.geomspace(smax, smin, r)
    A = low_rank(rng, m, n, s)
    return Workload(f"exact_rank_{m}x{n}_r{r}", A, "f64", 1e-10, 0, seed,
                    note="U diag(s) V^T, Haar U/V, s geometric 1 -> 1e-2, no noise",
                    meta={"r_true": r})


def image_like(m: int = 2048, n: int = 2048, r: int = 150, seed: int = 2,
               tol: float = 1e-3, dtype: str = "f64", noise_rel: float = 1e-4) -> Workload:
    """Image-like matrix: rank-r U diag(s) V^T with s_i = 255 i^-1.5 plus
    i.i.d. Gaussian noise of std noise_rel * s_1, relative tol (stand-in for
    the 8-bit colour channels of Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, r + 1, dtype=np.float64)
    s = 255.0 * i ** -1.5
    A = low_rank(rng, m, n, s)
    A += (noise_rel * s[0]) * rng.standard_normal((m, n))
    A = np.asfortranarray(A)
    if dtype == "f32":
        A = np.asfortranarray(A.astype(np.float32))
    return Workload(f"image_like_{m}x{n}_r{r}_{dtype}", A, dtype, tol, 1, seed,
                    note="rank-r s_i=255 i^-1.5, Haar U/V, noise 1e-4 s_1, tol relative",
                    meta={"r_signal": r})


def harmonic(m: int = 8192, n: int = 8192, r: int = 400, seed: int = 3,
             tol: float = 0.0128, noise: float = 1e-6) -> Workload:
    """Rank-r U diag(1/i) V^T plus Gaussian noise (std 1e-6), FP32 storage,
    relative tol 0.0128 (twice the noise floor sigma*sqrt(mn)/||A||_F)."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, r + 1, dtype=np.float64)
    A = low_rank(rng, m, n, 1.0 / i)
    A += noise * rng.standard_normal((m, n))
    A = np.asfortranarray(A.astype(np.float32))
    return Workload(f"harmonic_{m}x{n}_r{r}_f32", A, "f32", tol, 1, seed,
                    note="rank-r s_i=1/i, Haar U/V, noise 1e-6, FP32",
                    meta={"r_signal": r})


def pixel_batch(count: int = 256, lo: int = 256, hi: int = 2048, rlo: int = 8, rhi: int = 128,
                seed: int = 4, tol: float = 1e-3, clip: bool = True) -> Workload:
    """Batch of image-like matrices of uneven size: m, n uniform in [lo, hi],
    r uniform in [rlo, rhi], s_i = 255 exp(-i/(r/4)), values clipped to
    [0, 255] like 8-bit pixels, FP32 storage, relative tol."""
    rng = np.random.default_rng(seed)
    mats, ranks = [], []
    for _ in range(count):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        r = int(rng.integers(rlo, rhi + 1))
        i = np.arange(1, r + 1, dtype=np.float64)
        s = 255.0 * np.exp(-i / (r / 4.0))
        A = low_rank(rng, m, n, s)
        if clip:
            A = np.clip(A, 0.0, 255.0)
        mats.append(np.asfortranarray(A.astype(np.float32)))
        ranks.append(r)
    return Workload(f"pixel_batch_{count}", mats, "f32", tol, 1, seed,
                    note="m,n~U[256,2048], r~U[8,128], s_i=255exp(-i/(r/4)), clip [0,255]",
                    meta={"r_signal": ranks})


def rgb_image(m: int = 220, n: int = 220, ranks=(50, 52, 53), seed: int = 6) -> Workload:
    """Synthetic colour image: three nonnegative channels of exact ranks
    `ranks` (products of nonnegative uniform factors), scaled to [0, 255],
    FP64 storage -- the shape of the toy example of Sec. 1 (220 x 220,
    ranks 50, 52, 53).  Relative tol 1e-10 reveals the exact ranks."""
    rng = np.random.default_rng(seed)
    chans = []
    for r in ranks:
        W = rng.uniform(0.0, 1.0, (m, r))
        H = rng.uniform(0.0, 1.0, (r, n))
        C = W @ H
        chans.append(np.asfortranarray(255.0 * C / C.max()))
    return Workload(f"rgb_{m}x{n}", chans, "f64", 1e-10, 1, seed,
                    note="3 nonnegative channels, exact ranks " + ",".join(str(r) for r in ranks),
                    meta={"r_signal": list(ranks)})


def hyperspectral(pixels: int = 512 * 512, bands: int = 224, endmembers: int = 12, seed: int = 5,
                  tol: float = 0.047, snr_db: float = 30.0) -> Workload:
    """Unfolded hyperspectral cube (pixels x bands) = abundances (Dirichlet
    alpha=1 over the endmembers) x smooth positive spectra (each a sum of five
    Gaussians over the bands: centre U[0,bands), width U[4,40], amplitude
    U[0.1,1]) + white noise at the given SNR; FP32; relative tol.  Stand-in
    for the Indian Pines cube of Sec. 4.2."""
    rng = np.random.default_rng(seed)
    W = rng.dirichlet(np.ones(endmembers), size=pixels)
    b = np.arange(bands, dtype=np.float64)
    S = np.zeros((endmembers, bands))
    for e in range(endmembers):
        for _ in range(5):
            c = rng.uniform(0.0, bands)
            w = rng.uniform(4.0, 40.0)
            a = rng.uniform(0.1, 1.0)
            S[e] += a * np.exp(-((b - c) ** 2) / (2.0 * w * w))
    X = W @ S
    sigma = np.linalg.norm(X) / np.sqrt(X.size * 10.0 ** (snr_db / 10.0))
    A = X + sigma * rng.standard_normal(X.shape)
    A = np.asfortranarray(A.astype(np.float32))
    return Workload(f"hyperspectral_{pixels}x{bands}", A, "f32", tol, 1, seed,
                    note="Dirichlet(1) x 12 smooth spectra + 30 dB noise, FP32",
                    meta={"r_signal": endmembers})


def devils_stairs(n: int = 90, seed: int = 7, step: int = 15) -> np.ndarray:
    """Matrix II of Sec. 4.3: sigma_i = 10^(-4/5 floor((i-1)/step)), Haar U, V."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, n + 1)
    s = 10.0 ** (-0.8 * np.floor((i - 1) / step))
    return low_rank(rng, n, n, s)


def low_rank_plus_noise(n: int = 1000, r: int = 20, alpha: float = 0.005, seed: int = 8) -> np.ndarray:
    """Matrix I of Sec. 4.3 as printed: U diag(sigma) V^T + alpha sigma_r E
    with sigma_1..sigma_r linear from 1 down to 1e-25, sigma_{r+1..n} = 0, E a
    standard Gaussian n x n matrix, Haar U, V (only their first r columns
    meet a nonzero sigma)."""
    rng = np.random.default_rng(seed)
    s = np.linspace(1.0, 1e-25, r)
    A = low_rank(rng, n, n, s)
    return np.asfortranarray(A + alpha * s[-1] * rng.standard_normal((n, n)))


def fast_decay(n: int = 1000, seed: int = 9) -> np.ndarray:
    """Matrix III of Sec. 4.3: U diag(exp(-i/6)) V^T, Haar U, V."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, n + 1)
    return low_rank(rng, n, n, np.exp(-i / 6.0))


def slow_decay(n: int = 1000, seed: int = 10) -> np.ndarray:
    """Matrix IV of Sec. 4.3: U diag(i^-2) V^T, Haar U, V."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, n + 1, dtype=np.float64)
    return low_rank(rng, n, n, i ** -2.0)


def mat2(n: int = 4000, r: int | None = None, seed: int | None = None, tol: float = 1e-8) -> Workload:
    """The strictly rank-deficient test matrix of Sec. 4 (Eq. (mat2)):
    A = U diag(sigma_1..sigma_r, 0..0) V^T, n x n, with U, V orthogonal
    (Haar: only their first r columns meet a nonzero sigma, so those are
    drawn as Haar n x r frames) and sigma the r draws of uniform(0, 1) sorted
    in decreasing order; r = 0.4 n as in the paper's timing tables.  FP64,
    absolute tol 1e-8 (between sigma_r, about 1/r, and the rounding floor
    about 1e-12), Omega seed 7."""
    r = int(0.4 * n) if r is None else int(r)
    rng = np.random.default_rng(1000 + n if seed is None else seed)
    sig = np.sort(rng.uniform(0.0, 1.0, r))[::-1]
    A = low_rank(rng, n, n, sig)
    return Workload(f"mat2_{n}_r{r}", A, "f64", tol, 0, 7,
                    note="Eq. (mat2): Haar U, V, sigma = sorted uniform(0,1), r = 0.4n",
                    meta={"r_true": r})


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)))


def by_name(name: str, **kw) -> Workload:
    table = {
        "exact_rank": exact_rank,
        "image_like": image_like,
        "harmonic": harmonic,
        "pixel_batch": pixel_batch,
        "hyperspectral": hyperspectral,
        "mat2": mat2,
    }
    return table[name](**kw)

"""The oracle on the robustness matrices of Sec. 4.3 (n = 1000), pinned to
LAPACK's singular values: the diagonal of D-hat (the R-values of the
paper's figures) tracks sigma_i within a fixed factor, subspace iteration
(tau = 2, Alg. 2 steps 2-7) tightens it and brings RelErr to the SVD
optimum of the same rank, and with tau = 2 every step of the devil's
stairs shows as a jump of 10^0.8 in the R-values."""
import numpy as np
import pytest

import oracle
import workloads as W

CASES = {
    # name: (generator, tol, tol_mode)
    "I_alpha_0.005": (lambda: W.low_rank_plus_noise(alpha=0.005), 1e-12, 0),
    "I_alpha_0.02": (lambda: W.low_rank_plus_noise(alpha=0.02), 1e-12, 0),
    "III_fast_decay": (W.fast_decay, 1e-8, 1),
    "IV_slow_decay": (W.slow_decay, 1e-3, 1),
    "II_devils_stairs": (lambda: W.devils_stairs(1000), 1e-5, 1),
}


@pytest.fixture(scope="module")
def spectra():
    out = {}
    for name, (make, tol, mode) in CASES.items():
        A = make()
        s = np.linalg.svd(A, compute_uv=False)
        runs = {tau: oracle.eod_abe(A, tol, mode, k=32, seed=5, tau=tau) for tau in (0, 2)}
        out[name] = (s, runs)
    return out


def _log_ratio(run, s):
    r = run["r"]
    d = np.abs(np.diag(run["D"]))
    return np.abs(np.log10(d[:r] / s[:r]))


@pytest.mark.parametrize("name", sorted(CASES))
def test_r_values_track_singular_values(spectra, name):
    s, runs = spectra[name]
    lr0, lr2 = _log_ratio(runs[0], s), _log_ratio(runs[2], s)
    assert runs[0]["r"] == runs[2]["r"]
    assert lr0.max() <= 0.45          # within a factor 2.8 without subspace iteration
    assert lr2.max() <= 0.15          # within a factor 1.42 with tau = 2
    assert lr2.mean() <= lr0.mean()


@pytest.mark.parametrize("name", ["III_fast_decay", "IV_slow_decay", "II_devils_stairs"])
def test_subspace_iteration_reaches_the_svd_optimum(spectra, name):
    s, runs = spectra[name]
    r = runs[2]["r"]
    opt = np.sqrt((s[r:] ** 2).sum() / (s ** 2).sum())   # Eckart-Young error of rank r
    assert runs[2]["rel_err"] >= opt * (1 - 1e-9)
    assert runs[2]["rel_err"] <= 1.1 * opt
    assert runs[2]["rel_err"] <= runs[0]["rel_err"]


def test_devils_stairs_steps_revealed_with_subspace_iteration(spectra):
    s, runs = spectra["II_devils_stairs"]
    run = runs[2]
    r = run["r"]
    d = np.abs(np.diag(run["D"]))
    steps = r // 15
    for j in range(steps):
        blk = d[15 * j: 15 * j + 15]
        assert blk.max() / blk.min() <= 1.01            # a flat step
        if 15 * j + 15 < r:
            assert d[15 * j + 14] / d[15 * j + 15] >= 10 ** 0.75   # the printed 10^0.8 gap


def test_matrix_i_as_printed_is_numerically_rank_19(spectra):
    """With sigma_1..sigma_20 linear from 1 to 1e-25 (as printed), sigma_20
    and the alpha sigma_20 E noise lie far below FP64 resolution, so both
    alphas give the same rank 19 and the same factors."""
    s_a, runs_a = spectra["I_alpha_0.005"]
    s_b, runs_b = spectra["I_alpha_0.02"]
    assert runs_a[0]["r"] == runs_b[0]["r"] == 19
    assert s_a[18] > 0.05 and s_a[19] < 1e-14
    assert np.allclose(runs_a[0]["D"], runs_b[0]["D"], rtol=0, atol=1e-14)

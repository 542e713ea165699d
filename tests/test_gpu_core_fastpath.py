"""The second pass of each core CholQR2 (Alg. 2 steps 9-10) takes the
first-order factor of its near-identity Gram instead of leaf factorisations.
Its Gram is within the threshold only while the first pass's solve is
accurate enough, so a less accurate first solve shows up here as extra leaf
launches, not as wrong results.

Bound on the one-CTA leaf launches of a factorisation that keeps the fast
path: Alg. 1 runs at most two per inner iteration (the rank-test leaf and
the panel's second CholQR pass), and there are blocks + restarts
iterations; the core runs ceil(r / 64) leaves for each of its two first
passes and none for the second passes (64 = the tuned leaf width)."""
import math

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


@pytest.mark.parametrize("form", ["mixed", "mixed_tf32", "plain_f64"])
def test_core_second_passes_take_the_fast_path(eod, form):
    w = W.harmonic(m=2048, n=2048)
    if form == "plain_f64":
        A = torch.from_numpy(np.asfortranarray(w.A.astype(np.float64))).cuda()
        prec = "plain"
    else:
        A = torch.from_numpy(w.A).cuda()
        prec = form
    f = eod.factor(A, w.tol, w.seed, block_k=64, tol_mode="rel", precision=prec)   # warm-up
    f.close()
    torch.cuda.synchronize()
    eod.eod_abe_debug_profile(1)
    try:
        f = eod.factor(A, w.tol, w.seed, block_k=64, tol_mode="rel", precision=prec)
        torch.cuda.synchronize()
        leaves = eod.profile_read(eod.PROF_CHOL)["launches"]
    finally:
        eod.eod_abe_debug_profile(0)
    r, blocks, restarts = f.rank, f.blocks, f.restarts
    f.close()
    assert r > 256   # more than one 256-column panel in the core
    bound = 2 * (blocks + restarts) + 2 * math.ceil(r / 64)
    assert leaves <= bound, (leaves, bound, r, blocks, restarts)

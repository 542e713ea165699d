"""The bounded device-side waits: a wait that nobody completes runs out,
the kernel returns with an error flag, the call reports EOD_ETIMEOUT, and the
context stays usable (a factorisation right after it still matches the
oracle).  The wait is on an mbarrier with no copy or MMA in flight, so no
GPU fault or hang is involved."""
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


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_wait_that_is_completed_returns_ok(eod):
    assert eod.eod_abe_debug_bounded_wait(1_000_000, 1, _stream()) == eod.EOD_OK


@pytest.mark.parametrize("budget", [2_000, 200_000])
def test_wait_that_runs_out_reports_timeout_and_context_survives(eod, budget):
    assert eod.eod_abe_debug_bounded_wait(budget, 0, _stream()) == eod.EOD_ETIMEOUT
    # the context is still usable: a completed wait, then a factorisation
    assert eod.eod_abe_debug_bounded_wait(budget, 1, _stream()) == eod.EOD_OK
    w = W.exact_rank(m=300, n=200, r=12, seed=5)
    ref = oracle.eod_abe(w.A, w.tol, 0, k=16, seed=w.seed)
    f = eod.factor(torch.from_numpy(w.A).cuda(), w.tol, w.seed, block_k=16)
    assert f.rank == ref["r"] == 12
    assert abs(f.rel_err - ref["rel_err"]) <= 1e-10
    f.close()
    torch.cuda.synchronize()

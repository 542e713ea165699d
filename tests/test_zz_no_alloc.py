"""The allocation-free norm entry point, eod_abe_fro_norm_noalloc.

Callers that cannot allocate device memory -- code that runs while another
framework owns the device allocator, real-time loops that forbid allocation
once they are running (an allocation can block or synchronise the device),
services with a fixed memory budget -- use this entry point instead of the
norm inside eod_abe_factor.  Its
scratch is a fixed device array inside the library, so these tests check it
against the existing entry point (the norm_a eod_abe_factor_ex reports) on
two calls in a row, and that a call never sees the previous call's leftovers.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _noalloc(eod, A, dtype_code):
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")    # stale value: the call must clear it
    s = torch.cuda.current_stream()
    st = eod.eod_abe_fro_norm_noalloc(ctypes.c_void_p(A.data_ptr()), A.shape[0], A.shape[1], A.stride(1),
                                      dtype_code, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(flag.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert st == eod.EOD_OK, eod.status_string(st)
    torch.cuda.synchronize()
    return out.item(), flag.item()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_norm_matches_factor_twice(eod, dtype):
    rng = np.random.default_rng(31)
    # a large matrix first, then a small one: the second call must not read
    # partial sums the first call left in the shared scratch
    for m, n in [(3000, 2100), (37, 29)]:
        A = torch.from_numpy(np.asfortranarray(rng.standard_normal((m, n)))).to(dtype).cuda()
        code = eod.EOD_F64 if dtype == torch.float64 else eod.EOD_F32
        # the tolerance only decides the rank; norm_a does not depend on it
        f = eod.factor(A, 0.5, 3, block_k=16, compute_err=False, tol_mode="rel")
        ref = f.norm_a
        f.close()
        for _ in range(2):
            got, bad = _noalloc(eod, A, code)
            assert bad == 0
            # same kernels, grid and reduction order as eod_abe_factor: same bits
            assert got == ref


def test_noalloc_flags_nonfinite_then_recovers(eod):
    A = torch.ones((64, 48), dtype=torch.float64).t().contiguous().t().cuda()
    A[5, 7] = float("nan")
    _, bad = _noalloc(eod, A, eod.EOD_F64)
    assert bad == 1
    with pytest.raises(eod.EodError) as ei:
        eod.factor(A, 1e-6, 1)
    assert ei.value.status == eod.EOD_ENONFINITE
    A[5, 7] = 1.0
    got, bad = _noalloc(eod, A, eod.EOD_F64)
    assert bad == 0 and abs(got - np.sqrt(64 * 48)) <= 1e-13


def test_noalloc_rejects_bad_arguments(eod):
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    assert eod.eod_abe_fro_norm_noalloc(None, 8, 8, 8, 0, P(out), P(flag), None) == eod.EOD_EINVAL
    assert eod.eod_abe_fro_norm_noalloc(P(A), 8, 8, 7, 0, P(out), P(flag), None) == eod.EOD_EINVAL
    assert eod.eod_abe_fro_norm_noalloc(P(A), 8, 8, 8, 5, P(out), P(flag), None) == eod.EOD_EINVAL
    assert eod.eod_abe_fro_norm_noalloc(P(A), 1 << 21, 1 << 20, 1 << 21, 0, P(out), P(flag), None) == eod.EOD_EINVAL

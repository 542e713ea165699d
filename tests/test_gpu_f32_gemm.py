"""The FP32 SIMT product the FP32-data paths use (deflation, CholQR solves,
U = Q Qh), through the autotuner's timing hook with every tile forced and
with the library's own choice, against an FP64 product of the same inputs:
|C - ref| <= K * 2^-22 * (|A| |B|) entrywise (FP32 accumulation), on ragged
shapes, both transposes, beta != 0 and the K splits the plan takes."""
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


def _cm(t):
    return t.t().contiguous().t()


@pytest.mark.parametrize("ts", [0, 16, 32, 64, 128])
@pytest.mark.parametrize("M,N,K,ta,tb,beta", [(8192, 455, 455, 0, 0, 0.0), (1000, 130, 777, 0, 0, 0.5),
                                               (257, 64, 4099, 1, 0, 0.0), (300, 200, 100, 0, 1, -1.0),
                                               (129, 65, 17, 1, 1, 0.0), (4096, 64, 64, 0, 0, 1.0)])
def test_f32_gemm_every_tile(eod, ts, M, N, K, ta, tb, beta):
    g = torch.Generator().manual_seed(M + 3 * N + 7 * K + ts)
    A = _cm(torch.randn((K, M) if ta else (M, K), generator=g)).cuda()
    B = _cm(torch.randn((N, K) if tb else (K, N), generator=g)).cuda()
    C0 = _cm(torch.randn((M, N), generator=g)).cuda()
    C = C0.clone().t().contiguous().t()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    st = eod.eod_abe_debug_f32_gemm(ts, ta, tb, M, N, K, 1.5, P(A), A.stride(1), P(B), B.stride(1), beta, P(C),
                                    C.stride(1), s)
    assert st == eod.EOD_OK
    opA = A.double().t() if ta else A.double()
    opB = B.double().t() if tb else B.double()
    ref = 1.5 * (opA @ opB) + beta * C0.double()
    scale = 1.5 * (opA.abs() @ opB.abs()) + abs(beta) * C0.double().abs()
    err = (C.double() - ref).abs()
    assert torch.isfinite(C).all()
    assert (err <= K * 2.0 ** -22 * scale + 1e-30).all(), float((err / scale).max())

"""Image compression with adaptive rank (Sec. 1's toy example and the
criteria of Sec. 4) through the batched path: ranks, stored entries and
PSNR against the FP64 oracle and the paper's worked example."""
import math

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


def test_rgb_exact_ranks_and_worked_example_storage(eod):
    """Three 220 x 220 channels of ranks 50, 52, 53: the ranks are revealed
    and the factors store 72284 of 145200 entries (Sec. 1), 50.22 % saved."""
    w = W.rgb_image()
    chans = [torch.from_numpy(a).cuda() for a in w.A]
    rep, fs = eod.compress_channels(chans, w.tol, w.seed, block_k=16)
    assert [c["rank"] for c in rep["channels"]] == [50, 52, 53]
    assert rep["total"]["entries"] == 72284 and rep["total"]["entries_full"] == 145200
    assert abs(rep["total"]["saved"] - 0.5022) < 5e-5
    for c in rep["channels"]:
        assert c["rel_err"] < 1e-12 and c["psnr_db"] > 250.0
    for f in fs:
        f.close()


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_lossy_compression_matches_oracle(eod, precision):
    """A lossy tolerance on clipped pixel data: per channel the rank equals
    the oracle's, the stored entries follow, and PSNR agrees to the RelErr
    bar (1e-10 FP64, 1e-4 mixed, both in relative error)."""
    w = W.pixel_batch(count=3, lo=200, hi=300, rlo=20, rhi=40, seed=9, tol=0.02)
    dt = np.float64 if precision == "plain" else np.float32
    chans = [torch.from_numpy(np.asfortranarray(a.astype(dt))).cuda() for a in w.A]
    rep, fs = eod.compress_channels(chans, 0.02, 11, precision=precision, block_k=16)
    bar = 1e-10 if precision == "plain" else 1e-4
    tot_err2, tot_px = 0.0, 0
    for i, (a, c) in enumerate(zip(w.A, rep["channels"])):
        ref = oracle.eod_abe(a.astype(np.float64), 0.02, 1, k=16, seed=11, batch=i)
        assert c["rank"] == ref["r"]
        assert c["entries"] == oracle.storage_entries(a.shape[0], a.shape[1], ref["r"])
        assert abs(c["rel_err"] - ref["rel_err"]) <= bar
        err2 = (ref["rel_err"] * ref["norm_a"]) ** 2
        psnr_ref = 10 * math.log10(255.0 ** 2 * a.size / err2)
        # d PSNR = 20/ln10 * d RelErr / RelErr
        assert abs(c["psnr_db"] - psnr_ref) <= 20 / math.log(10) * bar / ref["rel_err"] * 1.01 + 1e-9
        tot_err2 += err2
        tot_px += a.size
    assert rep["total"]["entries"] == sum(c["entries"] for c in rep["channels"])
    assert abs(rep["total"]["psnr_db"] - 10 * math.log10(255.0 ** 2 * tot_px / tot_err2)) < 0.01
    for f in fs:
        f.close()

"""The leaf width of the blocked Cholesky in the CholQR passes (the tuned key
core_leaf) changes only the blocking of Alg. 2 steps 9-10, never the result
beyond rounding: every width gives the same rank and the same basis Q (Alg. 1
does not use those passes, so Q is bit-identical), the same A_hat = U D V^T,
orthonormal U and V, and the same upper-triangular D up to rounding."""
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


def _with_leaf(eod, tmp_path, nb, fn):
    path = tmp_path / f"core_leaf_{nb}.txt"
    path.write_text(f"core_leaf 1 1000000 0 0 0 0 {nb}\n")
    assert eod.eod_abe_tuning_load(str(path).encode()) == eod.EOD_OK
    try:
        return fn()
    finally:
        eod.eod_abe_tuning_load(None)


def _summary(f):
    U, V, D = f.U.double(), f.V.double(), f.D.clone()
    return {"rank": f.rank, "Q": f.Q.clone(), "Ahat": U @ D @ V.t(), "D": D, "U": U, "V": V,
            "rel_err": f.rel_err}


@pytest.mark.parametrize("case", ["image2048_plain_f64", "harmonic2048_mixed"])
def test_core_leaf_width_changes_only_rounding(eod, tmp_path, case):
    if case == "image2048_plain_f64":
        w = W.image_like()
        A = torch.from_numpy(w.A).cuda()
        prec, k, tol_ahat, tol_d, tol_orth = "plain", 96, 1e-10, 1e-8, 1e-11
    else:
        w = W.harmonic(m=2048, n=2048)
        A = torch.from_numpy(w.A).cuda()
        prec, k, tol_ahat, tol_d, tol_orth = "mixed", 64, 1e-5, 1e-5, 1e-4

    def run():
        f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
        out = _summary(f)
        f.close()
        return out

    ref = _with_leaf(eod, tmp_path, 64, run)
    assert ref["rank"] > 256   # more than one 256-column panel in the core
    nrm = torch.linalg.norm(ref["Ahat"]).item()
    for nb in (16, 32, 128):
        got = _with_leaf(eod, tmp_path, nb, run)
        assert got["rank"] == ref["rank"], nb
        assert torch.equal(got["Q"], ref["Q"]), nb
        assert torch.linalg.norm(got["Ahat"] - ref["Ahat"]).item() <= tol_ahat * nrm, nb
        dn = torch.linalg.norm(ref["D"]).item()
        assert torch.linalg.norm(got["D"] - ref["D"]).item() <= tol_d * dn, nb
        assert torch.equal(torch.triu(got["D"]), got["D"]), nb
        eye = torch.eye(got["rank"], dtype=torch.float64, device="cuda")
        for X in (got["U"], got["V"]):
            assert (X.t() @ X - eye).abs().max().item() <= tol_orth, nb
        assert got["rel_err"] == pytest.approx(ref["rel_err"], rel=1e-9, abs=1e-12), nb

"""The persistent batched launch (csrc/batch.cu) against the FP64 oracle.

FP32 batches go through one persistent launch first: each CTA takes matrices
from a work queue and factors each one start to end (the Alg. 1 block loop
and its stop decision on the device).  Items whose rank exceeds the launch's
capacity (128) are handed to the single-matrix path.  The factor sets the
launch produced say precision EOD_PLAIN (their products are FP32), the
handed-back ones the requested precision, so the tests can tell them apart.

* the unclipped 256-item pixel batch (m, n ~ U[256, 2048], exact ranks 8 to
  128): every item persistent, rank exact and RelErr within 1e-4 of the
  oracle results stored in tests/golden/pixel_batch_unclipped_oracle.json
  (written by tests/golden/make_pixel_batch_oracle.py --unclipped);
* U, D, V, A_hat and the T diagonal entry by entry on a spread of items, at
  the FP32 form's bounds of test_gpu_oracle_fullsize.compare;
* edge cases (zero matrix, 1 x 1, wide, full rank below the capacity, a
  non-finite item beside good ones), a batch mixing persistent and
  handed-back items, run-to-run determinism and freeing in any order;
* pairs of CTAs (the largest items, rows split between the two): the edge
  cases and the mixed batch with every item on pairs and with none, and the
  two schedules agreeing to FP32 rounding.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from test_gpu_oracle_fullsize import compare, RELERR_TOL

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pixel_batch_unclipped_oracle.json")
EOD_PLAIN, EOD_MIXED_BF16 = 0, 1


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    oracle.set_threads(0)
    return eod


@pytest.fixture(autouse=True)
def persistent_on(monkeypatch):
    monkeypatch.delenv("EOD_BATCH_PERSISTENT", raising=False)


def _dev32(a):
    return torch.from_numpy(np.asfortranarray(a, dtype=np.float32)).cuda()


def _dev64(a):
    return torch.from_numpy(np.asfortranarray(a, dtype=np.float64)).cuda()


def _refs(w):
    with open(GOLDEN) as fh:
        doc = json.load(fh)
    assert doc["k"] == 32 and doc["seed"] == w.seed and doc["tol"] == w.tol
    refs = []
    for i, a in enumerate(w.A):
        rec = doc["items"][i]
        h = hashlib.sha256(np.asfortranarray(a, dtype=np.float32).tobytes(order="F")).hexdigest()
        if h != rec["sha256"]:
            ref = oracle.eod_abe(a.astype(np.float64), w.tol, 1, k=32, seed=w.seed, batch=i)
            rec = {"rank": ref["r"], "rel_err": ref["rel_err"], "norm_a": ref["norm_a"]}
        refs.append(rec)
    return refs


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_unclipped_pixel_batch_every_item_vs_oracle(eod, precision):
    w = W.pixel_batch(clip=False)
    refs = _refs(w)
    mats = [_dev32(a) for a in w.A]
    res, st = eod.factor_batched(mats, w.tol, w.seed, block_k=32, tol_mode="rel", precision=precision)
    assert st == [0] * 256
    assert all(f.precision == EOD_PLAIN for f in res)          # every item in the persistent launch
    bad = [(i, res[i].rank, refs[i]["rank"]) for i in range(256) if res[i].rank != refs[i]["rank"]]
    assert not bad, bad[:10]
    drel = max(abs(res[i].rel_err - refs[i]["rel_err"]) for i in range(256))
    assert drel <= RELERR_TOL["plain_f32"], drel
    dnorm = max(abs(res[i].norm_a - refs[i]["norm_a"]) / refs[i]["norm_a"] for i in range(256))
    assert dnorm <= 1e-6, dnorm
    print(f"\n[unclipped pixel batch, persistent] 256/256 ranks equal, max |dRelErr| = {drel:.3g}")


def test_persistent_factors_vs_oracle_elementwise(eod):
    w = W.pixel_batch(clip=False)
    mats = [_dev32(a) for a in w.A]
    res, st = eod.factor_batched(mats, w.tol, w.seed, block_k=32, tol_mode="rel", precision="mixed")
    assert st == [0] * 256
    by_size = sorted(range(256), key=lambda i: w.A[i].size)
    by_rank = sorted(range(256), key=lambda i: res[i].rank)
    for i in sorted({by_size[0], by_size[1], by_size[128], by_size[-1], by_rank[-1], by_rank[0]}):
        A64 = w.A[i].astype(np.float64)
        ref = oracle.eod_abe(A64, w.tol, 1, k=32, seed=w.seed, batch=i)
        assert res[i].precision == EOD_PLAIN
        compare(res[i], ref, _dev64(A64), "plain_f32", f"persistent item {i} {w.A[i].shape}",
                signal=min(10, ref["r"]))


@pytest.mark.parametrize("pair", [None, "0"])
def test_persistent_edge_cases(eod, monkeypatch, pair):
    """Alone, and with every item on a pair of CTAs (EOD_BATCH_PAIR=0: the
    1 x 1 item leaves one rank no rows)."""
    if pair is not None:
        monkeypatch.setenv("EOD_BATCH_PAIR", pair)
    rng = np.random.default_rng(11)
    items = [
        np.zeros((50, 40)),                                   # rank 0
        rng.standard_normal((1, 1)),                          # 1 x 1
        rng.standard_normal((20, 300)),                       # wide, full rank
        rng.standard_normal((130, 100)),                      # full rank at min(m, n) = 100 <= 128
        W.exact_rank(m=300, n=260, r=37, seed=4).A,           # exact rank, two blocks
    ]
    bad = rng.standard_normal((40, 40))
    bad[3, 5] = np.inf
    mats = [_dev32(a) for a in items] + [_dev32(bad)]
    res, st = eod.factor_batched(mats, 1e-4, 6, block_k=32, tol_mode="rel", precision="mixed")
    assert st[:5] == [0] * 5
    assert st[5] == eod.EOD_ENONFINITE and res[5] is None
    for i, a in enumerate(items):
        ref = oracle.eod_abe(a.astype(np.float32).astype(np.float64), 1e-4, 1, k=32, seed=6, batch=i)
        f = res[i]
        assert f.precision == EOD_PLAIN
        assert f.rank == ref["r"], (i, f.rank, ref["r"])
        assert abs(f.rel_err - ref["rel_err"]) <= 1e-4, (i, f.rel_err, ref["rel_err"])
    assert res[0].rank == 0 and res[0].rel_err == 0.0 and res[0].U.numel() == 0
    assert res[4].rank == 37


@pytest.mark.parametrize("pair", [None, "0", "2"])
def test_mixed_batch_persistent_and_handed_back(eod, monkeypatch, pair):
    """Low-rank items finish in the persistent launch; a full-rank 300 x 260
    item exceeds its capacity and is factored by the single-matrix path with
    the requested precision.  Every item matches the oracle's rank: with the
    default split between pairs and single CTAs, every item on pairs, none."""
    if pair is not None:
        monkeypatch.setenv("EOD_BATCH_PAIR", pair)
    rng = np.random.default_rng(3)
    items = [W.exact_rank(m=400 + 10 * i, n=350, r=20 + 9 * i, seed=20 + i).A for i in range(4)]
    items.insert(2, rng.standard_normal((300, 260)))
    mats = [_dev32(a) for a in items]
    res, st = eod.factor_batched(mats, 1e-3, 8, block_k=32, tol_mode="rel", precision="mixed")
    assert st == [0] * 5
    assert [f.precision for f in res] == [EOD_PLAIN, EOD_PLAIN, EOD_MIXED_BF16, EOD_PLAIN, EOD_PLAIN]
    for i, a in enumerate(items):
        ref = oracle.eod_abe(a.astype(np.float32).astype(np.float64), 1e-3, 1, k=32, seed=8, batch=i)
        assert res[i].rank == ref["r"], (i, res[i].rank, ref["r"])
        assert abs(res[i].rel_err - ref["rel_err"]) <= 1e-4
    assert res[2].rank == 260


def test_pairs_and_single_ctas_agree(eod, monkeypatch):
    """The same batch with every item on a pair of CTAs and with none: equal
    ranks, RelErr and factors to FP32 rounding (the two differ only in the
    order of the cross-row sums)."""
    mats = [_dev32(W.exact_rank(m=900 + 57 * i, n=700 + 33 * i, r=10 + 9 * i, seed=30 + i).A) for i in range(8)]
    monkeypatch.setenv("EOD_BATCH_PAIR", "0")
    a, st_a = eod.factor_batched(mats, 1e-5, 3, block_k=32, tol_mode="rel", precision="mixed")
    monkeypatch.setenv("EOD_BATCH_PAIR", "2")
    b, st_b = eod.factor_batched(mats, 1e-5, 3, block_k=32, tol_mode="rel", precision="mixed")
    assert st_a == st_b == [0] * 8
    for x, y in zip(a, b):
        assert x.precision == y.precision == EOD_PLAIN
        assert x.rank == y.rank and x.blocks == y.blocks
        assert abs(x.rel_err - y.rel_err) <= 1e-6
        ax, ay = x.reconstruct(), y.reconstruct()
        assert (torch.linalg.norm(ax - ay) / torch.linalg.norm(ay)).item() <= 1e-5


def test_persistent_refuses_tol_below_the_fp32_floor(eod):
    """eps below 1e-5 ||A||_F: EOD_EPRECISION, as a single FP32 or mixed call
    answers (the FP32 rounding of the sketch reaches |T(l,l)| there)."""
    a = W.exact_rank(m=200, n=150, r=10, seed=2).A
    res, st = eod.factor_batched([_dev32(a), _dev32(a)], 1e-6, 1, block_k=16, tol_mode="rel", precision="mixed")
    assert st == [eod.EOD_EPRECISION] * 2 and res == [None, None]
    with pytest.raises(eod.EodError):
        eod.factor(_dev32(a), 1e-6, 1, block_k=16, tol_mode="rel", precision="mixed")


def test_persistent_is_deterministic_and_frees_in_any_order(eod):
    mats = [_dev32(W.exact_rank(m=200 + 31 * i, n=180 + 17 * i, r=5 + 7 * i, seed=i).A) for i in range(12)]
    a, st_a = eod.factor_batched(mats, 1e-5, 2, block_k=16, tol_mode="rel", precision="plain")
    b, st_b = eod.factor_batched(mats, 1e-5, 2, block_k=16, tol_mode="rel", precision="plain")
    assert st_a == st_b == [0] * 12
    for x, y in zip(a, b):
        assert x.precision == EOD_PLAIN
        assert x.rank == y.rank and x.rel_err == y.rel_err
        assert torch.equal(x.U, y.U) and torch.equal(x.V, y.V) and torch.equal(x.D, y.D)
    # release half of one batch in a scrambled order; the rest stay valid
    order = [7, 2, 11, 4, 0, 9]
    keep = [i for i in range(12) if i not in order]
    for i in order:
        a[i].close()
    for i in keep:
        Ah = a[i].reconstruct()
        ref = b[i].reconstruct()
        assert torch.equal(Ah, ref)
    for i in keep:
        a[i].close()
    for f in b:
        f.close()

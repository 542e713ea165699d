"""Writes pixel_batch_oracle.json: the FP64 oracle's result on every item of
the 256-matrix pixel batch (m, n ~ U[256, 2048], r ~ U[8, 128], s_i =
255 exp(-i/(r/4)), clipped to [0, 255], FP32 storage; relative tol 1e-3,
k = 32, Omega seed 4, batch index = item index), the batched configuration of
the benchmark.  With --unclipped: pixel_batch_unclipped_oracle.json, the same
batch without the clipping (every item of exact rank r <= 128, the regime of
the persistent batched launch).

Only the oracle and the seeded input generators are called.  Each record
carries the SHA-256 of the item's FP32 bytes, so a test that reads the file
can tell whether the generator produced the same matrix on its machine (and
recompute the oracle for any item where it did not).

  python tests/golden/make_pixel_batch_oracle.py [--threads N] [--unclipped]

The oracle runs single-threaded per item, items in parallel (ctypes releases
the GIL during the oracle call), so the file does not depend on N.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
K = 32


def item_hash(a: np.ndarray) -> str:
    return hashlib.sha256(np.asfortranarray(a, dtype=np.float32).tobytes(order="F")).hexdigest()


def oracle_record(a: np.ndarray, tol: float, seed: int, i: int) -> dict:
    ref = oracle.eod_abe(a.astype(np.float64), tol, 1, k=K, seed=seed, batch=i)
    td = np.abs(ref["tdiag"])
    eps = ref["eps"]
    tested = td[: ref["r"] + 1] if ref["r"] < min(a.shape) else td
    margin = float(np.min(np.abs(np.log10(np.maximum(tested, 1e-300) / eps)))) if eps > 0 else math.inf
    return {"i": i, "m": int(a.shape[0]), "n": int(a.shape[1]), "sha256": item_hash(a), "rank": int(ref["r"]),
            "rel_err": ref["rel_err"], "norm_a": ref["norm_a"], "eps": eps, "t_margin": margin}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    p.add_argument("--unclipped", action="store_true")
    args = p.parse_args()
    clip = not args.unclipped
    w = W.pixel_batch(clip=clip)
    out = os.path.join(HERE, "pixel_batch_oracle.json" if clip else "pixel_batch_unclipped_oracle.json")
    oracle.set_threads(1)
    with cf.ThreadPoolExecutor(max_workers=args.threads) as ex:
        recs = list(ex.map(lambda ia: oracle_record(ia[1], w.tol, w.seed, ia[0]), enumerate(w.A)))
    desc = "clipped [0,255]" if clip else "not clipped"
    doc = {"workload": f"pixel batch 256: m,n~U[256,2048], r~U[8,128], s_i=255exp(-i/(r/4)), {desc}, FP32",
           "tol": w.tol, "tol_mode": "relative", "k": K, "seed": w.seed,
           "generator": "workloads.pixel_batch()" if clip else "workloads.pixel_batch(clip=False)",
           "items": recs}
    with open(out, "w") as fh:
        json.dump(doc, fh, indent=0)
        fh.write("\n")
    print(f"wrote {out}: {len(recs)} items, ranks {min(r['rank'] for r in recs)}..{max(r['rank'] for r in recs)}")


if __name__ == "__main__":
    main()

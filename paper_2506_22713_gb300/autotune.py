"""Autotuner of the library's tile shapes and block sizes.

It times candidate settings on the GPU through the C ABI and writes the
table the library reads at load (tuning.txt beside libeodabe.so; format and
keys in include/eod_abe.h, eod_abe_tuning_load):

* f32_tile       the tile of the FP32 SIMT product, per (M, N, K): every
                 candidate tile (16, 32, 64, 128) is timed on the product
                 shapes the FP32-data paths run (the deflation, the CholQR
                 solves, U = Q Qh, ...), device time from the library's
                 per-launch CUDA events;
* block_k        k of Alg. 1 per precision form and size, for callers that
                 pass block_k = 0: whole factorisations of the workloads of
                 each size class timed with k in 16 ... 128 (CUDA events,
                 median of the repetitions, L2 flushed between them);
* batch_workers  the worker streams of the batched entry point on the
                 256-matrix pixel batch;
* batch_block_k  k of Alg. 1 for the items of a batched call that run on
                 the worker streams (block_k = 0): the whole clipped pixel
                 batch timed per k and form (under concurrency fewer,
                 wider blocks pay more than for one matrix of that size);
* core_leaf      the leaf width (16, 32, 64, 128) of the blocked Cholesky in
                 the CholQR passes, per Gram width p: whole factorisations
                 timed with a one-row table loaded per candidate (a narrower
                 leaf is faster per pivot but adds panel products).

Every row covers a range around the measured case (a factor of about 1.5
to each side of the sizes); of the rows that hold a case the nearest wins
(log distance to the centre of each range).

    python -m paper_2506_22713_gb300.autotune --out PATH [--quick] [--skip ...] [--merge]
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import sys
import time

FORMS = {"plain_f64": 0, "plain_f32": 1, "mixed": 2, "mixed_tf32": 3}


def _eod():
    import paper_2506_22713_gb300 as eod
    return eod


def _range(v, lo=0.67, hi=1.5):
    return max(1, int(v * lo)), int(v * hi) + 1


# ------------------------------------------------------------- FP32 tiles --
# (M, N, K, ta, tb): the FP32 products of the mixed and plain FP32 paths on
# the 8192^2 harmonic (rank 455) and 2048^2 image (rank 2037) workloads, at
# k = 64 and at the block sizes the table's block_k rows pick (96 mixed, 128
# plain): the deflation's K (or M) grows with the basis, so two points each
F32_SHAPES = [
    (8192, 96, 96, 0, 0),     # P = Y R^-1, k = 96
    (8192, 96, 192, 0, 0),    # Y -= Q S, k = 96
    (8192, 96, 384, 0, 0),
    (192, 96, 8192, 1, 0),    # S = Q^T Y, k = 96
    (384, 96, 8192, 1, 0),
    (8192, 128, 256, 0, 0),   # Y -= Q S, k = 128
    (256, 128, 8192, 1, 0),   # S = Q^T Y, k = 128
    (2048, 96, 96, 0, 0),
    (2048, 96, 768, 0, 0),
    (768, 96, 2048, 1, 0),
    (8192, 455, 455, 0, 0),   # U = Q Qh
    (8192, 256, 256, 0, 0),   # CholQR solve, diagonal panel
    (8192, 199, 256, 0, 0),   # CholQR solve, trailing columns
    (8192, 64, 64, 0, 0),     # P = Y R^-1
    (8192, 64, 384, 0, 0),    # Y -= Q S
    (384, 64, 8192, 1, 0),    # S = Q^T Y
    (2048, 2037, 2037, 0, 0),
    (2048, 1781, 256, 0, 0),
    (2048, 256, 256, 0, 0),
    (2048, 64, 1536, 0, 0),
    (1536, 64, 2048, 1, 0),
    (2048, 64, 64, 0, 0),
]


def tune_f32_tiles(eod, torch, reps=5, shapes=F32_SHAPES):
    rows, notes = [], []
    g = torch.Generator(device="cuda").manual_seed(11)
    s = torch.cuda.current_stream()
    for (M, N, K, ta, tb) in shapes:
        # column-major buffers of A (op(A) = M x K) and B (op(B) = K x N)
        rowsA, colsA = (M, K) if not ta else (K, M)
        rowsB, colsB = (K, N) if not tb else (N, K)
        A = torch.randn((colsA, rowsA), generator=g, device="cuda").t()
        B = torch.randn((colsB, rowsB), generator=g, device="cuda").t()
        C = torch.zeros((N, M), device="cuda").t()
        P = lambda t: t.data_ptr()
        res = {}
        for ts in (16, 32, 64, 128):
            def run():
                st = eod.eod_abe_debug_f32_gemm(ts, ta, tb, M, N, K, 1.0, P(A), rowsA, P(B), rowsB, 0.0, P(C), M,
                                                s.cuda_stream)
                assert st == eod.EOD_OK, st
            run()
            eod.eod_abe_debug_profile(1)
            for _ in range(reps):
                run()
            pr = eod.profile_read(eod.PROF_GEMM_SIMT32)
            eod.eod_abe_debug_profile(0)
            res[ts] = 1e3 * pr["ms"] / reps
        best = min(res, key=res.get)
        m0, m1 = _range(M)
        n0, n1 = _range(N)
        k0, k1 = _range(K)
        rows.append(("f32_tile", m0, m1, n0, n1, k0, k1, best))
        notes.append(f"f32_tile M={M} N={N} K={K} t{'T' if ta else 'N'}{'T' if tb else 'N'}: "
                     + ", ".join(f"{t}:{v:.1f}us" for t, v in res.items()) + f" -> {best}")
        del A, B, C
    return rows, notes


# ---------------------------------------------------------------- block_k --
def _block_k_cases():
    import numpy as np
    import workloads as W

    def harm():
        return W.harmonic()

    def img():
        return W.image_like()

    def hyp():
        return W.hyperspectral()

    return [
        ("harmonic 8192^2", harm, ["mixed", "mixed_tf32", "plain_f64", "plain_f32"], (16, 32, 64, 96, 128)),
        ("image 2048^2", img, ["plain_f64", "plain_f32", "mixed", "mixed_tf32"], (32, 64, 96, 128)),
        ("hyperspectral 262144x224", hyp, ["mixed", "mixed_tf32", "plain_f64", "plain_f32"], (8, 16, 32, 64)),
    ]


def tune_block_k(eod, torch, reps=3, quick=False):
    import numpy as np

    rows, notes = [], []
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name, make, forms, ks in _block_k_cases():
        w = make()
        m, n = w.A.shape
        A32 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float32))).cuda()
        A64 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float64))).cuda()
        for form in forms:
            A = A64 if form == "plain_f64" else A32
            prec = {"plain_f64": "plain", "plain_f32": "plain", "mixed": "mixed", "mixed_tf32": "mixed_tf32"}[form]
            res = {}
            for k in ks:
                if k > min(m, n):
                    continue
                times = []
                for rep in range(reps + 1):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
                    e1.record()
                    e1.synchronize()
                    f.close()
                    if rep:
                        times.append(e0.elapsed_time(e1))
                res[k] = statistics.median(times)
            best = min(res, key=res.get)
            m0, m1 = _range(m, 0.5, 2.0)
            n0, n1 = _range(n, 0.5, 2.0)
            rows.append(("block_k", FORMS[form], FORMS[form], m0, m1, n0, n1, best))
            notes.append(f"block_k {name} {form}: " + ", ".join(f"k={k}:{v:.2f}ms" for k, v in res.items())
                         + f" -> {best}")
            if quick:
                break
        del A32, A64
        torch.cuda.empty_cache()
    return rows, notes


# ---------------------------------------------------------- batch workers --
def tune_batch_workers(eod, torch, candidates=(4, 8, 12, 16, 24, 32)):
    import numpy as np
    import workloads as W

    w = W.pixel_batch()
    mats = [torch.from_numpy(a).cuda() for a in w.A]
    res = {}
    old = os.environ.get("EOD_BATCH_STREAMS")
    try:
        for c in candidates:
            os.environ["EOD_BATCH_STREAMS"] = str(c)
            r, st = eod.factor_batched(mats, w.tol, w.seed, block_k=32, tol_mode="rel", precision="mixed")
            del r
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r, st = eod.factor_batched(mats, w.tol, w.seed, block_k=32, tol_mode="rel", precision="mixed")
            torch.cuda.synchronize()
            res[c] = time.perf_counter() - t0
            assert all(x == 0 for x in st)
            del r
    finally:
        if old is None:
            os.environ.pop("EOD_BATCH_STREAMS", None)
        else:
            os.environ["EOD_BATCH_STREAMS"] = old
    best = min(res, key=res.get)
    mm = int(np.mean([a.shape[0] for a in w.A]))
    nn = int(np.mean([a.shape[1] for a in w.A]))
    row = ("batch_workers", 64, 4096, *_range(mm, 0.5, 2.0), *_range(nn, 0.5, 2.0), best)
    note = "batch_workers pixel batch 256 mixed: " + ", ".join(f"{c}:{v * 1e3:.0f}ms" for c, v in res.items()) \
           + f" -> {best}"
    return [row], [note]


# ---------------------------------------------------------- batch block_k --
def tune_batch_block_k(eod, torch, ks=(32, 64, 96, 128)):
    import numpy as np
    import workloads as W

    w = W.pixel_batch()
    mm = int(np.mean([a.shape[0] for a in w.A]))
    nn = int(np.mean([a.shape[1] for a in w.A]))
    rows, notes = [], []
    for form, dtype, prec in (("mixed", np.float32, "mixed"), ("plain_f64", np.float64, "plain")):
        mats = [torch.from_numpy(np.asfortranarray(a.astype(dtype))).cuda() for a in w.A]
        res = {}
        for k in ks:
            r, st = eod.factor_batched(mats, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
            del r
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r, st = eod.factor_batched(mats, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
            torch.cuda.synchronize()
            res[k] = time.perf_counter() - t0
            assert all(x == 0 for x in st)
            del r
        best = min(res, key=res.get)
        rows.append(("batch_block_k", FORMS[form], FORMS[form], *_range(mm, 0.5, 2.0), *_range(nn, 0.5, 2.0), best))
        notes.append(f"batch_block_k pixel batch 256 {form}: " + ", ".join(f"k={k}:{v * 1e3:.0f}ms" for k, v in res.items())
                     + f" -> {best}")
        del mats
        torch.cuda.empty_cache()
    return rows, notes


# -------------------------------------------------------------- core leaf --
def tune_core_leaf(eod, torch, tmp_path, widths=(16, 32, 64, 128), reps=3):
    import numpy as np
    import workloads as W

    # (name, workload, precision, dtype, k): the block sizes the block_k rows pick
    cases = [("harmonic 8192^2", W.harmonic, "mixed", np.float32, 96),
             ("harmonic 8192^2", W.harmonic, "plain", np.float64, 128),
             ("image 2048^2", W.image_like, "plain", np.float64, 96)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rows, notes = [], []
    try:
        for name, make, prec, dtype, k in cases:
            w = make()
            A = torch.from_numpy(np.asfortranarray(w.A.astype(dtype))).cuda()
            res, rank = {}, None
            for nb in widths:
                with open(tmp_path, "w") as fh:
                    fh.write(f"core_leaf 1 1000000 0 0 0 0 {nb}\n")
                if eod.eod_abe_tuning_load(tmp_path.encode()) != eod.EOD_OK:
                    raise RuntimeError("tuning table did not load")
                times = []
                for rep in range(reps + 1):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
                    e1.record()
                    e1.synchronize()
                    rank = f.rank
                    f.close()
                    if rep:
                        times.append(e0.elapsed_time(e1))
                res[nb] = statistics.median(times)
            best = min(res, key=res.get)
            form = "plain_f64" if dtype == np.float64 else prec
            rows.append(("core_leaf", *_range(rank), 0, 0, 0, 0, best))
            notes.append(f"core_leaf {name} {form} (p = {rank}): " + ", ".join(f"{nb}:{v:.2f}ms" for nb, v in res.items())
                         + f" -> {best}")
            del A
            torch.cuda.empty_cache()
    finally:
        if os.path.exists(tmp_path):
            os.remove(tmp_path)
        eod.eod_abe_tuning_load((tmp_path + ".none").encode())
    return rows, notes


def kept_rows(path, keys):
    """The rows and '# measured:' notes of the given keys in the table at
    path (what --merge keeps for the parts it skips)."""
    rows, notes = [], []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("# measured: "):
                note = line[len("# measured: "):]
                if note.split(" ", 1)[0] in keys:
                    notes.append(note)
            elif line and not line.startswith("#"):
                f = line.split()
                if f[0] in keys:
                    rows.append(tuple([f[0]] + [int(x) for x in f[1:]]))
    return rows, notes


def write_table(path, rows, notes, meta):
    with open(path, "w") as fh:
        fh.write("# Tuned parameters of libeodabe.so, written by paper_2506_22713_gb300/autotune.py\n")
        for k, v in meta.items():
            fh.write(f"# {k}: {v}\n")
        fh.write("# key a_lo a_hi b_lo b_hi c_lo c_hi value\n")
        for note in notes:
            fh.write(f"# measured: {note}\n")
        for r in rows:
            fh.write(" ".join(str(x) for x in r) + "\n")


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--out", required=True, help="where to write the table")
    p.add_argument("--quick", action="store_true", help="fewer cases (smoke run)")
    p.add_argument("--skip", default="", help="comma list of f32_tile,block_k,batch_workers,batch_block_k,core_leaf to skip")
    p.add_argument("--merge", action="store_true",
                   help="keep the rows (and their notes) of skipped parts from the table already at --out")
    args = p.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    eod = _eod()
    # measure against the fixed defaults, not an older table
    eod.eod_abe_tuning_load(os.path.join(args.out + ".none").encode())
    skip = set(filter(None, args.skip.split(",")))
    rows, notes = [], []
    t0 = time.time()
    if "f32_tile" not in skip:
        r, n = tune_f32_tiles(eod, torch, shapes=F32_SHAPES[:3] if args.quick else F32_SHAPES)
        rows += r
        notes += n
    if "block_k" not in skip:
        r, n = tune_block_k(eod, torch, quick=args.quick)
        rows += r
        notes += n
    if "batch_block_k" not in skip:
        r, n = tune_batch_block_k(eod, torch, ks=(32, 96) if args.quick else (32, 64, 96, 128))
        rows += r
        notes += n
    if "core_leaf" not in skip:
        r, n = tune_core_leaf(eod, torch, args.out + ".leaf", widths=(32, 64) if args.quick else (16, 32, 64, 128),
                              reps=1 if args.quick else 3)
        rows += r
        notes += n
    if "batch_workers" not in skip:
        r, n = tune_batch_workers(eod, torch, candidates=(8, 16) if args.quick else (4, 8, 12, 16, 24, 32))
        rows += r
        notes += n
    if args.merge and os.path.exists(args.out):
        r, n = kept_rows(args.out, skip)
        rows += r
        notes += n
    meta = {"when": datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%dT%H:%M:%SZ"),
            "gpu": torch.cuda.get_device_name(0), "torch": torch.__version__,
            "seconds": f"{time.time() - t0:.0f}"}
    write_table(args.out, rows, notes, meta)
    print(json.dumps({"rows": len(rows), "out": args.out, "notes": notes}))


if __name__ == "__main__":
    main()

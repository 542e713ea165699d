#!/usr/bin/env python3
"""Benchmark of power-free EOD-ABE on one GB300 (or N replicas).

Workload: the image-like 2048 x 2048 matrix (rank-150 U diag(255 i^-1.5) V^T
with Haar U, V plus Gaussian noise of std 1e-4 * 255), relative tolerance
1e-3, FP64 storage, plain FP64 path, k = 64.  One step = one complete
factorisation through the C ABI (Alg. 1 + Alg. 2 steps 8-11 + the
reconstruction error), inputs resident in HBM.  The metric is GFLOP/s of the
paper's cost model (Sec. 3.4) for tau = 0 plus the 2mnr of the
reconstruction; the same line reports the FP32-storage plain form, the
roofline of the dominant kernel, the host-buffer end-to-end rate and the
FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it runs under torch.distributed.run, one independent replica per
GPU (the single-matrix path does not shard), and reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EOD-ABE GFLOP/s & % roofline, mixed vs plain FP64 at rel-err ≤1e-4"
WORKLOAD = "image-like 2048x2048, rank-150 s_i=255 i^-1.5 + noise 1e-4*s_1, tol 1e-3 relative"
M = N = 2048
BLOCK_K = 64
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2070 MHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# FP32 (FFMA) peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]) * 1e3, float(d["hbm_gbs"]), "measured"
    except Exception:
        return 1.9e6, 6800.0, "fallback"
L2_BYTES = 129 * 1024 * 1024
# kernel kinds of the library's profile counters, in PROF_* order
KINDS = ["gemm_simt", "chol", "omega", "stream", "tc_gemm", "oz_gemm", "oz_slice"]
# BF16 slice-pair products per emulated FP64 multiply-add (8 slices, s + t <= 7)
OZ_PAIRS = 36


PROFILE_CASES = {
    "image2048_f64": ("image_like", {}, "f64", "plain", 64),
    "image2048_mixed": ("image_like", {}, "f32", "mixed", 64),
    "harmonic8192_mixed": ("harmonic", {}, "f32", "mixed", 64),
    "hyperspectral_mixed": ("hyperspectral", {}, "f32", "mixed", 16),
}


def run_profile_case(name):
    """One warm-up and one factorisation of a named workload, nothing timed:
    the command ncu captures (NVTX ranges eod.norm, eod.basis_ext_block,
    eod.projection, eod.reconstruction_error, eod.core select the phase)."""
    import numpy as np
    import torch

    import paper_2506_22713_gb300 as eod
    import workloads as W

    gen, kw, dt, prec, k = PROFILE_CASES[name]
    w = W.by_name(gen, **kw)
    A = torch.from_numpy(np.asfortranarray(w.A.astype(np.float64 if dt == "f64" else np.float32))).cuda()
    for _ in range(2):
        f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
        r, rel = f.rank, f.rel_err
        f.close()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "rank": r, "rel_err": rel}))


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the mixed-vs-plain comparison workloads")
    p.add_argument("--profile-case", choices=sorted(PROFILE_CASES), default=None,
                   help="run one warm-up and one factorisation of a named workload (for ncu) and exit")
    return p.parse_args()


def _max_over_ranks(x, dist, device):
    """The largest value of a host float over the ranks (an all-reduce on
    `device`: "cuda" under NCCL, "cpu" under gloo); x itself with one rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- oracle --
def oracle_sample(A_np, eps, seconds):
    """Times the FP64 oracle's Alg. 1 on the first b blocks of the same matrix
    (b chosen so the run takes about `seconds`); returns (GFLOP/s, sample text,
    elapsed).  The numerator is the cost model's Alg. 1 term mnr + 4mrk
    multiply-adds for the r = b*k columns processed."""
    import oracle
    m, n = A_np.shape
    t0 = time.perf_counter()
    oracle.basis_ext(A_np, eps, k=BLOCK_K, seed=2, max_blocks=1)
    t1 = time.perf_counter() - t0
    b = max(1, min(int(seconds / max(t1, 1e-6)), min(m, n) // BLOCK_K))
    t0 = time.perf_counter()
    Q, _ = oracle.basis_ext(A_np, eps, k=BLOCK_K, seed=2, max_blocks=b)
    el = time.perf_counter() - t0
    r = Q.shape[1]
    flops = 2.0 * (m * n * r + 4.0 * m * r * BLOCK_K)
    sample = (f"FP64 oracle (plain C, 1 thread), Alg. 1 on the first {b} blocks (k={BLOCK_K}, {r} columns) "
              f"of the same {m}x{n} matrix; GFLOP/s of the cost model's mnr+4mrk term")
    return flops / el / 1e9, sample, el


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _traffic_for(kind_name, source_files):
    """DRAM bytes per launch recorded from an ncu capture in profiles/, valid
    only while the kernel source is unchanged (sha256 recorded beside it)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for f in source_files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
    for line in open(path):
        parts = line.split(None, 3)
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kind_name and parts[1] == digest:
            return float(parts[2]), (parts[3].strip() if len(parts) > 3 else "")
    return None


# ---------------------------------------------------------------- our arm --
def run_ours(args):
    import numpy as np
    import torch

    import paper_2506_22713_gb300 as eod
    import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = W.image_like()                          # same seeded matrix on every replica
    A_np = w.A
    A = torch.from_numpy(A_np).cuda()
    A32 = torch.from_numpy(np.asfortranarray(A_np.astype(np.float32))).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(Ain):
        f = eod.factor(Ain, w.tol, w.seed, block_k=BLOCK_K, tol_mode="rel")
        r, rel = f.rank, f.rel_err
        f.close()
        return r, rel

    def timed(Ain, steps, warmup, profile=False):
        for _ in range(warmup):
            step(Ain)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = eod.eod_abe_debug_launch_count()
        if profile:
            eod.eod_abe_debug_profile(1)
        total_ms, info = 0.0, None
        for _ in range(steps):
            flush.zero_()                       # evict A from the 129 MB L2 between steps
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            info = step(Ain)
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
        torch.cuda.synchronize()
        prof = eod.profile_read(eod.PROF_OZ_GEMM) if profile else None
        kinds = {k: eod.profile_read(i) for i, k in enumerate(KINDS)} if profile else None
        if profile:
            eod.eod_abe_debug_profile(0)
        launches = eod.eod_abe_debug_launch_count() - launches0
        total_ms = _max_over_ranks(total_ms, dist, "cuda")
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        return total_ms, info, prof, kinds, launches

    clocks = ClockSampler(local)
    clocks.start()
    total_ms, (r, rel), prof, kinds, launches = timed(A, args.steps, args.warmup, profile=True)
    clk = clocks.stop()
    flops = eod.model_flops(M, N, r, BLOCK_K, True)
    value = ws * args.steps * flops / (total_ms / 1e3) / 1e9
    ms_step = total_ms / args.steps

    # FP32-storage plain form on the same matrix (context)
    t32, (r32, rel32), _, _, _ = timed(A32, max(2, args.steps // 2), 1)
    v32 = ws * max(2, args.steps // 2) * eod.model_flops(M, N, r32, BLOCK_K, True) / (t32 / 1e3) / 1e9

    # Alg. 2 with tau = 1, 2 subspace iterations on the same matrix (context;
    # the cost model adds tau (2mnr + 2mr^2 + 2nr^2) multiply-adds, Sec. 3.4)
    sub = {}
    for tau in (1, 2):
        def step_tau(Ain, tau=tau):
            f = eod.factor(Ain, w.tol, w.seed, block_k=BLOCK_K, tol_mode="rel", power_iters=tau)
            out = (f.rank, f.rel_err)
            f.close()
            return out
        for _ in range(2):
            step_tau(A)
        torch.cuda.synchronize()
        tt = 0.0
        nst = max(2, args.steps // 2)
        for _ in range(nst):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rt, relt = step_tau(A)
            e1.record(stream)
            e1.synchronize()
            tt += e0.elapsed_time(e1)
        mst = tt / nst
        fl = eod.model_flops(M, N, rt, BLOCK_K, True) + 2.0 * tau * (2.0 * M * N * rt + 2.0 * M * rt * rt +
                                                                     2.0 * N * rt * rt)
        sub[f"tau{tau}"] = {"ms_per_step": mst, "gflops": fl / (mst / 1e3) / 1e9, "rank": rt, "rel_err": relt}

    # end to end through the host-buffer entry point
    Ah = torch.from_numpy(A_np).pin_memory()
    cap = min(M, N)
    Uh = torch.empty((cap, M), dtype=torch.float64).pin_memory().t()
    Dh = torch.empty((cap, cap), dtype=torch.float64).pin_memory().t()
    Vh = torch.empty((cap, N), dtype=torch.float64).pin_memory().t()
    for _ in range(args.warmup):
        eod.factor_host(Ah, w.tol, w.seed, block_k=BLOCK_K, tol_mode="rel", U_out=Uh, D_out=Dh, V_out=Vh)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        re2e, _ = eod.factor_host(Ah, w.tol, w.seed, block_k=BLOCK_K, tol_mode="rel", U_out=Uh, D_out=Dh, V_out=Vh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = _max_over_ranks(e2e_s, dist, "cuda")
    e2e_val = ws * args.steps * eod.model_flops(M, N, re2e, BLOCK_K, True) / e2e_s / 1e9

    # roofline of the dominant kernel: the FP64 GEMM emulated on tcgen05
    bf16_peak, _, peak_src = _measured_peaks()
    oz_peak = bf16_peak / OZ_PAIRS
    achieved = prof["flops"] / (prof["ms"] / 1e3) / 1e9 if prof and prof["ms"] > 0 else None
    tr = _traffic_for("oz_gemm", ["paper_2506_22713_gb300/csrc/oz_gemm.cu", "paper_2506_22713_gb300/csrc/tc_ptx.cuh"])
    traffic = tr[0] if tr else None
    per_launch = (prof["flops"] / prof["launches"]) if prof and prof["launches"] else None
    roofline = {
        "bound": "tensor",
        "kernel": "oz_gemm (FP64 GEMM as 36 exact BF16 slice-pair products on tcgen05, FP64 accumulation)",
        "achieved": achieved,
        "peak": oz_peak,
        "unit": "GFLOP/s",
        "frac": (achieved / oz_peak) if achieved else None,
        "peak_source": f"{peak_src} bf16 burst {bf16_peak:.0f} GFLOP/s (MEASURED_PEAKS.json) / {OZ_PAIRS} "
                       "slice-pair products per FP64 multiply-add",
        "achieved_bf16_equivalent": achieved * OZ_PAIRS if achieved else None,
        "traffic": traffic,
        "traffic_launch": tr[1] if tr else None,
        "launches": prof["launches"] if prof else None,
        "flops_per_launch": per_launch,
        "share_of_step": (prof["ms"] / total_ms) if prof else None,
        "fp64_simt_peak": FP64_PEAK_GFLOPS,
    }
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "GFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded image-like low-rank + noise; no dataset)",
        "config": {"workload": WORKLOAD + ", FP64 plain, k=64", "m": M, "n": N, "rank": r, "rel_err": rel,
                   "parallelism": f"replicas x{ws}", "l2": "flushed between timed steps (256 MB write)"},
        "roofline": roofline,
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * M * N,
                "d2h_bytes_per_step": 8 * (M * re2e + N * re2e + re2e * re2e)},
        "gpu_launches": int(launches),
        "kernel_ms": {k: round(v["ms"], 3) for k, v in (kinds or {}).items()},
        "forms": {"f32_plain": {"value": v32, "unit": "GFLOP/s", "rank": r32, "rel_err": rel32,
                                "ms_per_step": t32 / max(2, args.steps // 2)}},
        "subspace_iteration_f64": sub,
        "clocks": clk,
    }
    if not args.no_compare:
        comp, troof = compare_forms(eod, 3, 1, flush)
        out["mixed_vs_plain"] = comp
        out["roofline_tensor"] = troof
        out["batched_mixed_vs_plain"] = compare_batched(eod, 1, 1)
        out["paper_table_mat2_f64"] = paper_mat2(eod)
        out["robustness_matrices_f64"] = robustness_matrices(eod)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, sample, el = oracle_sample(A_np, w.tol * float(np.linalg.norm(A_np)), 15.0)
        out["cpu_baseline"] = {"value": v, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample,
                               "seconds": el}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def compare_forms(eod, steps, warmup, flush):
    """Mixed (BF16 split on tcgen05) against the plain FP64 path on the same
    inputs: the image-like 2048^2 matrix, the 8192^2 harmonic matrix and the
    262144 x 224 hyperspectral matrix.  Returns a list of result dicts and
    the tensor-core kernel's roofline over the mixed runs."""
    import numpy as np
    import torch
    import workloads as W

    bf16_peak, _, src = _measured_peaks()
    out, tc_fl, tc_ms, tc_n = [], 0.0, 0.0, 0
    cases = [("image-like 2048x2048 tol 1e-3 rel", lambda: W.image_like(), 64),
             ("harmonic 8192x8192 rank-400 1/i + noise 1e-6, tol 0.0128 rel", lambda: W.harmonic(), 64),
             ("hyperspectral 262144x224, 12 endmembers, 30 dB, tol 0.047 rel", lambda: W.hyperspectral(), 16)]
    for name, make, k in cases:
        w = make()
        A64 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float64))).cuda()
        A32 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float32))).cuda()
        del w.A
        m, n = A64.shape
        res = {}
        for form, A, prec in (("plain_f64", A64, "plain"), ("plain_f32", A32, "plain"), ("mixed_bf16", A32, "mixed"),
                              ("mixed_tf32", A32, "mixed_tf32")):
            for _ in range(warmup):
                f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
                f.close()
            torch.cuda.synchronize()
            if prec == "mixed":
                eod.eod_abe_debug_profile(1)
            tot = 0.0
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec)
                e1.record()
                e1.synchronize()
                tot += e0.elapsed_time(e1)
                r, rel = f.rank, f.rel_err
                f.close()
            if prec == "mixed":
                pr = eod.profile_read(eod.PROF_TC_GEMM)
                eod.eod_abe_debug_profile(0)
                tc_fl += pr["flops"]
                tc_ms += pr["ms"]
                tc_n += pr["launches"]
            ms = tot / steps
            res[form] = {"gflops": eod.model_flops(m, n, r, k, True) / (ms / 1e3) / 1e9, "ms": ms, "rank": r,
                         "rel_err": rel}
        base = res["plain_f64"]
        for form, v in res.items():
            v["rank_equal_f64"] = v["rank"] == base["rank"]
            v["d_rel_err_vs_f64"] = abs(v["rel_err"] - base["rel_err"])
        out.append({"workload": name, "m": m, "n": n, "k": k, "forms": res,
                    "mixed_speedup_vs_f64": base["ms"] / res["mixed_bf16"]["ms"],
                    "mixed_tf32_speedup_vs_f64": base["ms"] / res["mixed_tf32"]["ms"]})
        del A64, A32
        torch.cuda.empty_cache()
    ach = tc_fl / (tc_ms / 1e3) / 1e9 if tc_ms > 0 else None
    roof = {"bound": "tensor", "kernel": "tc_gemm (tcgen05 kind::f16, BF16 split pairs)", "achieved": ach,
            "peak": bf16_peak, "unit": "GFLOP/s", "frac": (ach / bf16_peak) if ach else None,
            "peak_source": f"{src} bf16 burst (MEASURED_PEAKS.json)", "launches": tc_n,
            "flops_per_launch": tc_fl / tc_n if tc_n else None, "traffic": None}
    return out, roof


# Alg. 2 on the paper's strictly rank-deficient test matrix (Sec. 4, Eq.
# (mat2)): A = U diag(sigma) V^T with Haar U, V (n x r blocks) and sigma the
# sorted uniform(0, 1) draws, r = 0.4 n; the paper's own times in seconds
# (MATLAB, its hardware) for tau = 0, 1, 2.
PAPER_MAT2_SECONDS = {4000: (1.5, 2.3, 3.3), 8000: (10.6, 18.0, 25.6), 12000: (29.3, 52.5, 75.5)}


def paper_mat2(eod, sizes=(4000, 8000, 12000)):
    """One timed factorisation (after one warm-up) per size and tau, plain
    FP64, k = 64, eps = 1e-8 absolute (between sigma_r ~ 1e-4 and the
    rounding floor ~ 1e-12).  The matrices are drawn on the GPU with torch's
    generator (seeded): at these sizes the host would take minutes."""
    import torch

    out = []
    for n in sizes:
        r = int(0.4 * n)
        g = torch.Generator(device="cuda").manual_seed(1000 + n)
        U, _ = torch.linalg.qr(torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64))
        V, _ = torch.linalg.qr(torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64))
        sig = torch.sort(torch.rand(r, generator=g, device="cuda", dtype=torch.float64), descending=True).values
        A = ((U * sig) @ V.t()).t().contiguous().t()
        del U, V
        torch.cuda.synchronize()
        for tau in (0, 1, 2):
            f = eod.factor(A, 1e-8, 7, block_k=64, tol_mode="abs", power_iters=tau)
            f.close()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = eod.factor(A, 1e-8, 7, block_k=64, tol_mode="abs", power_iters=tau)
            e1.record()
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            out.append({"n": n, "r_true": r, "tau": tau, "rank": f.rank, "rel_err": f.rel_err, "seconds": sec,
                        "paper_seconds": PAPER_MAT2_SECONDS[n][tau],
                        "paper_over_ours": PAPER_MAT2_SECONDS[n][tau] / sec})
            f.close()
        del A
        torch.cuda.empty_cache()
    return out


def robustness_matrices(eod):
    """The four matrix classes of Sec. 4.3 at n = 1000, plain FP64, k = 32,
    tau = 0 and 2: one timed factorisation after one warm-up each, with the
    rank, RelErr and the largest deviation of the R-values (|diag D-hat|) from
    the singular values, max |log10(|D(i,i)| / sigma_i)| over i <= rank."""
    import numpy as np
    import torch
    import workloads as W

    cases = [("I (low rank + noise, alpha 0.005)", lambda: W.low_rank_plus_noise(alpha=0.005), 1e-12, "abs"),
             ("I (low rank + noise, alpha 0.02)", lambda: W.low_rank_plus_noise(alpha=0.02), 1e-12, "abs"),
             ("II (devil's stairs)", lambda: W.devils_stairs(1000), 1e-5, "rel"),
             ("III (fast decay)", W.fast_decay, 1e-8, "rel"),
             ("IV (slow decay)", W.slow_decay, 1e-3, "rel")]
    out = []
    for name, make, tol, mode in cases:
        A_np = make()
        s = np.linalg.svd(A_np, compute_uv=False)
        A = torch.from_numpy(np.asfortranarray(A_np)).cuda()
        for tau in (0, 2):
            f = eod.factor(A, tol, 5, block_k=32, tol_mode=mode, power_iters=tau)
            f.close()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = eod.factor(A, tol, 5, block_k=32, tol_mode=mode, power_iters=tau)
            e1.record()
            e1.synchronize()
            r = f.rank
            d = np.abs(np.diag(f.D.cpu().numpy()))
            dev = float(np.abs(np.log10(d[:r] / s[:r])).max()) if r > 0 else None
            out.append({"matrix": name, "n": 1000, "tol": tol, "tol_mode": mode, "tau": tau, "rank": r,
                        "rel_err": f.rel_err, "ms": e0.elapsed_time(e1), "max_log10_rvalue_over_sigma": dev})
            f.close()
        del A
    return out


def compare_batched(eod, steps, warmup):
    """Factorisations per second of the 256-matrix pixel batch, mixed against
    plain FP64, as stated (clipped to [0, 255], tol 1e-3 relative) and
    unclipped (same tolerance)."""
    import numpy as np
    import torch
    import workloads as W

    out = []
    for name, clip, tol in (("pixel batch 256 (m,n~U[256,2048], r~U[8,128]), clipped [0,255], tol 1e-3 rel", True, 1e-3),
                            ("pixel batch 256, unclipped (no noise tail from clipping), tol 1e-3 rel", False, 1e-3)):
        w = W.pixel_batch(clip=clip, tol=tol)
        sets = {"plain_f64": ([torch.from_numpy(np.asfortranarray(a.astype(np.float64))).cuda() for a in w.A], "plain"),
                "mixed_bf16": ([torch.from_numpy(a).cuda() for a in w.A], "mixed")}
        res = {}
        ranks = {}
        rels = {}
        for form, (mats, prec) in sets.items():
            for _ in range(warmup):
                r, st = eod.factor_batched(mats, tol, w.seed, block_k=32, tol_mode="rel", precision=prec)
                del r
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                r, st = eod.factor_batched(mats, tol, w.seed, block_k=32, tol_mode="rel", precision=prec)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / steps
            ranks[form] = [x.rank for x in r]
            rels[form] = [x.rel_err for x in r]
            flops = sum(eod.model_flops(a.shape[0], a.shape[1], x.rank, 32, True) for a, x in zip(w.A, r))
            res[form] = {"fact_per_s": len(mats) / dt, "ms_per_batch": dt * 1e3, "gflops": flops / dt / 1e9,
                         "statuses_ok": all(x == 0 for x in st),
                         "rank_mean": float(np.mean(ranks[form])), "rank_max": int(np.max(ranks[form]))}
            del r
        eq = sum(a == b for a, b in zip(ranks["mixed_bf16"], ranks["plain_f64"]))
        drel = max(abs(a - b) for a, b in zip(rels["mixed_bf16"], rels["plain_f64"]))
        out.append({"workload": name, "forms": res, "mixed_rank_equal_f64": f"{eq}/{len(ranks['plain_f64'])}",
                    "mixed_max_d_rel_err_vs_f64": drel,
                    "mixed_speedup_vs_f64": res["mixed_bf16"]["fact_per_s"] / res["plain_f64"]["fact_per_s"]})
        del sets
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------- reference arm --
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import workloads as W
    w = W.image_like()
    A_np = w.A
    eps = w.tol * float(np.linalg.norm(A_np))
    for _ in range(args.warmup):
        oracle_sample(A_np, eps, 4.0)
    vals, secs, sample = [], 0.0, ""
    for _ in range(args.steps):
        v, sample, el = oracle_sample(A_np, eps, 6.0)
        vals.append(v)
        secs += el
    value = statistics.mean(vals)
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "GFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded image-like low-rank + noise; no dataset)",
        "config": {"workload": WORKLOAD + ", FP64 plain, k=64", "m": M, "n": N, "parallelism": "host, 1 thread"},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = _args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark of power-free EOD-ABE on one GB300 (or N replicas).

Headline workload: the harmonic 8192 x 8192 FP32 matrix (rank-400
U diag(1/i) V^T with Haar U, V plus Gaussian noise of std 1e-6; relative
tolerance 0.0128, twice the noise floor; the method reveals rank 455), k = 64.
One step = one complete factorisation through the C ABI (Alg. 1 + Alg. 2
steps 8-11 + the reconstruction error), inputs resident in HBM, L2 flushed
between steps.  The metric is GFLOP/s of the paper's cost model (Sec. 3.4,
tau = 0, plus the 2mnr of the reconstruction) for the mixed BF16 form, with
the plain FP64 form timed on the same matrix (widened to FP64) beside it and
their ratio at equal rank and |dRelErr| <= 1e-4.  The headline steps run
with the library's instrumentation off; the roofline of the dominant kernel
comes from a separate profiled pass.  The same line reports the host-buffer
end-to-end rate, the other precision forms, the other workloads (image-like
2048^2, hyperspectral 262144 x 224, the 256-matrix pixel batch), and the FP64
oracle timed on the host cores.

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
WORKLOAD = ("harmonic 8192x8192 FP32: rank-400 s_i=1/i (Haar U, V) + Gaussian noise 1e-6, tol 0.0128 relative, "
            "tuned k; mixed BF16 form (plain FP64 form on the same matrix beside it)")
HEAD_K = 64          # the fixed k reported beside the tuned one


def tuned_k(form, m, n, default=32):
    """k the library takes for block_k = 0: the first "block_k" row of the
    autotuner's table (paper_2506_22713_gb300/tuning.txt) covering (form, m,
    n), read as text so that the reference arm needs no GPU library."""
    code = {"plain_f64": 0, "plain_f32": 1, "mixed": 2, "mixed_tf32": 3}[form]
    path = os.path.join(ROOT, "paper_2506_22713_gb300", "tuning.txt")
    try:
        for line in open(path):
            f = line.split("#")[0].split()
            if len(f) == 8 and f[0] == "block_k":
                v = [int(x) for x in f[1:]]
                if v[0] <= code <= v[1] and v[2] <= m <= v[3] and v[4] <= n <= v[5]:
                    return v[6]
    except OSError:
        pass
    return default


# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2070 MHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
FP64_SM_PEAK_GFLOPS = FP64_PEAK_GFLOPS / 152
# FP32 (FFMA) peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070
L2_BYTES = 129 * 1024 * 1024
# kernel kinds of the library's profile counters, in PROF_* order
KINDS = ["gemm_simt", "chol", "omega", "stream", "tc_gemm", "oz_gemm", "oz_slice", "gemm_simt_f32", "batch"]
# BF16 slice-pair products per emulated FP64 multiply-add (8 slices, s + t <= 7)
OZ_PAIRS = 36


def _measured_peaks():
    """(bf16 burst GFLOP/s, bf16 sustained GFLOP/s, HBM GB/s, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return (float(d["bf16_tflops"]) * 1e3, float(d.get("bf16_tflops_sustained", d["bf16_tflops"])) * 1e3,
                float(d["hbm_gbs"]), "measured")
    except Exception:
        return 1.9e6, 1.7e6, 6800.0, "fallback"


# named workloads for ncu (k = 0: the autotuner's k, as the bench runs them)
PROFILE_CASES = {
    "image2048_f64": ("image_like", {}, "f64", "plain", 0),
    "image2048_mixed": ("image_like", {}, "f32", "mixed", 0),
    "harmonic8192_mixed": ("harmonic", {}, "f32", "mixed", 0),
    "harmonic8192_f64": ("harmonic", {}, "f64", "plain", 0),
    "hyperspectral_mixed": ("hyperspectral", {}, "f32", "mixed", 0),
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
    p.add_argument("--cpu-one-core", action="store_true",
                   help="also time the whole oracle on one host core (minutes)")
    p.add_argument("--no-compare", action="store_true", help="skip the other workloads")
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
def oracle_whole(A64, tol, k, seed, threads):
    """The FP64 oracle's whole method (Alg. 1, Alg. 2 steps 8-11 and the
    explicit reconstruction error) on `threads` host threads (0 = all cores);
    returns (GFLOP/s of the cost model at the oracle's rank, seconds, rank,
    threads used)."""
    import oracle
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    ref = oracle.eod_abe(A64, tol, 1, k=k, seed=seed)
    el = time.perf_counter() - t0
    m, n = A64.shape
    r = ref["r"]
    flops = 2.0 * (2.0 * m * n * r + m * r * r + 2.0 * n * r * r + 2.0 * r ** 3 + 4.0 * m * r * k) + 2.0 * m * n * r
    return flops / el / 1e9, el, r, used


def _oracle_sample_text(cores, r, k):
    return (f"whole method (Alg. 1 + Alg. 2 steps 8-11 + explicit RelErr) of the FP64 oracle (plain C, naive "
            f"loops, OpenMP over output columns) on the same 8192x8192 harmonic matrix widened to FP64, "
            f"k={k} (the GPU headline's), one run on {cores} host thread(s); rank {r}; GFLOP/s of the same cost "
            f"model as value")


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
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            # the first sample comes a few hundred ms after the start: let it
            # begin before the (short) timed region
            time.sleep(0.5)
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


KIND_SOURCES = {
    "batch": ["paper_2506_22713_gb300/csrc/batch.cu", "paper_2506_22713_gb300/csrc/chol_leaf.cuh"],
    "oz_gemm": ["paper_2506_22713_gb300/csrc/oz_gemm.cu", "paper_2506_22713_gb300/csrc/tc_ptx.cuh"],
    "tc_gemm": ["paper_2506_22713_gb300/csrc/tc_gemm.cu", "paper_2506_22713_gb300/csrc/tc_ptx.cuh"],
    "chol": ["paper_2506_22713_gb300/csrc/chol.cu", "paper_2506_22713_gb300/csrc/chol_leaf.cuh"],
    "gemm_simt": ["paper_2506_22713_gb300/csrc/gemm_simt.cu"],
    "gemm_simt_f32": ["paper_2506_22713_gb300/csrc/gemm_simt.cu", "paper_2506_22713_gb300/csrc/gram.cu"],
    "stream": ["paper_2506_22713_gb300/csrc/stream_kernels.cu"],
}


def roofline_of(kind, rec, peaks):
    """Roofline entry of one kernel kind from its profiled launches: achieved
    = the launches' algorithmic flops (or bytes) / their summed device time."""
    bf16_burst, bf16_sus, hbm, src = peaks
    ms = rec["ms"]
    fl, by, n = rec["flops"], rec["bytes"], rec["launches"]
    out = {"kernel_kind": kind, "launches": n, "ms": ms}
    if kind == "tc_gemm":
        ach = fl / (ms / 1e3) / 1e9
        out.update(bound="tensor", achieved=ach, peak=bf16_sus, unit="GFLOP/s",
                   peak_source=f"{src} BF16 sustained (MEASURED_PEAKS.json)",
                   note="achieved counts one product per launch (the method's flops); the BF16 split executes "
                        "two or three")
    elif kind == "oz_gemm":
        ach = fl / (ms / 1e3) / 1e9
        out.update(bound="tensor", achieved=ach, peak=bf16_sus / OZ_PAIRS, unit="GFLOP/s",
                   peak_source=f"{src} BF16 sustained / {OZ_PAIRS} slice-pair products per FP64 multiply-add",
                   note="FP64 flops of the method (upper-only and triangular launches counted at their share)")
    elif kind == "chol":
        ach = fl / (ms / 1e3) / 1e9
        out.update(bound="alu", achieved=ach, peak=FP64_SM_PEAK_GFLOPS, unit="GFLOP/s",
                   peak_source="FP64 of one SM from unit counts: 2 DFMA/clk x 2 flop x 2070 MHz (the kernel is one "
                               "CTA)")
    elif kind == "gemm_simt":
        ach = fl / (ms / 1e3) / 1e9
        out.update(bound="alu", achieved=ach, peak=FP64_PEAK_GFLOPS, unit="GFLOP/s",
                   peak_source="FP64 from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz")
    elif kind == "gemm_simt_f32":
        ach = fl / (ms / 1e3) / 1e9
        out.update(bound="alu", achieved=ach, peak=FP32_PEAK_GFLOPS, unit="GFLOP/s",
                   peak_source="FP32 from unit counts: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz",
                   note="the FP32 Gram forms each product exactly and sums with TwoSum (~9 FP32 operations "
                        "per multiply-add); achieved counts 2 flops per multiply-add")
    else:
        ach = by / (ms / 1e3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s",
                   peak_source=f"{src} HBM copy bandwidth (MEASURED_PEAKS.json)")
    out["frac"] = out["achieved"] / out["peak"] if out["peak"] else None
    out["flops_per_launch"] = fl / n if n else None
    out["bytes_per_launch"] = by / n if n else None
    tr = _traffic_for(kind, KIND_SOURCES.get(kind, []))
    out["traffic"] = tr[0] if tr else None
    out["traffic_launch"] = tr[1] if tr else None
    return out


# ---------------------------------------------------------------- our arm --
class Stepper:
    """Times whole factorisations with CUDA events on the launching stream,
    L2 flushed (a 258 MB write) before every timed step."""

    def __init__(self, eod, torch, dist, flush):
        self.eod, self.torch, self.dist, self.flush = eod, torch, dist, flush
        self.stream = torch.cuda.current_stream()

    def run(self, fn, steps, warmup):
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        l0 = self.eod.eod_abe_debug_launch_count()
        total, info = 0.0, None
        for _ in range(steps):
            self.flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            info = fn()
            e1.record(self.stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        launches = self.eod.eod_abe_debug_launch_count() - l0
        total = _max_over_ranks(total, self.dist, "cuda")
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        return total, info, launches

    def profile(self, fn, steps):
        """Per-kind launches, device ms, flops and bytes over `steps` steps."""
        eod = self.eod
        fn()
        self.torch.cuda.synchronize()
        eod.eod_abe_debug_profile(1)
        for _ in range(steps):
            self.flush.zero_()
            fn()
        self.torch.cuda.synchronize()
        kinds = {k: eod.profile_read(i) for i, k in enumerate(KINDS)}
        eod.eod_abe_debug_profile(0)
        return kinds


def _factor_fn(eod, A, w, k, prec, **kw):
    """One factorisation; k = 0 takes the autotuner's k.  Returns (rank,
    RelErr, k used)."""
    def fn():
        f = eod.factor(A, w.tol, w.seed, block_k=k, tol_mode="rel", precision=prec, **kw)
        out = (f.rank, f.rel_err, f.block_k)
        f.close()
        return out
    return fn


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

    peaks = _measured_peaks()
    w = W.harmonic()                            # same seeded matrix on every replica
    A32_np = w.A
    m, n = A32_np.shape
    A32 = torch.from_numpy(A32_np).cuda()
    A64 = torch.from_numpy(np.asfortranarray(A32_np.astype(np.float64))).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    st = Stepper(eod, torch, dist, flush)

    # ---- headline: mixed BF16, instrumentation off ----
    clocks = ClockSampler(local)
    clocks.start()
    t_mx, (r_mx, rel_mx, k_mx), launches = st.run(_factor_fn(eod, A32, w, 0, "mixed"), args.steps, args.warmup)
    clk = clocks.stop()
    flops_mx = eod.model_flops(m, n, r_mx, k_mx, True)
    value = ws * args.steps * flops_mx / (t_mx / 1e3) / 1e9
    ms_step = t_mx / args.steps

    # ---- plain FP64 on the same matrix (widened), same steps ----
    t_64, (r_64, rel_64, k_64), _ = st.run(_factor_fn(eod, A64, w, 0, "plain"), args.steps, args.warmup)
    ms_64 = t_64 / args.steps
    gf_64 = ws * args.steps * eod.model_flops(m, n, r_64, k_64, True) / (t_64 / 1e3) / 1e9
    forms = {"mixed_bf16": {"gflops": value, "ms": ms_step, "rank": r_mx, "rel_err": rel_mx, "k": k_mx},
             "plain_f64": {"gflops": gf_64, "ms": ms_64, "rank": r_64, "rel_err": rel_64, "k": k_64}}
    ctx_steps = max(2, args.steps // 2)
    for name, A, prec, k in (("plain_f32", A32, "plain", 0), ("mixed_tf32", A32, "mixed_tf32", 0),
                             ("mixed_bf16_fixed_k64", A32, "mixed", HEAD_K), ("plain_f64_fixed_k64", A64, "plain", HEAD_K)):
        t, (r, rel, kk), _ = st.run(_factor_fn(eod, A, w, k, prec), ctx_steps, 1)
        forms[name] = {"gflops": ws * ctx_steps * eod.model_flops(m, n, r, kk, True) / (t / 1e3) / 1e9,
                       "ms": t / ctx_steps, "rank": r, "rel_err": rel, "k": kk}
    for v in forms.values():
        v["rank_equal_f64"] = v["rank"] == r_64
        v["d_rel_err_vs_f64"] = abs(v["rel_err"] - rel_64)
    mixed_vs_plain = {"speedup_mixed_bf16_over_plain_f64": ms_64 / ms_step,
                      "rank_equal": r_mx == r_64, "d_rel_err": abs(rel_mx - rel_64),
                      "parity_ok": (r_mx == r_64) and abs(rel_mx - rel_64) <= 1e-4}

    # ---- roofline: a separate profiled pass of the headline form ----
    kinds = st.profile(_factor_fn(eod, A32, w, 0, "mixed"), 2)
    prof_total = sum(v["ms"] for v in kinds.values())
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    roofline = roofline_of(dom, kinds[dom], peaks)
    roofline["share_of_kernel_time"] = kinds[dom]["ms"] / prof_total if prof_total else None
    kernel_share = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / 2,
                        "share": (v["ms"] / prof_total if prof_total else None)} for k, v in kinds.items()}
    roofline_tensor = roofline_of("tc_gemm", kinds["tc_gemm"], peaks) if kinds["tc_gemm"]["launches"] else None

    # ---- end to end through the host-buffer entry point (mixed) ----
    Ah = torch.from_numpy(A32_np).pin_memory()
    cap = min(m, n)
    Uh = torch.empty((cap, m), dtype=torch.float32).pin_memory().t()
    Dh = torch.empty((cap, cap), dtype=torch.float64).pin_memory().t()
    Vh = torch.empty((cap, n), dtype=torch.float32).pin_memory().t()

    def e2e_step():
        return eod.factor_host(Ah, w.tol, w.seed, block_k=0, tol_mode="rel", precision="mixed",
                               U_out=Uh, D_out=Dh, V_out=Vh)
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        re2e, _ = e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_val = ws * args.steps * eod.model_flops(m, n, re2e, k_mx, True) / e2e_s / 1e9

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
        "dtype": "bf16",
        "data": "synthetic (seeded harmonic low-rank + noise; no dataset)",
        "config": {"workload": WORKLOAD, "m": m, "n": n, "rank": r_mx, "rel_err": rel_mx, "block_k": k_mx,
                   "tuning": "k, FP32 tiles and batch workers from the autotuner's table "
                             "(paper_2506_22713_gb300/tuning.txt); forms *_fixed_k64 beside with k = 64",
                   "form": "mixed BF16: sketch/projection/error on tcgen05 (BF16 split, FP32 accumulation); "
                           "Gram/Cholesky/rank test/core in FP64",
                   "parallelism": f"replicas x{ws}", "l2": "flushed between timed steps (258 MB write)",
                   "instrumentation": "off in the timed steps; roofline from a separate profiled pass"},
        "mixed_vs_plain": mixed_vs_plain,
        "forms": forms,
        "roofline": roofline,
        "roofline_tensor": roofline_tensor,
        "kernel_share": kernel_share,
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": 4 * m * n,
                "d2h_bytes_per_step": 4 * (m * re2e + n * re2e) + 8 * re2e * re2e},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    del A64
    torch.cuda.empty_cache()
    if not args.no_compare:
        out["workloads"] = compare_workloads(eod, st, max(2, args.steps // 2), 1)
        out["batched_mixed_vs_plain"] = compare_batched(eod, 3, 1)
        out["subspace_iteration_f64"] = subspace_iterations(eod, st, max(2, args.steps // 2))
        out["paper_table_mat2_f64"] = paper_mat2(eod)
        out["robustness_matrices_f64"] = robustness_matrices(eod)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        A64_np = np.asfortranarray(A32_np.astype(np.float64))
        v, el, r_o, cores = oracle_whole(A64_np, w.tol, k_mx, w.seed, 0)
        out["cpu_baseline"] = {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                               "sample": _oracle_sample_text(cores, r_o, k_mx), "seconds": el,
                               "rank": r_o, "rank_equal_gpu": r_o == r_mx}
        if args.cpu_one_core:
            v1, el1, _, _ = oracle_whole(A64_np, w.tol, k_mx, w.seed, 1)
            out["cpu_baseline"]["one_core"] = {"value": v1, "seconds": el1, "cores": 1}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def compare_workloads(eod, st, steps, warmup):
    """The other single-matrix workloads in all four precision forms: the
    image-like 2048^2 matrix (FP64 storage; its FP32 rounding for the FP32
    forms) and the 262144 x 224 hyperspectral matrix."""
    import numpy as np
    import torch
    import workloads as W

    out = []
    cases = [("image-like 2048x2048 rank-150 s_i=255 i^-1.5 + noise 1e-4 s_1, tol 1e-3 rel", W.image_like, 64),
             ("hyperspectral 262144x224, 12 endmembers, 30 dB, tol 0.047 rel", W.hyperspectral, 16)]
    for name, make, k in cases:
        w = make()
        A64 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float64))).cuda()
        A32 = torch.from_numpy(np.asfortranarray(w.A.astype(np.float32))).cuda()
        m, n = A64.shape
        res = {}
        for form, A, prec, kk in (("plain_f64", A64, "plain", 0), ("plain_f32", A32, "plain", 0),
                                  ("mixed_bf16", A32, "mixed", 0), ("mixed_tf32", A32, "mixed_tf32", 0),
                                  ("plain_f64_fixed_k", A64, "plain", k), ("mixed_bf16_fixed_k", A32, "mixed", k)):
            t, (r, rel, ku), _ = st.run(_factor_fn(eod, A, w, kk, prec), steps, warmup)
            ms = t / steps
            res[form] = {"gflops": eod.model_flops(m, n, r, ku, True) / (ms / 1e3) / 1e9, "ms": ms, "rank": r,
                         "rel_err": rel, "k": ku}
        base = res["plain_f64"]
        for v in res.values():
            v["rank_equal_f64"] = v["rank"] == base["rank"]
            v["d_rel_err_vs_f64"] = abs(v["rel_err"] - base["rel_err"])
        out.append({"workload": name, "m": m, "n": n, "k": k, "forms": res,
                    "mixed_speedup_vs_f64": base["ms"] / res["mixed_bf16"]["ms"],
                    "mixed_tf32_speedup_vs_f64": base["ms"] / res["mixed_tf32"]["ms"]})
        del A64, A32
        torch.cuda.empty_cache()
    return out


def subspace_iterations(eod, st, steps):
    """Alg. 2 with tau = 1, 2 subspace iterations on the image-like 2048^2
    FP64 matrix (the cost model adds tau (2mnr + 2mr^2 + 2nr^2) multiply-adds,
    Sec. 3.4)."""
    import torch
    import workloads as W

    w = W.image_like()
    A = torch.from_numpy(w.A).cuda()
    m, n = w.A.shape
    out = {}
    for tau in (0, 1, 2):
        t, (r, rel, ku), _ = st.run(_factor_fn(eod, A, w, 0, "plain", power_iters=tau), steps, 2)
        ms = t / steps
        fl = eod.model_flops(m, n, r, ku, True) + 2.0 * tau * (2.0 * m * n * r + 2.0 * m * r * r + 2.0 * n * r * r)
        out[f"tau{tau}"] = {"ms_per_step": ms, "gflops": fl / (ms / 1e3) / 1e9, "rank": r, "rel_err": rel}
    return out


# Alg. 2 on the paper's strictly rank-deficient test matrix (Sec. 4, Eq.
# (mat2)): A = U diag(sigma) V^T with Haar U, V (n x r blocks) and sigma the
# sorted uniform(0, 1) draws, r = 0.4 n; the paper's own times in seconds
# (MATLAB, its hardware) for tau = 0, 1, 2.
PAPER_MAT2_SECONDS = {4000: (1.5, 2.3, 3.3), 8000: (10.6, 18.0, 25.6), 12000: (29.3, 52.5, 75.5)}


def paper_mat2(eod, sizes=(4000, 8000, 12000)):
    """One timed factorisation (after one warm-up) per size and tau, plain
    FP64, k = 64, eps = 1e-8 absolute (between sigma_r ~ 1e-4 and the
    rounding floor ~ 1e-12).  The matrices are drawn on the GPU with torch's
    generator (seeded) from the recipe of workloads.mat2: at these sizes the
    host would take minutes (the oracle-parity tests use the numpy generator
    at n = 1000 and 4000)."""
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
    """Factorisations per second of the 256-matrix pixel batch, as stated
    (clipped to [0, 255], tol 1e-3 relative) and unclipped (same tolerance),
    at block_k = 0 (the persistent launch's k = 32; the tuned batch k on the
    worker streams):
    plain FP64 (worker streams), the FP32 batch through the library's default
    route (the persistent launch, items above its rank capacity handed to the
    worker streams in the mixed BF16 form) and the same FP32 batch on the
    worker streams alone (EOD_BATCH_PERSISTENT=0)."""
    import numpy as np
    import torch
    import workloads as W

    def timed(mats, prec, tol, seed, env):
        saved = {k: os.environ.get(k) for k in env}
        os.environ.update(env)
        try:
            for _ in range(warmup):
                r, st = eod.factor_batched(mats, tol, seed, block_k=0, tol_mode="rel", precision=prec)
                del r
            torch.cuda.synchronize()
            keep = []   # factor sets are released after the clock stops (eod_abe_free synchronises)
            t0 = time.perf_counter()
            for _ in range(steps):
                r, st = eod.factor_batched(mats, tol, seed, block_k=0, tol_mode="rel", precision=prec)
                keep.append(r)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / steps
            del keep[:-1]
            return dt, r, st
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    out = []
    for name, clip, tol in (("pixel batch 256 (m,n~U[256,2048], r~U[8,128]), clipped [0,255], tol 1e-3 rel", True, 1e-3),
                            ("pixel batch 256, unclipped (no noise tail from clipping), tol 1e-3 rel", False, 1e-3)):
        w = W.pixel_batch(clip=clip, tol=tol)
        m32 = [torch.from_numpy(a).cuda() for a in w.A]
        m64 = [torch.from_numpy(np.asfortranarray(a.astype(np.float64))).cuda() for a in w.A]
        legs = {"plain_f64": (m64, "plain", {}),
                "mixed_bf16": (m32, "mixed", {}),
                "mixed_bf16_worker_streams": (m32, "mixed", {"EOD_BATCH_PERSISTENT": "0"})}
        res, ranks, rels = {}, {}, {}
        for form, (mats, prec, env) in legs.items():
            dt, r, st = timed(mats, prec, tol, w.seed, env)
            ranks[form] = [x.rank for x in r]
            rels[form] = [x.rel_err for x in r]
            flops = sum(eod.model_flops(a.shape[0], a.shape[1], x.rank, x.block_k, True) for a, x in zip(w.A, r))
            res[form] = {"fact_per_s": len(mats) / dt, "ms_per_batch": dt * 1e3, "gflops": flops / dt / 1e9,
                         "statuses_ok": all(x == 0 for x in st),
                         "block_k_used": sorted(set(int(x.block_k) for x in r)),
                         "rank_mean": float(np.mean(ranks[form])), "rank_max": int(np.max(ranks[form]))}
            if form == "mixed_bf16":
                # items the persistent launch finished (its factor sets say EOD_PLAIN)
                res[form]["items_in_persistent_launch"] = sum(1 for x in r if x.precision == 0)
            if form != "mixed_bf16":
                res[form]["worker_streams"] = eod.tuning_lookup(
                    "batch_workers", len(mats), int(np.mean([a.shape[0] for a in w.A])),
                    int(np.mean([a.shape[1] for a in w.A]))) or 8
            del r
        # the persistent kernel alone: its device time (CUDA events around
        # the graph launch) against the cost model's flops of the items it
        # finished, on the FP32 CUDA-core peak (its products are FP32 SIMT)
        eod.eod_abe_debug_profile(1)
        r, st = eod.factor_batched(m32, tol, w.seed, block_k=0, tol_mode="rel", precision="mixed")
        pk = eod.profile_read(eod.PROF_BATCH)
        eod.eod_abe_debug_profile(0)
        fl = sum(eod.model_flops(a.shape[0], a.shape[1], x.rank, x.block_k, True) for a, x in zip(w.A, r)
                 if x.precision == 0)
        if pk["launches"] and pk["ms"] > 0:
            ach = fl / (pk["ms"] / 1e3) / 1e9
            res["mixed_bf16"]["persistent_kernel"] = {
                "ms": pk["ms"], "model_gflop": fl / 1e9, "achieved_gflops": ach, "bound": "alu",
                "peak_gflops": FP32_PEAK_GFLOPS, "frac": ach / FP32_PEAK_GFLOPS,
                "peak_source": "FP32 from unit counts: 152 SMs x 128 FFMA/clk x 2 flop x 2070 MHz"}
            if not clip:
                tr = _traffic_for("batch", KIND_SOURCES["batch"])
                res["mixed_bf16"]["persistent_kernel"]["traffic"] = tr[0] if tr else None
                res["mixed_bf16"]["persistent_kernel"]["traffic_launch"] = tr[1] if tr else None
        del r
        eq = sum(a == b for a, b in zip(ranks["mixed_bf16"], ranks["plain_f64"]))
        drel = max(abs(a - b) for a, b in zip(rels["mixed_bf16"], rels["plain_f64"]))
        out.append({"workload": name, "forms": res, "mixed_rank_equal_f64": f"{eq}/{len(ranks['plain_f64'])}",
                    "mixed_max_d_rel_err_vs_f64": drel,
                    "mixed_speedup_vs_f64": res["mixed_bf16"]["fact_per_s"] / res["plain_f64"]["fact_per_s"],
                    "persistent_speedup_vs_worker_streams":
                        res["mixed_bf16"]["fact_per_s"] / res["mixed_bf16_worker_streams"]["fact_per_s"]})
        del m32, m64
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------- reference arm --
def run_reference(args):
    """The FP64 oracle as the reference arm: each step is its whole method on
    the headline matrix, on every host core; GFLOP/s of the same cost model."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import workloads as W
    w = W.harmonic()
    A64 = np.asfortranarray(w.A.astype(np.float64))
    m, n = A64.shape
    k = tuned_k("mixed", m, n)
    for _ in range(args.warmup):
        oracle_whole(A64, w.tol, k, w.seed, 0)
    secs, flops, r, cores = 0.0, 0.0, 0, 1
    for _ in range(args.steps):
        v, el, r, cores = oracle_whole(A64, w.tol, k, w.seed, 0)
        secs += el
        flops += v * el * 1e9
    value = flops / secs / 1e9
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
        "data": "synthetic (seeded harmonic low-rank + noise; no dataset)",
        "config": {"workload": WORKLOAD, "m": m, "n": n, "rank": r, "block_k": k,
                   "parallelism": f"host, {cores} threads"},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": _oracle_sample_text(cores, r, k)},
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

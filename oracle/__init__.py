"""FP64 CPU oracle for power-free EOD-ABE (arXiv 2506.22713, Alg. 1 and Alg. 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark import this package.  The CUDA library never
loads it, and this package never loads the CUDA library.

The arithmetic lives in ``eod_oracle.c`` (plain C, naive loops, IEEE double);
this module compiles it with gcc (``build()``) and marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eod_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)


_CFLAGS = ["-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _compile(src: str, out: str) -> None:
    """gcc with OpenMP (the column loops shared among threads, bit-identical
    to one thread); without OpenMP if this compiler lacks it."""
    base = ["gcc", *_CFLAGS]
    res = subprocess.run(base + ["-fopenmp", "-o", out, src, "-lm"], capture_output=True, text=True)
    if res.returncode != 0:
        subprocess.run(base + ["-o", out, src, "-lm"], check=True)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (no fast-math, no FMA
    contraction, so x86 and Arm hosts give the same bits)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB + ".tmp")
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def configure(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    lib.orc_philox4x32_10.restype = None
    lib.orc_omega_entry.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    lib.orc_omega_entry.restype = ctypes.c_double
    lib.orc_round_to_bf16.argtypes = [ctypes.c_double]
    lib.orc_round_to_bf16.restype = ctypes.c_double
    lib.orc_omega.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_uint64, _f64p]
    lib.orc_omega.restype = None
    lib.orc_householder_qr.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64,
                                       _f64p, ctypes.c_int64, _f64p, ctypes.c_int64]
    lib.orc_householder_qr.restype = ctypes.c_int
    lib.orc_fro_norm.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, ctypes.c_int64]
    lib.orc_fro_norm.restype = ctypes.c_double
    lib.orc_basis_ext.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                  _f64p, _i64p, _f64p, _i64p, ctypes.c_int64]
    lib.orc_basis_ext.restype = ctypes.c_int
    lib.orc_eod_abe.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p, _i64p,
                                _f64p, _f64p, _i64p]
    lib.orc_eod_abe.restype = ctypes.c_int
    lib.orc_storage_entries.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    lib.orc_storage_entries.restype = ctypes.c_int64
    lib.orc_storage_rank_bound.argtypes = [ctypes.c_int64, ctypes.c_int64]
    lib.orc_storage_rank_bound.restype = ctypes.c_double
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_set_threads.restype = ctypes.c_int
    lib.orc_get_threads.argtypes = []
    lib.orc_get_threads.restype = ctypes.c_int
    return lib


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (possibly edited) copy of the oracle source to out_path with
    the same flags as build(); used by the tests that plant mistakes."""
    src = out_path + ".c"
    with open(src, "w") as fh:
        fh.write(src_text)
    _compile(src, out_path)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = configure(ctypes.CDLL(_LIB))
    return _lib


def set_threads(n: int) -> int:
    """Threads for the oracle's column loops (n <= 0: the OpenMP default,
    OMP_NUM_THREADS or every core); returns the count in effect (1 when built
    without OpenMP).  Results do not depend on it."""
    return int(_load().orc_set_threads(int(n)))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _ptr(a: np.ndarray, t=_f64p):
    return a.ctypes.data_as(t)


def _colmajor(A) -> np.ndarray:
    return np.asfortranarray(np.asarray(A, dtype=np.float64))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of a 4-word counter under a 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def round_to_bf16(x) -> np.ndarray:
    """Round each double to the nearest BF16 value, ties to even."""
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    return np.array([lib.orc_round_to_bf16(float(v)) for v in x.ravel()]).reshape(x.shape)


def omega(n: int, col0: int, ncols: int, seed: int, batch: int = 0) -> np.ndarray:
    """Columns col0 .. col0+ncols-1 of the Gaussian test matrix (n rows)."""
    lib = _load()
    out = np.zeros((n, ncols), dtype=np.float64, order="F")
    lib.orc_omega(n, col0, ncols, seed, batch, _ptr(out))
    return out


def householder_qr(W):
    """Thin Householder QR with a non-negative diagonal: W = Q R."""
    lib = _load()
    W = _colmajor(W).copy(order="F")
    m, p = W.shape
    Q = np.zeros((m, p), order="F")
    R = np.zeros((p, p), order="F")
    st = lib.orc_householder_qr(m, p, _ptr(W), m, _ptr(Q), m, _ptr(R), p)
    if st:
        raise ValueError(f"householder_qr status {st}")
    return Q, R


def fro_norm(A) -> float:
    lib = _load()
    A = _colmajor(A)
    return lib.orc_fro_norm(A.shape[0], A.shape[1], _ptr(A), A.shape[0])


def basis_ext(A, eps: float, k: int = 32, seed: int = 0, batch: int = 0, max_blocks: int = 0):
    """Alg. 1: returns (Q (m x r), tdiag) for the absolute threshold eps.
    max_blocks > 0 stops after that many blocks (a bounded timing sample)."""
    lib = _load()
    A = _colmajor(A)
    m, n = A.shape
    cap = min(m, n)
    Q = np.zeros((m, max(cap, 1)), order="F")
    td = np.zeros(max(cap, 1))
    r = ctypes.c_int64(0)
    nt = ctypes.c_int64(0)
    st = lib.orc_basis_ext(_ptr(A), m, n, m, eps, k, seed, batch, _ptr(Q), ctypes.byref(r),
                           _ptr(td), ctypes.byref(nt), int(max_blocks))
    if st:
        raise MemoryError("oracle allocation failed")
    return Q[:, : r.value].copy(order="F"), td[: nt.value].copy()


def eod_abe(A, tol: float, tol_mode: int = 0, k: int = 32, seed: int = 0, batch: int = 0, tau: int = 0) -> dict:
    """Alg. 2 (tau subspace iterations, 0 = power-free) plus the
    reconstruction error.

    tol_mode 0 uses eps = tol; tol_mode 1 uses eps = tol * ||A||_F.
    Returns a dict with r, U, D, V, Q, C, rel_err, norm_a, eps, tdiag.
    """
    lib = _load()
    A = _colmajor(A)
    m, n = A.shape
    cap = max(min(m, n), 1)
    U = np.zeros((m, cap), order="F")
    D = np.zeros((cap, cap), order="F")
    V = np.zeros((n, cap), order="F")
    Q = np.zeros((m, cap), order="F")
    C = np.zeros((cap, n), order="F")
    td = np.zeros(cap)
    res = np.zeros(3)
    r = ctypes.c_int64(0)
    nt = ctypes.c_int64(0)
    st = lib.orc_eod_abe(_ptr(A), m, n, m, tol, tol_mode, k, seed, batch, int(tau), _ptr(U), _ptr(D), _ptr(V),
                         _ptr(Q), _ptr(C), ctypes.byref(r), _ptr(res), _ptr(td), ctypes.byref(nt))
    if st:
        raise MemoryError("oracle allocation failed")
    rr = r.value
    return {
        "r": rr,
        "U": U[:, :rr].copy(order="F"),
        "D": D[:rr, :rr].copy(order="F"),
        "V": V[:, :rr].copy(order="F"),
        "Q": Q[:, :rr].copy(order="F"),
        "C": C[:rr, :].copy(order="F"),
        "rel_err": float(res[0]),
        "norm_a": float(res[1]),
        "eps": float(res[2]),
        "tdiag": td[: nt.value].copy(),
    }


def storage_entries(m: int, n: int, r: int) -> int:
    return int(_load().orc_storage_entries(m, n, r))


def storage_rank_bound(m: int, n: int) -> float:
    return float(_load().orc_storage_rank_bound(m, n))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))

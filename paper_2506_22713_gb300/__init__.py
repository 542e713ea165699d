"""Python binding of libeodabe.so, the GB300 (sm_103a) implementation of
EOD-ABE (arXiv 2506.22713, Alg. 1 and Alg. 2; power-free or with tau
subspace iterations).

This module only marshals arguments: every step of the factorisation runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.
Importing the module loads the library and fails loudly when it is missing
(run ``__graft_entry__.build()`` or ``python -m paper_2506_22713_gb300._build``).

The low-level functions carry the C names (``eod_abe_factor`` ...) and take
raw pointers; ``factor``, ``reconstruct``, ``omega``, ``factor_host`` and
``factor_batched`` wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libeodabe.so")

EOD_OK, EOD_EINVAL, EOD_ENOMEM, EOD_ECUDA, EOD_ENONFINITE, EOD_ETIMEOUT, EOD_EPRECISION, EOD_EUNSUPPORTED = range(8)
EOD_F64, EOD_F32 = 0, 1
EOD_PLAIN, EOD_MIXED_BF16, EOD_MIXED_TF32 = 0, 1, 2
EOD_TOL_ABS, EOD_TOL_REL_FRO = 0, 1

EXPORTED = [
    "eod_opts_default", "eod_abe_factor", "eod_abe_factor_ex", "eod_abe_factor_host",
    "eod_abe_reconstruct", "eod_abe_factor_batched", "eod_abe_omega", "eod_abe_free",
    "eod_status_string", "eod_abe_storage_entries", "eod_abe_model_flops",
    "eod_abe_debug_fail_alloc_after", "eod_abe_version", "eod_abe_debug_profile",
    "eod_abe_debug_profile_read", "eod_abe_debug_launch_count", "eod_abe_fro_norm_noalloc",
    "eod_abe_debug_tc_gemm", "eod_abe_debug_f64_gemm", "eod_abe_debug_chol", "eod_abe_debug_bounded_wait",
    "eod_abe_debug_recip", "eod_abe_tuning_load", "eod_abe_tuning_lookup", "eod_abe_debug_f32_gemm",
    "eod_abe_debug_batch_phases",
]


class EodOpts(ctypes.Structure):
    _fields_ = [
        ("a_dtype", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("tol_mode", ctypes.c_int32),
        ("block_k", ctypes.c_int32),
        ("power_iters", ctypes.c_int32),
        ("compute_err", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("batch_index", ctypes.c_uint64),
    ]


class EodFactors(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("rank", ctypes.c_int64),
        ("f_dtype", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("U", ctypes.c_void_p), ("D", ctypes.c_void_p), ("V", ctypes.c_void_p),
        ("Q", ctypes.c_void_p), ("C", ctypes.c_void_p),
        ("tdiag", ctypes.POINTER(ctypes.c_double)), ("ntdiag", ctypes.c_int64),
        ("rel_err", ctypes.c_double), ("norm_a", ctypes.c_double), ("eps", ctypes.c_double),
        ("t_margin", ctypes.c_double),
        ("blocks", ctypes.c_int64), ("restarts", ctypes.c_int64), ("block_k", ctypes.c_int64),
    ]


class EodError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, F64, I32, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64
    FP = ctypes.POINTER(ctypes.POINTER(EodFactors))
    OP = ctypes.POINTER(EodOpts)
    lib.eod_opts_default.argtypes = [OP]
    lib.eod_opts_default.restype = None
    lib.eod_abe_factor.argtypes = [P, I64, I64, I64, F64, U64, FP]
    lib.eod_abe_factor.restype = I32
    lib.eod_abe_factor_ex.argtypes = [P, I64, I64, I64, F64, U64, OP, FP]
    lib.eod_abe_factor_ex.restype = I32
    lib.eod_abe_factor_host.argtypes = [P, I64, I64, I64, F64, U64, OP, P, P, P, I64,
                                        ctypes.POINTER(I64), ctypes.POINTER(F64)]
    lib.eod_abe_factor_host.restype = I32
    lib.eod_abe_reconstruct.argtypes = [ctypes.POINTER(EodFactors), P, I64, OP]
    lib.eod_abe_reconstruct.restype = I32
    lib.eod_abe_factor_batched.argtypes = [ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                           ctypes.POINTER(I64), I64, F64, U64, OP,
                                           ctypes.POINTER(ctypes.POINTER(EodFactors)), ctypes.POINTER(I32)]
    lib.eod_abe_factor_batched.restype = I32
    lib.eod_abe_omega.argtypes = [I64, I64, I64, U64, U64, P, P]
    lib.eod_abe_omega.restype = I32
    lib.eod_abe_free.argtypes = [ctypes.POINTER(EodFactors)]
    lib.eod_abe_free.restype = None
    lib.eod_status_string.argtypes = [I32]
    lib.eod_status_string.restype = ctypes.c_char_p
    lib.eod_abe_storage_entries.argtypes = [I64, I64, I64]
    lib.eod_abe_storage_entries.restype = I64
    lib.eod_abe_model_flops.argtypes = [I64, I64, I64, I64, I32]
    lib.eod_abe_model_flops.restype = F64
    lib.eod_abe_debug_fail_alloc_after.argtypes = [I32]
    lib.eod_abe_debug_fail_alloc_after.restype = None
    lib.eod_abe_debug_profile.argtypes = [I32]
    lib.eod_abe_debug_profile.restype = None
    lib.eod_abe_debug_profile_read.argtypes = [I32, ctypes.POINTER(I64), ctypes.POINTER(F64), ctypes.POINTER(F64),
                                               ctypes.POINTER(F64)]
    lib.eod_abe_debug_profile_read.restype = I32
    lib.eod_abe_debug_launch_count.argtypes = []
    lib.eod_abe_debug_launch_count.restype = I64
    lib.eod_abe_fro_norm_noalloc.argtypes = [P, I64, I64, I64, I32, P, P, P]
    lib.eod_abe_fro_norm_noalloc.restype = I32
    lib.eod_abe_debug_tc_gemm.argtypes = [I32, I64, I64, I64, P, I64, P, I64, P, I64, P, P]
    lib.eod_abe_debug_tc_gemm.restype = I32
    lib.eod_abe_debug_bounded_wait.argtypes = [I64, I32, P]
    lib.eod_abe_debug_bounded_wait.restype = I32
    lib.eod_abe_debug_recip.argtypes = [P, P, I64, P]
    lib.eod_abe_debug_recip.restype = I32
    lib.eod_abe_tuning_load.argtypes = [ctypes.c_char_p]
    lib.eod_abe_tuning_load.restype = I32
    lib.eod_abe_tuning_lookup.argtypes = [ctypes.c_char_p, I64, I64, I64, ctypes.POINTER(I64)]
    lib.eod_abe_tuning_lookup.restype = I32
    lib.eod_abe_debug_f32_gemm.argtypes = [I32, I32, I32, I64, I64, I64, F64, P, I64, P, I64, F64, P, I64, P]
    lib.eod_abe_debug_f32_gemm.restype = I32
    lib.eod_abe_debug_batch_phases.argtypes = [I32, P, I64]
    lib.eod_abe_debug_batch_phases.restype = I32
    lib.eod_abe_debug_f64_gemm.argtypes = [I32, I32, I32, I64, I64, I64, F64, P, I64, P, I64, F64, P, I64, P]
    lib.eod_abe_debug_f64_gemm.restype = I32
    lib.eod_abe_debug_chol.argtypes = [P, I64, I32, I32, F64, F64, F64, F64, P, P, I64, P, P]
    lib.eod_abe_debug_chol.restype = I32
    lib.eod_abe_version.argtypes = []
    lib.eod_abe_version.restype = ctypes.c_char_p
    return lib


_lib = _load()

# ---------------------------------------------------------------- C names --
eod_opts_default = _lib.eod_opts_default
eod_abe_factor = _lib.eod_abe_factor
eod_abe_factor_ex = _lib.eod_abe_factor_ex
eod_abe_factor_host = _lib.eod_abe_factor_host
eod_abe_reconstruct = _lib.eod_abe_reconstruct
eod_abe_factor_batched = _lib.eod_abe_factor_batched
eod_abe_omega = _lib.eod_abe_omega
eod_abe_free = _lib.eod_abe_free
eod_status_string = _lib.eod_status_string
eod_abe_storage_entries = _lib.eod_abe_storage_entries
eod_abe_model_flops = _lib.eod_abe_model_flops
eod_abe_debug_fail_alloc_after = _lib.eod_abe_debug_fail_alloc_after
eod_abe_version = _lib.eod_abe_version
eod_abe_debug_profile = _lib.eod_abe_debug_profile
eod_abe_debug_profile_read = _lib.eod_abe_debug_profile_read
eod_abe_debug_launch_count = _lib.eod_abe_debug_launch_count
eod_abe_fro_norm_noalloc = _lib.eod_abe_fro_norm_noalloc
eod_abe_debug_tc_gemm = _lib.eod_abe_debug_tc_gemm
eod_abe_debug_bounded_wait = _lib.eod_abe_debug_bounded_wait
eod_abe_debug_recip = _lib.eod_abe_debug_recip
eod_abe_tuning_load = _lib.eod_abe_tuning_load
eod_abe_tuning_lookup = _lib.eod_abe_tuning_lookup
eod_abe_debug_f32_gemm = _lib.eod_abe_debug_f32_gemm
eod_abe_debug_batch_phases = _lib.eod_abe_debug_batch_phases

BATCH_PHASES = ("norm", "omega", "sketch", "deflate", "gram_leaf", "panel", "residual", "project", "err", "core",
                "u")


def batch_phases(enable: bool = True) -> dict:
    """Turns the persistent launch's per-phase clock accounting on or off and
    returns the last launch's counters (SM clock ticks summed over items)."""
    out = (ctypes.c_double * len(BATCH_PHASES))()
    st = _lib.eod_abe_debug_batch_phases(1 if enable else 0, out, len(BATCH_PHASES))
    if st != EOD_OK:
        raise EodError(st, "eod_abe_debug_batch_phases")
    return dict(zip(BATCH_PHASES, list(out)))


def tuning_lookup(key: str, a: int, b: int = 0, c: int = 0):
    """The autotuner's value for key at (a, b, c), or None."""
    v = ctypes.c_int64(0)
    return v.value if _lib.eod_abe_tuning_lookup(key.encode(), int(a), int(b), int(c), ctypes.byref(v)) else None
eod_abe_debug_f64_gemm = _lib.eod_abe_debug_f64_gemm
eod_abe_debug_chol = _lib.eod_abe_debug_chol

(PROF_GEMM_SIMT, PROF_CHOL, PROF_OMEGA, PROF_STREAM, PROF_TC_GEMM, PROF_OZ_GEMM, PROF_OZ_SLICE,
 PROF_GEMM_SIMT32, PROF_BATCH) = range(9)


def profile_read(kind: int) -> dict:
    """Launch count, device ms, algorithmic flops and bytes of one kernel kind
    since eod_abe_debug_profile(1)."""
    n = ctypes.c_int64(0)
    ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    st = _lib.eod_abe_debug_profile_read(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by))
    if st != EOD_OK:
        raise EodError(st, "eod_abe_debug_profile_read")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def status_string(status: int) -> str:
    return _lib.eod_status_string(status).decode()


def library() -> ctypes.CDLL:
    return _lib


# ------------------------------------------------------------ conveniences --
_DT = {torch.float64: EOD_F64, torch.float32: EOD_F32}
_TORCH = {EOD_F64: torch.float64, EOD_F32: torch.float32}
_PREC = {"plain": EOD_PLAIN, "mixed": EOD_MIXED_BF16, "mixed_bf16": EOD_MIXED_BF16, "mixed_tf32": EOD_MIXED_TF32}
_TOLM = {"abs": EOD_TOL_ABS, "rel": EOD_TOL_REL_FRO}


def make_opts(dtype=EOD_F64, precision="plain", tol_mode="abs", block_k=0, compute_err=True,
              stream=None, batch_index=0, power_iters=0) -> EodOpts:
    o = EodOpts()
    _lib.eod_opts_default(ctypes.byref(o))
    o.a_dtype = dtype
    o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    o.tol_mode = _TOLM[tol_mode] if isinstance(tol_mode, str) else int(tol_mode)
    o.block_k = int(block_k)
    o.compute_err = 1 if compute_err else 0
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    o.batch_index = int(batch_index)
    o.power_iters = int(power_iters)
    return o


def _colmajor_ld(A: torch.Tensor) -> int:
    if A.dim() != 2:
        raise ValueError("A must be a matrix")
    if A.stride(0) != 1 and A.shape[0] > 1:
        raise ValueError("A must be column-major (stride(0) == 1); use A.t().contiguous().t()")
    return max(A.stride(1), A.shape[0]) if A.shape[1] > 1 else A.shape[0]


class _DevArray:
    """A device buffer owned by an eod_factors struct, exposed to torch."""

    def __init__(self, ptr, rows, cols, ld, dtype, owner):
        es = torch.empty((), dtype=dtype).element_size()
        self._owner = owner
        self.__cuda_array_interface__ = {
            "shape": (rows, cols),
            "typestr": "<f8" if dtype == torch.float64 else "<f4",
            "data": (ptr, False),
            "version": 3,
            "strides": (es, es * ld),
            "stream": None,
        }


class Factors:
    """Owns one eod_factors*; matrix properties are torch views of the
    library's device buffers (valid while this object lives)."""

    def __init__(self, ptr):
        self._ptr = ptr
        f = ptr.contents
        self.m, self.n, self.rank = f.m, f.n, f.rank
        self.f_dtype = _TORCH[f.f_dtype]
        self.precision = f.precision
        self.rel_err, self.norm_a, self.eps, self.t_margin = f.rel_err, f.norm_a, f.eps, f.t_margin
        self.blocks, self.restarts, self.block_k = f.blocks, f.restarts, f.block_k
        self.tdiag = [f.tdiag[i] for i in range(f.ntdiag)]

    def _view(self, name, rows, cols, ld, dtype):
        ptr = getattr(self._ptr.contents, name)
        if self.rank == 0 or not ptr:
            return torch.zeros((rows, cols), dtype=dtype, device="cuda")
        return torch.as_tensor(_DevArray(ptr, rows, cols, ld, dtype, self), device="cuda")

    @property
    def U(self):
        return self._view("U", self.m, self.rank, self.m, self.f_dtype)

    @property
    def V(self):
        return self._view("V", self.n, self.rank, self.n, self.f_dtype)

    @property
    def Q(self):
        return self._view("Q", self.m, self.rank, self.m, self.f_dtype)

    @property
    def Ct(self):
        return self._view("C", self.n, self.rank, self.n, self.f_dtype)

    @property
    def D(self):
        return self._view("D", self.rank, self.rank, self.rank, torch.float64)

    def reconstruct(self, stream=None) -> torch.Tensor:
        dt = self.f_dtype
        out = torch.empty((self.n, self.m), dtype=dt, device="cuda").t()
        o = make_opts(dtype=_DT[dt], stream=stream)
        st = _lib.eod_abe_reconstruct(self._ptr, ctypes.c_void_p(out.data_ptr()), self.m, ctypes.byref(o))
        if st != EOD_OK:
            raise EodError(st, "eod_abe_reconstruct")
        return out

    def close(self):
        if self._ptr is not None:
            _lib.eod_abe_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor(A: torch.Tensor, tol: float, seed: int = 0, *, precision="plain", tol_mode="abs", block_k=0,
           compute_err=True, stream=None, batch_index=0, power_iters=0) -> Factors:
    """Alg. 2 (power_iters = tau subspace iterations, 0 = power-free) on a
    column-major CUDA matrix (float64 or float32)."""
    if not A.is_cuda:
        raise ValueError("A must live on the GPU; use factor_host for host matrices")
    if A.dtype not in _DT:
        raise ValueError("A must be float64 or float32")
    lda = _colmajor_ld(A)
    o = make_opts(_DT[A.dtype], precision, tol_mode, block_k, compute_err, stream, batch_index, power_iters)
    out = ctypes.POINTER(EodFactors)()
    st = _lib.eod_abe_factor_ex(ctypes.c_void_p(A.data_ptr()), A.shape[0], A.shape[1], lda, float(tol),
                                int(seed), ctypes.byref(o), ctypes.byref(out))
    if st != EOD_OK:
        raise EodError(st, "eod_abe_factor_ex")
    return Factors(out)


def factor_host(A: torch.Tensor, tol: float, seed: int = 0, *, precision="plain", tol_mode="abs", block_k=0,
                compute_err=True, stream=None, U_out=None, D_out=None, V_out=None, power_iters=0):
    """Host matrix in, host factors out (through eod_abe_factor_host).
    Returns (rank, rel_err)."""
    if A.is_cuda:
        raise ValueError("factor_host takes a host matrix")
    lda = _colmajor_ld(A)
    m, n = A.shape
    cap = min(m, n)
    o = make_opts(_DT[A.dtype], precision, tol_mode, block_k, compute_err, stream, 0, power_iters)
    rank = ctypes.c_int64(0)
    rel = ctypes.c_double(0.0)

    def p(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    st = _lib.eod_abe_factor_host(ctypes.c_void_p(A.data_ptr()), m, n, lda, float(tol), int(seed), ctypes.byref(o),
                                  p(U_out), p(D_out), p(V_out), cap, ctypes.byref(rank), ctypes.byref(rel))
    if st != EOD_OK:
        raise EodError(st, "eod_abe_factor_host")
    return rank.value, rel.value


def factor_batched(mats, tol: float, seed: int = 0, *, precision="plain", tol_mode="abs", block_k=0,
                   compute_err=True, stream=None, power_iters=0):
    """Factors a list of column-major CUDA matrices of one dtype; returns
    (list of Factors or None, list of statuses)."""
    count = len(mats)
    dt = mats[0].dtype
    P = (ctypes.c_void_p * count)(*[ctypes.c_void_p(a.data_ptr()) for a in mats])
    Ms = (ctypes.c_int64 * count)(*[a.shape[0] for a in mats])
    Ns = (ctypes.c_int64 * count)(*[a.shape[1] for a in mats])
    Ls = (ctypes.c_int64 * count)(*[_colmajor_ld(a) for a in mats])
    outs = (ctypes.POINTER(EodFactors) * count)()
    stat = (ctypes.c_int32 * count)()
    o = make_opts(_DT[dt], precision, tol_mode, block_k, compute_err, stream, 0, power_iters)
    _lib.eod_abe_factor_batched(P, Ms, Ns, Ls, count, float(tol), int(seed), ctypes.byref(o), outs, stat)
    res = [Factors(outs[i]) if stat[i] == EOD_OK else None for i in range(count)]
    return res, [int(s) for s in stat]


def compress_channels(channels, tol: float, seed: int = 0, *, precision="plain", tol_mode="rel", block_k=0,
                      power_iters=0, peak: float = 255.0):
    """Image compression with adaptive rank (Sec. 1 and Sec. 4): every
    channel (a column-major CUDA matrix, one dtype) is factored as
    U D V^T through the batched entry point; the report gives each
    channel's rank, the entries its factors store (U, the upper triangle of
    D, V) against m n, RelErr, and PSNR = 10 log10(peak^2 m n / ||A - A_hat||_F^2)
    from the library's own error pass (||A - A_hat||_F = RelErr ||A||_F), plus
    the totals over the channels.  Returns (report dict, list of Factors)."""
    res, st = factor_batched(list(channels), tol, seed, precision=precision, tol_mode=tol_mode, block_k=block_k,
                             compute_err=True, power_iters=power_iters)
    for s in st:
        if s != EOD_OK:
            raise EodError(s, "eod_abe_factor_batched")
    per = []
    tot_err2, tot_px, tot_entries, tot_orig = 0.0, 0, 0, 0
    for A, f in zip(channels, res):
        m, n = A.shape
        err2 = (f.rel_err * f.norm_a) ** 2
        psnr = float("inf") if err2 == 0.0 else 10.0 * math.log10(peak * peak * m * n / err2)
        ent = storage_entries(m, n, f.rank)
        per.append({"m": m, "n": n, "rank": f.rank, "entries": ent, "entries_full": m * n,
                    "rel_err": f.rel_err, "psnr_db": psnr})
        tot_err2 += err2
        tot_px += m * n
        tot_entries += ent
        tot_orig += m * n
    total = {"entries": tot_entries, "entries_full": tot_orig, "saved": 1.0 - tot_entries / tot_orig,
             "psnr_db": float("inf") if tot_err2 == 0.0 else 10.0 * math.log10(peak * peak * tot_px / tot_err2)}
    return {"channels": per, "total": total}, res


def omega(n: int, col0: int, ncols: int, seed: int, batch: int = 0, stream=None) -> torch.Tensor:
    """Columns col0 .. col0+ncols-1 of the Gaussian test matrix, FP64, on the GPU."""
    out = torch.empty((ncols, n), dtype=torch.float64, device="cuda").t()
    if stream is None:
        stream = torch.cuda.current_stream()
    st = _lib.eod_abe_omega(n, col0, ncols, int(seed), int(batch), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(stream.cuda_stream))
    if st != EOD_OK:
        raise EodError(st, "eod_abe_omega")
    return out


def model_flops(m: int, n: int, r: int, k: int, with_err: bool = True) -> float:
    return float(_lib.eod_abe_model_flops(m, n, r, k, 1 if with_err else 0))


def storage_entries(m: int, n: int, r: int) -> int:
    return int(_lib.eod_abe_storage_entries(m, n, r))

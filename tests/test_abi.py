"""The C-ABI library: loads, exports what include/*.h declares, and rejects
bad arguments on the host before any device work (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def eod():
    import __graft_entry__ as g
    g.build()
    import paper_2506_22713_gb300 as eod
    return eod


def _declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"EOD_API\s+[\w\s\*]+?\b(eod_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(eod):
    names = _declared_symbols()
    assert len(names) >= 12
    lib = ctypes.CDLL(eod.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(eod.EXPORTED) | set(names)


def test_status_strings_and_version(eod):
    assert eod.status_string(0) == "ok"
    assert "invalid" in eod.status_string(1)
    assert eod.eod_abe_version().decode().startswith("eod-abe-gb300")


def test_storage_entries_matches_worked_example(eod):
    # Sec. 1: ranks 50/52/53 of a 220 x 220 RGB image -> 72284 entries
    assert sum(eod.storage_entries(220, 220, r) for r in (50, 52, 53)) == 72284


def test_model_flops_cost_table(eod):
    # Sec. 3.4: 2mnr + mr^2 + 2nr^2 + 2r^3 + 4mrk multiply-adds (+ mnr for Q C)
    m, n, r, k = 512, 384, 20, 32
    ma = 2 * m * n * r + m * r * r + 2 * n * r * r + 2 * r ** 3 + 4 * m * r * k
    assert eod.model_flops(m, n, r, k, with_err=False) == 2 * ma
    assert eod.model_flops(m, n, r, k, with_err=True) == 2 * ma + 2 * m * n * r


@pytest.mark.parametrize("m,n,lda,tol", [(0, 5, 1, 1e-3), (5, 0, 5, 1e-3), (5, 5, 4, 1e-3), (5, 5, 5, 0.0),
                                         (5, 5, 5, -1.0), (5, 5, 5, float("nan")), (5, 5, 5, float("inf"))])
def test_factor_rejects_bad_arguments(eod, m, n, lda, tol):
    out = ctypes.POINTER(eod.EodFactors)()
    dummy = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    st = eod.eod_abe_factor(dummy, m, n, lda, tol, 1, ctypes.byref(out))
    assert st == eod.EOD_EINVAL
    assert not out


def test_factor_rejects_null_and_bad_options(eod):
    out = ctypes.POINTER(eod.EodFactors)()
    assert eod.eod_abe_factor(None, 4, 4, 4, 1e-3, 1, ctypes.byref(out)) == eod.EOD_EINVAL
    dummy = ctypes.c_void_p(0x1000)
    for field, val in [("power_iters", -1), ("power_iters", 17), ("a_dtype", 7), ("precision", 9), ("tol_mode", 3), ("block_k", 129),
                       ("block_k", -1)]:
        o = eod.EodOpts()
        eod.eod_opts_default(ctypes.byref(o))
        setattr(o, field, val)
        st = eod.eod_abe_factor_ex(dummy, 4, 4, 4, 1e-3, 1, ctypes.byref(o), ctypes.byref(out))
        assert st == eod.EOD_EINVAL, field
    assert eod.eod_abe_factor_ex(dummy, 4, 4, 4, 1e-3, 1, None, None) == eod.EOD_EINVAL


def test_omega_and_batched_reject_bad_arguments(eod):
    assert eod.eod_abe_omega(0, 0, 1, 1, 0, ctypes.c_void_p(0x1000), None) == eod.EOD_EINVAL
    assert eod.eod_abe_omega(4, -1, 1, 1, 0, ctypes.c_void_p(0x1000), None) == eod.EOD_EINVAL
    assert eod.eod_abe_omega(4, 0, 1, 1, 0, None, None) == eod.EOD_EINVAL
    assert eod.eod_abe_omega(1 << 33, 0, 1, 1, 0, ctypes.c_void_p(0x1000), None) == eod.EOD_EINVAL
    assert eod.eod_abe_factor_batched(None, None, None, None, 0, 1e-3, 1, None, None, None) == eod.EOD_EINVAL


def test_opts_default_layout(eod):
    o = eod.EodOpts()
    eod.eod_opts_default(ctypes.byref(o))
    assert (o.a_dtype, o.precision, o.tol_mode, o.block_k, o.power_iters, o.compute_err) == (0, 0, 0, 0, 0, 1)
    assert ctypes.sizeof(eod.EodOpts) == 40
    assert ctypes.sizeof(eod.EodFactors) == 8 * 3 + 4 * 2 + 8 * 5 + 8 + 8 + 8 * 4 + 8 * 3


def test_free_null_is_noop(eod):
    eod.eod_abe_free(None)


def test_bounded_wait_hook_rejects_bad_budgets(eod):
    # checked on the host before any launch
    assert eod.eod_abe_debug_bounded_wait(0, 1, None) == eod.EOD_EINVAL
    assert eod.eod_abe_debug_bounded_wait(-5, 0, None) == eod.EOD_EINVAL
    assert eod.eod_abe_debug_bounded_wait(4000000001, 0, None) == eod.EOD_EINVAL


def test_tuning_table_parse_lookup_and_reload(eod, tmp_path):
    """The autotuner's table: ranges match inclusively, of several matching
    rows the nearest (log distance to the centre of each range) wins, a
    malformed file is refused without touching the loaded table, a missing
    file empties it (host-side only)."""
    good = tmp_path / "t.txt"
    good.write_text("# comment\n"
                    "block_k 2 2 4096 16384 4096 16384 96   # mixed, large\n"
                    "block_k 0 3 1 100000 1 100000 48\n"
                    "f32_tile 4096 1000000 256 512 128 100000 128\n"
                    "f32_tile 5488 12289 42 97 257 577 128   # measured at N = 64, K = 384\n"
                    "f32_tile 5488 12289 64 145 128 577 64   # measured at N = 96, K = 272\n")
    try:
        assert eod.eod_abe_tuning_load(str(good).encode()) == eod.EOD_OK
        assert eod.tuning_lookup("block_k", 2, 8192, 8192) == 96
        assert eod.tuning_lookup("block_k", 2, 16384, 4096) == 96
        assert eod.tuning_lookup("block_k", 2, 2048, 8192) == 48
        assert eod.tuning_lookup("block_k", 4, 10, 10) is None
        assert eod.tuning_lookup("f32_tile", 8192, 455, 455) == 128
        assert eod.tuning_lookup("f32_tile", 8192, 64, 455) == 128      # only the N = 64 row holds it
        assert eod.tuning_lookup("f32_tile", 8192, 96, 384) == 64       # both hold it; N = 96 is nearer
        assert eod.tuning_lookup("f32_tile", 8192, 64, 384) == 128      # both hold it; N = 64 is nearer
        assert eod.tuning_lookup("f32_tile", 8192, 30, 384) is None
        assert eod.tuning_lookup("batch_workers", 256, 1000, 1000) is None
        bad = tmp_path / "bad.txt"
        bad.write_text("block_k 2 1 1 2 1 2 7\n")          # lo > hi
        assert eod.eod_abe_tuning_load(str(bad).encode()) == eod.EOD_EINVAL
        assert eod.tuning_lookup("block_k", 2, 8192, 8192) == 96
        bad.write_text("block_k 1 2 3\n")                   # too few fields
        assert eod.eod_abe_tuning_load(str(bad).encode()) == eod.EOD_EINVAL
        assert eod.eod_abe_tuning_load(str(tmp_path / "missing.txt").encode()) == eod.EOD_OK
        assert eod.tuning_lookup("block_k", 2, 8192, 8192) is None
    finally:
        eod.eod_abe_tuning_load(None)


def test_autotune_merge_keeps_skipped_keys_and_round_trips(eod, tmp_path):
    """autotune --merge keeps the rows and notes of the skipped keys from the
    table already at --out; the table it writes parses in the library, and
    the committed table holds the measured core leaf width at both ranks."""
    from paper_2506_22713_gb300 import autotune

    old = tmp_path / "old.txt"
    old.write_text("# measured: block_k harmonic 8192^2 mixed: k=64:6.5ms -> 64\n"
                   "# measured: core_leaf harmonic 8192^2 mixed (p = 455): 32:6.6ms, 64:6.3ms -> 64\n"
                   "# measured: batch_workers pixel batch 256 mixed: 8:884ms, 12:834ms -> 12\n"
                   "block_k 2 2 4096 16384 4096 16384 64\n"
                   "core_leaf 304 683 0 0 0 0 64\n"
                   "batch_workers 64 4096 563 2253 592 2371 12\n")
    rows, notes = autotune.kept_rows(str(old), {"core_leaf", "batch_workers"})
    assert rows == [("core_leaf", 304, 683, 0, 0, 0, 0, 64), ("batch_workers", 64, 4096, 563, 2253, 592, 2371, 12)]
    assert [n.split(" ", 1)[0] for n in notes] == ["core_leaf", "batch_workers"]
    new = tmp_path / "new.txt"
    autotune.write_table(str(new), [("block_k", 2, 2, 4096, 16384, 4096, 16384, 96)] + rows,
                         ["block_k harmonic 8192^2 mixed: k=96:6.3ms -> 96"] + notes, {"gpu": "test"})
    text = new.read_text()
    assert text.count("# measured: ") == 3
    try:
        assert eod.eod_abe_tuning_load(str(new).encode()) == eod.EOD_OK
        assert eod.tuning_lookup("block_k", 2, 8192, 8192) == 96
        assert eod.tuning_lookup("core_leaf", 455, 0, 0) == 64
        assert eod.tuning_lookup("core_leaf", 2037, 0, 0) is None
        assert eod.tuning_lookup("batch_workers", 256, 1100, 1100) == 12
        committed = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                 "paper_2506_22713_gb300", "tuning.txt")
        assert eod.eod_abe_tuning_load(committed.encode()) == eod.EOD_OK
        assert eod.tuning_lookup("core_leaf", 455, 0, 0) == 64
        assert eod.tuning_lookup("core_leaf", 2037, 0, 0) == 64
    finally:
        eod.eod_abe_tuning_load(None)


def test_f32_gemm_hook_rejects_bad_arguments(eod):
    P = ctypes.c_void_p(16)   # never dereferenced: rejected before any launch
    assert eod.eod_abe_debug_f32_gemm(48, 0, 0, 8, 8, 8, 1.0, P, 8, P, 8, 0.0, P, 8, None) == eod.EOD_EINVAL
    assert eod.eod_abe_debug_f32_gemm(0, 0, 0, 8, 8, 8, 1.0, P, 7, P, 8, 0.0, P, 8, None) == eod.EOD_EINVAL
    assert eod.eod_abe_debug_f32_gemm(0, 0, 0, 0, 8, 8, 1.0, P, 8, P, 8, 0.0, P, 8, None) == eod.EOD_EINVAL

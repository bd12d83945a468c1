"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/sirius.h
declares; host-side argument checks answer without touching a GPU (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sirius.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    return sirius.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sirius_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_operator_calls():
    names = declared_functions()
    for want in ("sirius_filter", "sirius_hash_join_build", "sirius_hash_join_probe",
                 "sirius_groupby_agg", "sirius_run_pipeline", "sirius_gather_i64"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_2508_04701_gb300 import sirius
    assert set(declared_functions()) <= set(sirius.SIGNATURES), \
        set(declared_functions()) - set(sirius.SIGNATURES)


def test_host_side_queries(lib):
    assert lib.sirius_version() >= 100
    assert lib.sirius_join_table_capacity(1000, 0.5) > 1000
    assert lib.sirius_join_table_capacity(1000, 0.9) > 1000
    assert lib.sirius_join_table_bytes(lib.sirius_join_table_capacity(1000, 0.5), 4) >= 256 + 8 * 2000
    assert lib.sirius_join_table_bytes(10, 3) == 0
    assert lib.sirius_groupby_capacity(1000) >= 2000
    assert lib.sirius_filter_scratch_bytes(0) >= 256
    assert lib.sirius_filter_scratch_bytes(10**9) >= 8 * (10**9 // 32768)   # a status word per 32768-row tile


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_2508_04701_gb300 import sirius as S
    # n out of range, bad op, NULL column: all INVALID with a message
    assert lib.sirius_filter(None, -1, 0, 0, None, None, None, None, 0, None) == S.ERR_INVALID
    assert "out of range" in S.last_error()
    assert lib.sirius_filter(None, 10, 9, 0, None, None, None, None, 0, None) == S.ERR_INVALID
    assert lib.sirius_filter(None, 10, 0, 0, None, None, None, None, 0, None) == S.ERR_INVALID
    assert lib.sirius_filter(None, 1 << 32, 0, 0, None, None, None, None, 0, None) == S.ERR_INVALID
    t = S.JoinTable(None, 100, 4, 0)
    assert lib.sirius_hash_join_build(None, None, 10, ctypes.byref(t), None, None) == S.ERR_INVALID
    t = S.JoinTable(4096, 10, 4, 0)
    assert lib.sirius_hash_join_build(8, None, 10, ctypes.byref(t), None, None) == S.ERR_INVALID
    assert "capacity" in S.last_error()
    assert lib.sirius_groupby_agg(None, 3, None, 0, 15, 10, None, None, None, None, None, 0, None,
                                  None, None, 0, None) == S.ERR_INVALID
    d = S.PipelineDesc()
    d.n, d.m, d.op = 5, 5, 0
    r = S.Result()
    assert lib.sirius_run_pipeline(ctypes.byref(d), ctypes.byref(r), None, 0, None) == S.ERR_INVALID
    d.fk = d.pred = d.val = d.pk = d.grp = 4096
    d.op = 17
    assert lib.sirius_run_pipeline(ctypes.byref(d), ctypes.byref(r), None, 0, None) == S.ERR_INVALID
    d.op = 0
    d.load_factor = 0.99
    assert lib.sirius_run_pipeline(ctypes.byref(d), ctypes.byref(r), None, 0, None) == S.ERR_INVALID
    d.load_factor = 0
    d.split_probe = 3
    assert lib.sirius_run_pipeline(ctypes.byref(d), ctypes.byref(r), None, 0, None) == S.ERR_INVALID
    assert "split_probe" in S.last_error()


def test_scratch_size_query_grows_with_inputs(lib):
    from paper_2508_04701_gb300 import sirius as S
    d = S.PipelineDesc()
    d.m = 1000
    small = lib.sirius_pipeline_scratch_bytes(ctypes.byref(d))
    d.m = 1_000_000
    big = lib.sirius_pipeline_scratch_bytes(ctypes.byref(d))
    assert big > small > 0
    d.group_cap_hint = 100
    assert lib.sirius_pipeline_scratch_bytes(ctypes.byref(d)) < big


def test_struct_layouts_match_header(tmp_path):
    """Every struct the binding passes through the C ABI has the header's size and field offsets
    (a small C program built against include/sirius.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2508_04701_gb300 import sirius as S
    structs = {"sirius_pipeline_desc": S.PipelineDesc, "sirius_result": S.Result,
               "sirius_dim_index": S.DimIndex, "sirius_join_table": S.JoinTable,
               "sirius_semijoin": S.Semijoin}
    lines = ['#include "sirius.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, v = line.split()
        got[(cname, field)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_string_calls_reject_bad_arguments_on_the_host(lib):
    from paper_2508_04701_gb300 import sirius as S
    h = ctypes.c_int64(0)
    enc = lib.sirius_dict_encode
    assert enc(None, None, 0, 5, 10, 0, None, None, 0, None, ctypes.byref(h), None, 0, None) == S.ERR_INVALID
    assert enc(None, None, 0, 0, 10, 2, None, None, 0, None, ctypes.byref(h), None, 0, None) == S.ERR_INVALID
    assert enc(None, None, 1 << 31, 0, 10, 0, None, None, 0, None, None, None, 0, None) == S.ERR_INVALID
    assert enc(None, None, 0, -1, 10, 0, None, None, 0, None, None, None, 0, None) == S.ERR_INVALID
    gb = lib.sirius_groupby_string
    assert gb(None, None, 0, None, 0, 10, 0, 15, None, None, None, None, None, 0, None, None, None, 0,
              None) == S.ERR_INVALID  # NULL count output
    assert lib.sirius_dict_capacity(1000) >= 1000
    assert lib.sirius_groupby_string_scratch_bytes(10**6, 1000) > lib.sirius_dict_scratch_bytes(10**6, 1000)


def test_wait_selftests_reject_bad_arguments_on_the_host(lib):
    from paper_2508_04701_gb300 import sirius as S
    st, passed = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.sirius_selftest_grid_barrier(0, 0, 16, None, 0, ctypes.byref(st), ctypes.byref(passed),
                                            None) == S.ERR_INVALID
    assert "blocks" in S.last_error()
    assert lib.sirius_selftest_lookback_timeout(None, 0, ctypes.byref(st), None) == S.ERR_INVALID
    assert "256 bytes" in S.last_error()


def test_injected_allocation_failure_host_side(lib):
    """The failure-injection hook fails the next library-owned scratch allocation with OOM before
    any device work (here: a group-by over no rows with no caller scratch), and counts down."""
    from paper_2508_04701_gb300 import sirius as S
    assert lib.sirius_inject_alloc_failures(2) == 0
    st = lib.sirius_groupby_agg(None, 4, None, 0, 15, 10, None, None, None, None, None, 0, None, None,
                                None, 0, None)
    assert st == S.ERR_OOM and "injected" in S.last_error()
    assert lib.sirius_inject_alloc_failures(0) == 1      # one was used, one still pending; cancelled
    assert lib.sirius_inject_alloc_failures(0) == 0

"""The C ABI library (no GPU needed): it loads, exports every symbol that
include/mf.h declares, its structs match the binding, and argument errors are
reported before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

import __graft_entry__
from paper_1109_1146_gb300 import mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mf.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return mf.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_binding_exports():
    assert _declared() == sorted(mf.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", mf.LIBPATH]).decode()
    exported = set(re.findall(r" T (mf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    for s in _declared():
        assert hasattr(lib, s)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mf.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(mf_opts), sizeof(mf_stats),'
                   ' offsetof(mf_stats, ms_init), offsetof(mf_stats, flow_value));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    a, b, c, d = map(int, subprocess.check_output([str(exe)]).split())
    assert a == ctypes.sizeof(mf.mf_opts)
    assert b == ctypes.sizeof(mf.mf_stats)
    assert c == mf.mf_stats.ms_init.offset and d == mf.mf_stats.flow_value.offset


def test_default_opts(lib):
    o = mf.default_opts()
    assert (o.max_sweeps, o.partial_discharge, o.global_gap, o.global_relabel_period, o.max_rounds) == (0, 0, 1, 4, 0)


@pytest.mark.parametrize("ndim,dims,conn,tile,frag", [
    (2, (10, 10, 1), 6, None, "connectivity"),
    (3, (10, 10, 10), 4, None, "connectivity"),
    (2, (0, 10, 1), 4, None, "dims"),
    (2, (10, 10, 1), 4, (48, 48, 1), "tile"),
    (3, (10, 10, 10), 6, (32, 32, 32), "tile"),
])
def test_create_rejects_bad_arguments(lib, ndim, dims, conn, tile, frag):
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 3)(*dims)
    t = None if tile is None else (ctypes.c_int32 * 3)(*tile)
    st = lib.mf_create_grid(ctypes.byref(h), ndim, d, conn, t, None)
    assert st == mf.MF_EINVAL
    assert h.value is None
    assert frag in lib.mf_last_error(None).decode()


def test_null_handle_calls(lib):
    assert lib.mf_destroy(None) == mf.MF_OK
    assert lib.mf_solve(None, None, None) == mf.MF_EINVAL
    assert lib.mf_set_caps(None, None, None, None, 0) == mf.MF_EINVAL
    v = ctypes.c_int64()
    assert lib.mf_flow_value(None, ctypes.byref(v)) == mf.MF_EINVAL


def test_every_export_has_a_ctypes_signature():
    # a call without argtypes would pass 64-bit device pointers as C int
    assert set(mf.SIGNATURES) == set(mf.EXPORTS)

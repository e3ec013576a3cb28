"""The C ABI library loads on a CPU-only host, exports every function that
include/qedpic.h declares, and the Python binding's structures have the
header's layout.  Only argument checks that run before any CUDA call are
exercised here (no compute without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1311_1107_gb300 import build as B
from paper_1311_1107_gb300 import qedpic as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qedpic.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qp_init_tables", "qp_create_species", "qp_step", "qp_diagnostics",
                     "qp_destroy", "qp_status_string", "qp_export_tables"):
        assert required in names


def test_binding_constants_match_the_header():
    text = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(QP_\w+)\s+(-?\d+)\b", text))
    for name in ("QP_MAX_EMISSIONS", "QP_MAX_BATCH", "QP_STEP_TILE"):
        assert int(defs[name]) == getattr(Q, name), name


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (qp_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(Q.EXPORTS) <= exported


def test_struct_layouts_match_header(tmp_path):
    structs = {"qp_table_params": Q.qp_table_params, "qp_species_desc": Q.qp_species_desc,
               "qp_field": Q.qp_field, "qp_step_params": Q.qp_step_params,
               "qp_diag": Q.qp_diag, "qp_tables_export": Q.qp_tables_export,
               "qp_coalesce_params": Q.qp_coalesce_params,
               "qp_coalesce_stats": Q.qp_coalesce_stats, "qp_pulse2d": Q.qp_pulse2d,
               "qp_host_state": Q.qp_host_state}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qedpic.h"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in got.splitlines():
        name, field, value = line.split()
        cls = structs[name]
        if field == "size":
            assert C.sizeof(cls) == int(value), name
        else:
            assert getattr(cls, field).offset == int(value), (name, field)


def test_status_strings(lib):
    assert Q.qp_status_string(0) == "QP_OK"
    assert Q.qp_status_string(Q.QP_ERR_TIMEOUT) == "QP_ERR_TIMEOUT"
    assert Q.qp_status_string(Q.QP_WARN_BUFFER_FULL) == "QP_WARN_BUFFER_FULL"
    assert Q.qp_status_string(12345) == "QP_UNKNOWN_STATUS"


def test_arguments_rejected_before_any_device_work(lib):
    ctx = C.c_void_p()
    bad = Q.qp_table_params(-1.0, 0, 0)
    assert lib.qp_init_tables(C.byref(bad), C.byref(ctx)) == Q.QP_ERR_INVALID_ARG
    assert ctx.value is None
    assert lib.qp_init_tables(None, C.byref(ctx)) == Q.QP_ERR_INVALID_ARG
    bad2 = Q.qp_table_params(0.8e-6, 0, 7)
    assert lib.qp_init_tables(C.byref(bad2), C.byref(ctx)) == Q.QP_ERR_INVALID_ARG
    s = Q.qp_step_params()
    assert lib.qp_step(None, C.byref(s), None) == Q.QP_ERR_NOT_INITIALIZED
    d = Q.qp_diag()
    assert lib.qp_diagnostics(None, 0, C.byref(d), None) == Q.QP_ERR_NOT_INITIALIZED
    desc = Q.qp_species_desc()
    h = C.c_int32()
    assert lib.qp_create_species(None, C.byref(desc), C.byref(h)) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_selftest_wait_timeout(None, 10) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_destroy(None) == Q.QP_OK
    assert lib.qp_destroy_species(None, 0) == Q.QP_ERR_NOT_INITIALIZED
    b = C.c_void_p()
    assert lib.qp_batch_create(None, 4, Q.QP_MIXED, Q.QP_FIELD_GAUSSIAN,
                               C.byref(b)) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_batch_set(None, 0, C.byref(s), None, 0, None) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_batch_step(None, 1, None) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_batch_clear(None, 0, None) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_batch_progress(None, None, None, None, None) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_batch_destroy(None) == Q.QP_ERR_NOT_INITIALIZED
    assert lib.qp_species_copy(None, 0, None, 8, 1, 1, None) == Q.QP_ERR_NOT_INITIALIZED
    hs = (Q.qp_host_state * 3)()
    assert lib.qp_step_host(None, C.byref(s), hs, None) == Q.QP_ERR_NOT_INITIALIZED


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(Q, "_lib", None)
    monkeypatch.setattr(Q._build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        Q.lib()

"""The C-ABI library loads and exports every function include/bcd.h
declares; the binding's signature table covers the same set. No GPU needed:
nothing here calls into device code."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bcd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(bc_[A-Za-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_1708_08739_gb300 import build
    build.build()
    import paper_1708_08739_gb300 as bcd
    return bcd


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["bc_graph_create", "bc_graph_destroy", "bc_rv_compute", "bc_exact", "bc_approx", "bc_approx_T",
              "bc_batch", "bc_draw_samples", "bc_spd_probe", "bc_last_error"]:
        assert f in names


def test_library_exports_every_declared_symbol(built_lib):
    import ctypes
    L = ctypes.CDLL(built_lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(built_lib._SIGNATURES) == declared_functions()


def test_binding_loads_and_reports_version(built_lib):
    assert "sm_103a" in built_lib.bc_version()
    assert built_lib.bc_last_error() == ""
    assert built_lib.bc_samples_for(0.01, 0.1) == 14979
    assert built_lib.bc_samples_for(0.02, 0.1) == 3745
    with pytest.raises(built_lib.BCError):
        built_lib.bc_samples_for(0.0, 0.1)


def test_no_oracle_in_product_path():
    """The CUDA library and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1708_08739_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "bc_oracle" not in src and "liboracle" not in src, f


STRUCTS = ["bc_graph_desc", "bc_info", "bc_query", "bc_result", "bc_batch_info", "bc_config", "bc_server_config",
           "bc_server_stats", "bc_tune_report"]


def test_binding_struct_layouts_match_the_header(built_lib, tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets, as a C compiler lays them out (gcc on the header itself)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bcd.h"', "int main(void) {"]
    for name in STRUCTS:
        py = getattr(built_lib, name)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        name, field, value = line.split()
        py = getattr(built_lib, name)
        if field == "size":
            assert ctypes.sizeof(py) == int(value), name
        else:
            assert getattr(py, field).offset == int(value), (name, field)
        seen += 1
    assert seen == sum(1 + len(getattr(built_lib, n)._fields_) for n in STRUCTS)


def test_host_only_argument_checks(built_lib):
    """Calls whose argument checks run on the host before any device work."""
    b = built_lib
    with pytest.raises(b.BCError) as e:
        b.bc_debug_fail_alloc(-1)
    assert e.value.status == b.BC_E_INVALID_ARG
    b.bc_debug_fail_alloc(0)
    assert b.lib().bc_cancel(None) == b.BC_E_INVALID_ARG
    assert b.lib().bc_set_config(None, None) == b.BC_E_INVALID_ARG

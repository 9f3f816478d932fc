"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/theseus_gb.h declares; the Python binding covers
the same names.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2508_05029_gb300 import build, theseus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tp_init", "tp_shutdown", "tp_page_alloc", "tp_table_append", "tp_plan_create",
                 "tp_execute", "tp_result_sum", "tp_last_error", "tp_set_device_budget"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header():
    assert set(theseus.SIGNATURES) == declared_functions()


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2508_05029_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "liboracle" not in src, f
                assert "orc_" not in src, f


def test_struct_layout_matches_c(tmp_path):
    """ctypes mirrors of the header structs have the C compiler's sizes and offsets."""
    import subprocess
    checks = {
        "tp_config": ["page_bytes", "n_pages", "device_budget_bytes", "prefetch_depth", "batch_rows",
                      "load_factor", "agg_strategy", "compute_stream"],
        "tp_plan_desc": ["fact", "dim", "filter", "join", "n_group", "group", "n_agg", "aggs",
                         "agg_strategy", "load_factor", "expected_groups", "join_partitions", "dim_filter",
                         "dim_filter_on", "lip", "n_extra_dims", "extra_dim", "extra_join", "extra_dim_filter",
                         "extra_dim_filter_on", "join_many"],
        "tp_stats": ["h2d_bytes", "retries", "pages_in_use", "pages_total", "agg_kernel_rows", "jit_compiles",
                     "jit_launches", "jit_compile_ms", "agg_split_passes", "lip_filters",
                     "part_build_ms", "part_stream_ms", "part_spilled_ms"],
        "tp_i128": ["lo", "hi"],
        "tp_agg": ["kind", "col_a", "col_b", "k"],
        "tp_table_desc": ["n_cols", "cols", "batch_rows"],
        "tp_column_desc": ["name", "type", "scale"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "theseus_gb.h"', "int main(void){"]
    for st, fields in checks.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, fields in checks.items():
        cls = getattr(theseus, st)
        assert ctypes.sizeof(cls) == int(out[st]), st
        for f in fields:
            assert getattr(cls, f).offset == int(out[f"{st}.{f}"]), (st, f)

"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
and exports every function that include/*.h declares; host-side argument
validation that runs before any device call."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(vx_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("vx_open", "vx_register_host_column", "vx_filter", "vx_run_plan", "vx_groupby"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2502_09541_gb300 as vx
    lib = vx.load()  # builds in-tree with nvcc if needed; loading needs no GPU
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding marshals exactly the declared names
    assert set(vx.SIGNATURES) <= declared_functions()


STRUCTS = ["vx_config", "vx_pred", "vx_plan_dim", "vx_plan_gkey", "vx_plan", "vx_query_stats", "vx_result",
           "vx_sort_opts", "vx_sort_stats", "vx_join_opts", "vx_join_result", "vx_serve_opts", "vx_serve_stats",
           "vx_op_request", "vx_op_result"]


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets the C
    compiler gives the header's structures."""
    import subprocess

    import paper_2502_09541_gb300 as vx
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vx.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(vx, s)._fields_:
            lines.append(f'  printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for s in STRUCTS:
        cls = getattr(vx, s)
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(out[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_null_and_bad_arguments_fail_without_a_device():
    import paper_2502_09541_gb300 as vx
    lib = vx.load()
    out = ctypes.c_void_p()
    assert lib.vx_open(0, ctypes.byref(out)) == vx.VX_E_INVAL
    assert lib.vx_close(None) == vx.VX_OK
    assert lib.vx_run_plan(None, None, None) == vx.VX_E_INVAL
    assert "null context" in vx.vx_last_error()
    assert lib.vx_set_config(None, None) == vx.VX_E_INVAL

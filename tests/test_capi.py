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


def test_struct_layouts_match_header():
    import paper_2502_09541_gb300 as vx
    # sizes follow the C layout of include/vx.h on LP64 targets
    assert ctypes.sizeof(vx.vx_pred) == 16
    assert ctypes.sizeof(vx.vx_plan_gkey) == 16
    assert ctypes.sizeof(vx.vx_plan_dim) == 4 * (3 + 4 + 1 + 16)
    assert ctypes.sizeof(vx.vx_config) == 48


def test_null_and_bad_arguments_fail_without_a_device():
    import paper_2502_09541_gb300 as vx
    lib = vx.load()
    out = ctypes.c_void_p()
    assert lib.vx_open(0, ctypes.byref(out)) == vx.VX_E_INVAL
    assert lib.vx_close(None) == vx.VX_OK
    assert lib.vx_run_plan(None, None, None) == vx.VX_E_INVAL
    assert "null context" in vx.vx_last_error()
    assert lib.vx_set_config(None, None) == vx.VX_E_INVAL

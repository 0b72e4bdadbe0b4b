"""The C-ABI library loads and exports every entry point include/bemgb.h declares.

CPU only: no compute calls (only the pure-host default-options call).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bemgb.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("bem_", "lm_"))))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._load_build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("bem_create", "bem_setup", "bem_factor", "bem_eval", "bem_vjp", "bem_jtj",
              "lm_step", "bem_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    import paper_2602_05492_gb300 as bg
    assert sorted(bg.EXPORTED) == _declared()


def test_default_opts(lib):
    import paper_2602_05492_gb300 as bg
    o = bg.bem_opts()
    assert bg.bem_default_opts(ctypes.byref(o)) == 0
    assert o.precision == bg.BEM_FP64 and o.eps_d == 1e-2 and o.eps_c == 1e-2
    assert o.segs_per_side == 256 and o.near_factor == 0.5
    assert o.jtj_mode == bg.BEM_JTJ_FP64 and o.lm_solver == bg.BEM_LM_AUTO
    assert o.galerkin_mode == 0
    assert bg.bem_default_opts(None) == bg.BEM_EINVAL


def test_struct_layout_matches_header():
    """bem_opts / lm_result sizes agree with the C compiler's layout."""
    import subprocess
    import tempfile
    import paper_2602_05492_gb300 as bg
    src = ('#include "bemgb.h"\n#include <stdio.h>\n#include <stddef.h>\n'
           'int main(void){printf("%zu %zu %zu\\n", sizeof(bem_opts), sizeof(lm_result),'
           ' offsetof(bem_opts, galerkin_mode));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        a, b, off = map(int, subprocess.run([exe], capture_output=True, text=True,
                                            check=True).stdout.split())
    assert a == ctypes.sizeof(bg.bem_opts) and b == ctypes.sizeof(bg.lm_result)
    assert off == bg.bem_opts.galerkin_mode.offset

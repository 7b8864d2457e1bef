"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/zda.h declares; the binding's descriptor matches the header; host-side
argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "zda.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zda_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    build = __graft_entry__._build_module()
    p = build.lib_path()
    srcs = [os.path.join(build.CSRC, s) for s in build.SOURCES] + [os.path.join(ROOT, "include", "zda.h")]
    if not os.path.exists(p) or os.path.getmtime(p) < max(os.path.getmtime(s) for s in srcs):
        build.build()
    return p


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert "zda_forward" in names and "zda_adjoint" in names and len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2501_07979_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_descriptor_layout_matches_header(libpath):
    """sizeof/offsets of the ctypes descriptor equal the C compiler's."""
    import subprocess
    import tempfile
    from paper_2501_07979_gb300 import _lib
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "zda.h"
int main(void){
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(zda_zone_desc), offsetof(zda_zone_desc, layer_eps),
         offsetof(zda_zone_desc, focal), sizeof(zda_zone_info), offsetof(zda_zone_info, workspace_bytes),
         offsetof(zda_zone_info, cells));
  return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    D, Inf = _lib.ZoneDesc, _lib.ZoneInfo
    want = [ctypes.sizeof(D), D.layer_eps.offset, D.focal.offset, ctypes.sizeof(Inf),
            Inf.workspace_bytes.offset, Inf.cells.offset]
    assert got == want


def test_invalid_arguments_return_status_not_crash(libpath):
    from paper_2501_07979_gb300 import _lib
    L = _lib.load(libpath)
    h = ctypes.c_void_p()
    # no context: ZDA_ERR_ARG, and a message
    assert L.zda_zone_create(None, None, ctypes.byref(h)) == _lib.ERR_ARG
    assert L.zda_last_error()
    assert L.zda_zone_query(None, None) == _lib.ERR_ARG
    assert L.zda_zone_launch_count(None) == -1

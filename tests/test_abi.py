"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/zda.h declares; the binding's descriptor matches the header; host-side
argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


HEADERS = ["zda.h", "zda_nn.h"]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(zda_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    build = __graft_entry__._build_module()
    p = build.lib_path()
    srcs = [os.path.join(build.CSRC, s) for s in build.SOURCES] + [os.path.join(ROOT, "include", h) for h in HEADERS]
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
    form = ctypes.c_int()
    assert L.zda_zone_set_radial_pml(None, 1) == _lib.ERR_ARG
    assert L.zda_zone_get_radial_pml(None, ctypes.byref(form)) == _lib.ERR_ARG
    # the order bound is host-only: bad stride, no points, non-positive wavelengths
    from paper_2501_07979_gb300.zone import make_desc
    from zda_inputs import zone_tiny
    d = make_desc(zone_tiny())
    lam = (ctypes.c_double * 1)(1.0)
    pts = (ctypes.c_double * 3)(0.5, 0.0, 0.0)
    b = ctypes.c_double()
    assert L.zda_zone_order_bound(ctypes.byref(d), lam, 1, pts, 1, 4, ctypes.byref(b)) == _lib.ERR_ARG
    assert L.zda_zone_order_bound(ctypes.byref(d), lam, 1, pts, 0, 2, ctypes.byref(b)) == _lib.ERR_ARG
    assert L.zda_zone_order_bound(ctypes.byref(d), (ctypes.c_double * 1)(0.0), 1, pts, 1, 2,
                                  ctypes.byref(b)) == _lib.ERR_ARG
    assert L.zda_zone_order_bound(ctypes.byref(d), lam, 1, pts, 1, 3, ctypes.byref(b)) == 0 and b.value > 0


def test_surrogate_descriptor_checks_and_sizes_need_no_gpu(libpath):
    """zda_nn_create validates its descriptor on the host and reports the
    parameter count and forward FLOPs of the architecture the oracle defines."""
    from oracle import surrogate as S
    from paper_2501_07979_gb300 import _lib
    L = _lib.load(libpath)
    h = ctypes.c_void_p()
    bad = _lib.NnDesc(batch=2, height=12, width=16, in_ch=1, out_ch=24)      # H not a multiple of 8
    assert L.zda_nn_create(0, ctypes.byref(bad), ctypes.byref(h)) == _lib.ERR_ARG
    bad = _lib.NnDesc(batch=2, height=16, width=16, in_ch=17, out_ch=24)
    assert L.zda_nn_create(0, ctypes.byref(bad), ctypes.byref(h)) == _lib.ERR_ARG
    bad = _lib.NnDesc(batch=2, height=16, width=184, in_ch=1, out_ch=24)      # window would not fit
    assert L.zda_nn_create(0, ctypes.byref(bad), ctypes.byref(h)) == _lib.ERR_ARG
    d = _lib.NnDesc(batch=4, height=32, width=24, in_ch=2, out_ch=24)
    assert L.zda_nn_create(0, ctypes.byref(d), ctypes.byref(h)) == _lib.OK
    n = ctypes.c_size_t()
    f = ctypes.c_double()
    ws = ctypes.c_size_t()
    assert L.zda_nn_param_count(h, ctypes.byref(n)) == _lib.OK
    assert L.zda_nn_forward_flops(h, ctypes.byref(f)) == _lib.OK
    assert L.zda_nn_workspace_bytes(h, ctypes.byref(ws)) == _lib.OK
    assert n.value == S.param_count(2, 24)
    assert f.value == S.forward_flops(32, 24, 2, 24)
    assert ws.value > 4 * 4 * n.value
    # unbound: calls that need the workspace report a state error
    assert L.zda_nn_adam(h, 1e-3, 0.9, 0.999, 1e-8, None) == _lib.ERR_STATE
    L.zda_nn_destroy(h)


def test_filter_radius_beyond_the_tap_limit_is_refused(libpath):
    """A conic-filter radius spanning more than ZDA_MAX_FILTER_TAPS taps per
    pixel is refused by zone creation and by the allocation-free filter call
    (host-side checks, before any device work)."""
    from paper_2501_07979_gb300 import _lib
    from paper_2501_07979_gb300.zone import make_desc
    from zda_inputs import zone_tiny
    L = _lib.load(libpath)
    big = zone_tiny(filter_radius=150.0)          # 31 x 2803 taps: the radial span is clipped to the design rows
    ok = zone_tiny(filter_radius=0.25)
    ctx = ctypes.create_string_buffer(64)         # zone creation only stores the context pointer
    h = ctypes.c_void_p()
    assert L.zda_zone_create(ctx, ctypes.byref(make_desc(big)), ctypes.byref(h)) == _lib.ERR_ARG
    assert b"taps" in L.zda_last_error()
    assert L.zda_zone_create(ctx, ctypes.byref(make_desc(ok)), ctypes.byref(h)) == _lib.OK
    L.zda_zone_destroy(h)
    x = ctypes.c_void_p(16)                       # never dereferenced: the call fails first
    assert L.zda_filter_project_noalloc(ctypes.byref(make_desc(big)), x, x, None) == _lib.ERR_ARG
    assert b"taps" in L.zda_last_error()
    neg = zone_tiny(pml_r_in=-2)
    assert L.zda_filter_project_noalloc(ctypes.byref(make_desc(neg)), x, x, None) == _lib.ERR_ARG


def test_evaluation_calls_check_their_arguments_before_any_device_work(libpath):
    from paper_2501_07979_gb300 import _lib
    L = _lib.load(libpath)
    out = (ctypes.c_double * 16)()
    inc = (ctypes.c_double * 2)(1.0, 1.0)
    nb = ctypes.c_size_t()
    assert L.zda_lens_evaluate_scratch_bytes(None, 8, 4, 4, ctypes.byref(nb)) == _lib.ERR_ARG
    assert L.zda_lens_evaluate(None, 10.0, 20.0, inc, 1.0, 8, 4.0, 4, 4, 64, None, 0, out, None, None) == _lib.ERR_ARG
    assert L.zda_zone_incident_intensity(None, None, None) == _lib.ERR_ARG
    assert L.zda_field_intensity(None, 1, 1, 1.0, None, None) == _lib.ERR_ARG
    assert L.zda_encircled_power(None, None, 1, 0, None, None) == _lib.ERR_ARG
    assert b"bad argument" in L.zda_last_error() or b"null" in L.zda_last_error()

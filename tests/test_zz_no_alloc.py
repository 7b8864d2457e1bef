"""The allocation-free filter + projection entry point.

zda_filter_project_noalloc serves callers that cannot call cudaMalloc (their
device memory belongs to another framework's pool, or their loop may not
allocate once running): it takes only the zone description, the input and
the output, and keeps its scratch in a fixed device array inside the library.
This file is collected last on purpose.  Two calls in a row, on different
densities, must each match zda_filter_project (the workspace-based entry
point) within the filter tests' tolerance.
"""
import ctypes

import numpy as np
import pytest
import torch

from zda_inputs import zone_cfg2, zone_tiny, rho_for, smoothed_rho

pytestmark = pytest.mark.gpu

TOL = 5e-6       # same as the filter/projection parity tests


@pytest.mark.parametrize("which", ["wide", "ragged", "axis"])
def test_noalloc_filter_project_matches_workspace_entry_point(which):
    from paper_2501_07979_gb300 import Zone, _lib, make_desc
    if which == "wide":
        spec = zone_cfg2(n_steps=10)
    elif which == "ragged":
        spec = zone_tiny(n_r=27, n_phi=7, pml_r_in=3, pml_r_out=5, filter_radius=0.2, beta=3.0, n_steps=10)
    else:                                                        # continuous axisymmetry, axis inside
        spec = zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, filter_radius=0.25, beta=4.0, n_steps=10)
    desc = make_desc(spec)
    L = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    zone = Zone(spec, device=0)
    for call, seed in enumerate((21, 22)):                      # two calls in a row
        rho = torch.tensor(smoothed_rho(spec.n_r_design, spec.n_phi, seed, mode="minmax"),
                           dtype=torch.float32, device="cuda:0")
        out = torch.full_like(rho, float("nan"))
        rc = L.zda_filter_project_noalloc(ctypes.byref(desc), ctypes.c_void_p(rho.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.zda_last_error()
        want = zone.filter_project(rho)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out - want).abs().max().item() < TOL, call


def test_noalloc_rejects_too_many_rows():
    from paper_2501_07979_gb300 import _lib, make_desc
    spec = zone_tiny(n_r=16384 + 9, pml_r_in=4, pml_r_out=4, filter_radius=0.2)
    L = _lib.lib()
    x = torch.zeros(8, device="cuda:0")
    rc = L.zda_filter_project_noalloc(ctypes.byref(make_desc(spec)), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), None)
    assert rc == _lib.ERR_ARG
    assert b"no-allocation limit" in L.zda_last_error()

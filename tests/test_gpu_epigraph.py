"""Max-min over wavelengths (Eqs. 7-8) on the GPU zone: per-wavelength
adjoint gradients against the oracle's, and a CCSA epigraph run that raises
the weakest wavelength's focal intensity."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2501_07979_gb300.topopt import (Epigraph, wavelength_intensities, wavelength_sensitivity,
                                             zone_wavelength_objectives)
from zda_inputs import smoothed_rho, zone_tiny

pytestmark = pytest.mark.gpu

SPEC = zone_tiny(n_steps=700, filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1), eps_hi=2.1,
                 pulse_sigma=0.4, pulse_t0=1.6)


def test_per_wavelength_gradients_match_oracle():
    from paper_2501_07979_gb300 import Zone
    zone = Zone(SPEC, device=0)
    obj = zone_wavelength_objectives(zone, 2)
    rho = smoothed_rho(SPEC.n_r_design, SPEC.n_phi, 21, mode="minmax")
    I, grads = obj(rho)
    fwd = O.forward(SPEC, rho)
    fwd["rho"] = rho
    geom = fwd["geom"]
    rbar = O.conic_filter(SPEC, geom, rho)
    assert np.allclose(I, wavelength_intensities(fwd["S"], 2), rtol=2e-4)
    for l in range(2):
        adj = O.adjoint(SPEC, fwd, wavelength_sensitivity(fwd["S"], 2, l))
        ref = O.conic_filter_T(SPEC, geom, adj["grad_rho_tilde"] * O.project_grad(SPEC, rbar))
        rel = np.linalg.norm(grads[l] - ref) / np.linalg.norm(ref)
        assert rel < 1e-3, (l, rel)


def test_epigraph_raises_the_weakest_wavelength():
    from paper_2501_07979_gb300 import Zone
    zone = Zone(SPEC, device=0)
    obj = zone_wavelength_objectives(zone, 2)
    rho0 = np.full((SPEC.n_r_design, SPEC.n_phi), 0.5)
    I0 = obj(rho0, False)
    ep = Epigraph(obj, rho0)
    ep.run(6)
    assert ep.history[-1]["min_I"] > 1.5 * float(np.min(I0))
    assert all(h["q"] <= h["min_I"] * (1 + 1e-6) + 1e-12 for h in ep.history)

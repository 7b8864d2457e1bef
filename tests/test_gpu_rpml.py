"""The stretched-coordinate r-PML (form 1, zda_zone_set_radial_pml) on the
GPU against the oracle (section "Differentiable FDTD in cylindrical
coordinates": stretched radius in the equations, regularised r-PML).

Forward DFTs, fields and phasors (pair kernels, one-cell kernels, the axis
zone) and the adjoint gradient at the parity tolerances of the default form,
and the reflection of the outer r-PML measured through the C ABI against a
radially larger zone (same r_lo, so the same time step)."""
import numpy as np
import pytest
import torch

import oracle as O
from zda_inputs import ZoneSpec, zone_tiny, smoothed_rho, rho_for

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
GRAD_TOL = 1e-3
KERNELS = {"split": (0, 2, 0), "split1": (2, 2, 0)}


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda:0")


def _zone(spec, kernel="split", form=1):
    from paper_2501_07979_gb300 import Zone
    z = Zone(spec, device=0)
    z.set_kernel(*KERNELS[kernel])
    z.set_radial_pml(form)
    return z


def _oracle(spec, rho):
    g = O.Geometry(spec)
    pml = O.cpml_coefficients(spec, g, metric=True)
    eps = O.site_eps(spec, g, O.rho_tilde(spec, g, rho))
    t = g.dt * (np.arange(spec.n_steps) + 0.5)
    mon, des, st = O.run(spec, g, eps, pml=pml, src_pat=O.plane_wave_pattern(spec, g),
                         src_time=O.pulse(spec, t)[:, None].astype(complex), twiddle=O.twiddles(g, spec.n_steps),
                         state=np.zeros((O.N_STATE, spec.n_r, spec.n_phi, spec.n_z), complex))
    return mon, des, st, O.focal_phasors(spec, g, mon)


def _probe(n_r, n_steps):
    """lambda/20 wedge at r = 5 lambda: substrate, 0.6 lambda design layer,
    monitor 0.5 lambda above it, 8-cell PMLs."""
    return ZoneSpec(r_lo=4.6, n_r=n_r, n_phi=4, n_z=64, n_fold=48, dr=0.05, dz=0.05, pml_r_in=8, pml_r_out=8,
                    pml_z=8, layer_k0=(0, 22, 34), layer_eps=(2.1, 1.0, 1.0), design_k0=22, design_k1=34,
                    eps_lo=1.0, eps_hi=5.76, source_k=12, monitor_k=44, courant=0.5, n_steps=n_steps,
                    wavelengths=(1.0,), pulse_sigma=0.5, pulse_t0=2.0)


SPECS = {
    "tiny": zone_tiny(n_steps=300),                                  # pair kernels
    "ragged": zone_tiny(n_r=27, n_phi=7, n_z=45, pml_r_in=3, pml_r_out=5, pml_z=5, n_steps=250,
                        layer_k0=(0, 15, 19), design_k0=15, design_k1=19, source_k=8, monitor_k=26,
                        wavelengths=(0.85, 1.0, 1.2), filter_radius=0.2, beta=3.0, pulse_sigma=0.4,
                        pulse_t0=1.6),                               # odd n_z: one-cell kernels
    "no_inner_pml": zone_tiny(pml_r_in=0, n_steps=200),
    "probe": _probe(56, 400),
}


@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("name", list(SPECS))
def test_stretched_rpml_forward_matches_oracle(name, kernel):
    spec = SPECS[name]
    rho = rho_for(spec, 1)
    z = _zone(spec, kernel)
    assert z.radial_pml() == 1
    S = z.forward(_dev(rho))
    mon, des, st, S_ref = _oracle(spec, rho)
    assert _rel(z.monitor_dft().cpu().numpy(), mon) < FIELD_TOL
    assert _rel(np.moveaxis(z.design_dft(0).cpu().numpy(), 4, 2), des) < FIELD_TOL
    assert _rel(z.fields().cpu().numpy(), st[:6]) < FIELD_TOL
    assert _rel(S, S_ref) < FIELD_TOL


def test_stretched_rpml_gradient_matches_oracle():
    spec = zone_tiny(n_steps=700, filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1), pulse_sigma=0.4,
                     pulse_t0=1.6)
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 5, mode="minmax")
    z = _zone(spec)
    S = z.forward(_dev(rho))
    grad = z.adjoint(4.0 * S).cpu().numpy()
    _, g_ref, fwd, adj = O.gradient(spec, rho, pml_form=1)
    assert _rel(S, fwd["S"]) < FIELD_TOL
    assert _rel(np.moveaxis(z.design_dft(1).cpu().numpy(), 4, 2), adj["des_adj"]) < GRAD_TOL
    assert _rel(grad, g_ref) < GRAD_TOL


def test_stretched_rpml_axis_zone_matches_oracle():
    """Continuous axisymmetry with the axis inside: outer slab only, i m / r~."""
    spec = zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_steps=700, filter_radius=0.25, beta=4.0,
                     wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6)
    rho = smoothed_rho(spec.n_r_design, 1, 8, mode="minmax")
    z = _zone(spec)
    S = z.forward(_dev(rho))
    mon, des, st, S_ref = _oracle(spec, rho)
    assert _rel(z.monitor_dft().cpu().numpy(), mon) < FIELD_TOL
    assert _rel(z.fields().cpu().numpy(), st[:6]) < FIELD_TOL
    assert _rel(S, S_ref) < FIELD_TOL
    grad = z.adjoint(4.0 * S).cpu().numpy()
    _, g_ref, _, _ = O.gradient(spec, rho, pml_form=1)
    assert _rel(grad, g_ref) < GRAD_TOL


def test_fused_step_refuses_the_stretched_form():
    from paper_2501_07979_gb300 import Zone, ZdaError
    spec = SPECS["tiny"]
    z = Zone(spec, device=0)
    assert z.radial_pml() == 0                              # default: real-radius CPML
    z.set_kernel(1, 2, 0)
    with pytest.raises(ZdaError, match="ZDA_ERR_ARG"):
        z.set_radial_pml(1)
    z.set_kernel(0, 2, 0)
    z.set_radial_pml(1)
    with pytest.raises(ZdaError, match="ZDA_ERR_ARG"):
        z.set_kernel(1, 2, 0)
    with pytest.raises(ZdaError, match="ZDA_ERR_ARG"):
        z.set_radial_pml(2)


def test_outer_r_pml_reflection_drops_with_the_stretched_form():
    """Monitor DFT over the interior of a zone against the same zone extended
    outwards by 10 lambda (whose outer wall is out of reach in the 10-period
    window; same r_lo, so the same time step), plane wave scattered by a
    random design: the difference is the outer r-PML's reflection.  Oracle
    (FP64): 5.2e-3 with the default form, 2.2e-4 with the stretched form."""
    W, L = 40, 200
    rho = smoothed_rho(W, 4, 7, mode="minmax")
    rho_ref = np.zeros((W + L, 4))
    rho_ref[:W] = rho
    out = {}
    for form in (0, 1):
        a = _zone(_probe(W + 16, 581), form=form)
        b = _zone(_probe(W + 16 + L, 581), form=form)
        assert a.dt == b.dt
        a.forward(_dev(rho))
        b.forward(_dev(rho_ref))
        ma = a.monitor_dft().cpu().numpy()[:, :, 8:8 + W]
        mb = b.monitor_dft().cpu().numpy()[:, :, 8:8 + W]
        out[form] = _rel(ma, mb)
    print("outer r-PML reflection (monitor DFT, r = 5.4 lambda): form 0 %.3e, form 1 %.3e" % (out[0], out[1]))
    assert out[0] > 2e-3
    assert out[1] < 5e-4 and out[1] < out[0] / 10

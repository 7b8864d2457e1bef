"""Direct pins of the oracle's smaller pieces (the time loop's pins live in
test_oracle_pins.py):

* site averaging (Eq. 6 + the arithmetic-mean reading): closed form for a
  uniform density, and site_eps_T is the exact transpose of site_eps;
* the broadband adjoint profiles (section "Differentiable FDTD": broadband
  adjoint sources): their discrete DFT at -w_j is delta_qj, and they carry no
  DC component;
* the objective's gradient convention (I = 2 sum abs(S)^2);
* the transmitted-power estimate: the plane-wave closed form
  (n/2) abs(E0)^2 pi (r1^2 - r0^2) of a uniform x-polarised field, and the
  circle average of a phi-dependent intensity.
"""
import math

import numpy as np

import oracle as O
from zda_inputs import zone_tiny


def _spec():
    return zone_tiny(n_r=14, n_phi=6, n_z=30, pml_r_in=3, pml_r_out=3, pml_z=4, layer_k0=(0, 12, 17),
                     layer_eps=(2.1, 1.0, 1.0), design_k0=12, design_k1=17, eps_lo=1.0, eps_hi=5.76,
                     source_k=6, monitor_k=22, n_fold=30, n_steps=200, wavelengths=(0.9, 1.0, 1.2))


def test_site_eps_of_a_uniform_density():
    spec = _spec()
    g = O.Geometry(spec)
    c = 0.37
    rt = np.full((spec.n_r_design, spec.n_phi), c)
    er, ep, ez = O.site_eps(spec, g, rt)
    design = spec.eps_lo + c * (spec.eps_hi - spec.eps_lo)
    i0, i1 = g.i_d0, g.i_d1
    k0, k1 = spec.design_k0, spec.design_k1
    # interior of the design layer, away from its radial edges: the design value everywhere
    assert np.allclose(er[i0 + 1:i1 - 1, :, k0 + 1:k1], design, rtol=0, atol=1e-14)
    assert np.allclose(ez[i0 + 1:i1 - 1, :, k0:k1], design, rtol=0, atol=1e-14)
    # the node plane at the layer's bottom averages the substrate below and the layer above
    assert np.allclose(er[i0 + 1:i1 - 1, :, k0], 0.5 * (spec.layer_eps[0] + design), atol=1e-14)
    # the PML columns hold eps_lo in the design layer, so the first interior E_phi column averages them
    assert np.allclose(ep[i0, :, k0 + 1:k1], 0.5 * (spec.eps_lo + design), atol=1e-14)


def test_site_eps_T_is_the_transpose_of_site_eps():
    spec = _spec()
    g = O.Geometry(spec)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((spec.n_r_design, spec.n_phi))
    base = O.site_eps(spec, g, np.zeros_like(x))
    lin = [a - b for a, b in zip(O.site_eps(spec, g, x), base)]          # the linear part
    gs = [rng.standard_normal(a.shape) for a in lin]
    lhs = sum(float(np.sum(a * b)) for a, b in zip(lin, gs))
    rhs = float(np.sum(x * O.site_eps_T(spec, g, *gs)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_profiles_have_the_required_spectrum():
    spec = _spec()
    g = O.Geometry(spec)
    n = 900
    k = O.adjoint_pulse_matrix(spec, g, n)                                 # [n][q]
    t_half = g.dt * (np.arange(n) + 0.5)
    D = (np.exp(-1j * np.outer(g.omega, t_half)) @ k) * g.dt            # [j][q]: DFT at -w_j
    assert np.abs(D - np.eye(g.n_freq)).max() < 1e-9
    # no DC component (first differences of pulses that vanish at both ends)
    assert np.abs(k.sum(axis=0)).max() < 1e-6 * np.abs(k).sum(axis=0).min()


def test_intensity_gradient_convention():
    rng = np.random.default_rng(2)
    S = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    g = O.intensity_grad(S)
    h = 1e-6
    for q in range(S.size):
        e = np.zeros(S.size, complex)
        e[q] = h
        d_re = (O.intensity(S + e) - O.intensity(S - e)) / (2 * h)
        d_im = (O.intensity(S + 1j * e) - O.intensity(S - 1j * e)) / (2 * h)
        assert abs(g[q] - (d_re + 1j * d_im)) < 1e-6 * abs(g[q])


def test_transmitted_power_of_a_uniform_plane_wave():
    """x-polarised field E0 (E_r = E0 cos phi, E_phi = -E0 sin phi): its m = +1
    part (E0/2, i E0/2) e^{i phi} goes to the +w entries, the conjugate of its
    m = -1 part to the -w entries (the signed-frequency reading)."""
    spec = _spec()
    g = O.Geometry(spec)
    nl = g.n_lambda
    E0 = np.array([1.3 - 0.4j, 0.7 + 0.2j, 2.0 + 0.0j])
    mon = np.zeros((g.n_freq, 2, spec.n_r, spec.n_phi), complex)
    ephn = np.exp(1j * g.phi_n)[None, :]
    ephh = np.exp(1j * g.phi_h)[None, :]
    for l in range(nl):
        mon[l, 0] = 0.5 * E0[l] * ephn
        mon[l, 1] = 0.5j * E0[l] * ephh
        mon[l + nl, 0] = 0.5 * np.conj(E0[l]) * ephn                     # conj of (E0/2) e^{-i phi}
        mon[l + nl, 1] = 0.5j * np.conj(E0[l]) * ephh                    # conj of (-i E0/2) e^{-i phi}
    P = O.transmitted_power(spec, g, mon)
    n_top = math.sqrt(spec.layer_eps[-1])
    want = 0.5 * n_top * np.abs(E0) ** 2 * math.pi * (g.r1 ** 2 - g.r0 ** 2)
    assert np.allclose(P, want, rtol=1e-12)


def test_transmitted_power_averages_a_phi_dependent_intensity():
    """E_r = 2 cos(phi), E_phi = 0 (orders +-1 with equal radial parts): the
    intensity 4 cos^2(phi) averages to 2 over the circle, not its value 4 near
    phi = 0 on the first wedge; with n = 2 the copies at phi and phi + pi
    carry the same intensity, so the wedge's own average counts."""
    spec = _spec()
    g = O.Geometry(spec)
    nl = g.n_lambda
    mon = np.zeros((g.n_freq, 2, spec.n_r, spec.n_phi), complex)
    for l in range(nl):
        mon[l, 0] = np.exp(1j * g.phi_n)[None, :]
        mon[l + nl, 0] = np.exp(1j * g.phi_n)[None, :]
    n_top = math.sqrt(spec.layer_eps[-1])
    area = math.pi * (g.r1 ** 2 - g.r0 ** 2)
    assert np.allclose(O.transmitted_power(spec, g, mon), 0.5 * n_top * 2.0 * area, rtol=1e-12)
    half = spec.replace(n_fold=2, n_phi=8)                 # wedge = half circle, 8 phi cells
    gh = O.Geometry(half)
    mh = np.zeros((gh.n_freq, 2, half.n_r, half.n_phi), complex)
    for l in range(nl):
        mh[l, 0] = np.exp(1j * gh.phi_n)[None, :]
        mh[l + nl, 0] = np.exp(1j * gh.phi_n)[None, :]
    want = 0.5 * n_top * np.mean(4 * np.cos(gh.phi_n) ** 2) * area     # the wedge samples' mean
    assert np.allclose(O.transmitted_power(half, gh, mh), want, rtol=1e-12)

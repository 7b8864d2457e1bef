"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: Bessel-zero
resonances of a PEC cavity, exact energy conservation of the leap-frog
scheme, the Yee dispersion relation, Fresnel transmission, the wedge/full-
circle Bloch identity, the weighted adjointness of the discrete curls, the
Rayleigh-Sommerfeld closed form for an annulus, filter/projection identities,
finite differences of the objective, and numbers printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special as sp
from scipy.optimize import brentq

import oracle as O
from zda_inputs import ZoneSpec, zone_tiny, smoothed_rho, focal_from_na, zone_cfg1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _first_root(f, lo, hi, n=2000):
    xs = np.linspace(lo, hi, n)
    fs = [f(x) for x in xs]
    for a, b, fa, fb in zip(xs[:-1], xs[1:], fs[:-1], fs[1:]):
        if fa * fb < 0:
            return brentq(f, a, b, xtol=1e-14)
    raise AssertionError("no root")


def _pec_spec(**kw):
    base = dict(pml_r_in=0, pml_r_out=0, pml_z=0, layer_k0=(0,), layer_eps=(1.0,),
                design_k0=0, design_k1=0, courant=0.5)
    base.update(kw)
    return ZoneSpec(**base)


def _enforce_pec(st):
    st[0][:, :, 0] = 0          # E_r on z = 0
    st[1][0] = 0                # E_phi on r = r_lo
    st[1][:, :, 0] = 0          # E_phi on z = 0
    st[2][0] = 0                # E_z on r = r_lo
    st[3][0] = 0                # H_r normal to r = r_lo
    st[5][:, :, 0] = 0          # H_z normal to z = 0
    return st


def _volumes(spec, geom):
    s = spec
    vh = (geom.r_h * s.dr * geom.dphi * s.dz)[:, None, None]
    vn = (geom.r_n[:s.n_r] * s.dr * geom.dphi * s.dz)[:, None, None]
    return [vh, vn, vn], [vn, vh, vh]     # E_r, E_phi, E_z ; H_r, H_phi, H_z


# ---------------------------------------------------------------- T1
def _cavity_error(dr, mode, a=5.0, b=6.0, n_fold=40, nphi=8, d=1.0, n_steps=3000):
    """Relative error of the discrete resonance wt^2 of the lowest TM_{1,1,0}
    or TE_{1,1,1} mode of a PEC annular wedge cavity against the Bessel
    cross-product zero (phi-difference order M_eff = (2/dphi) sin(dphi/2))."""
    nr = int(round((b - a) / dr))
    nz = 2 if mode == "TM" else int(round(d / dr))
    s = _pec_spec(r_lo=a, n_r=nr, n_phi=nphi, n_z=nz, n_fold=n_fold, dr=dr,
                  dz=(dr if mode == "TM" else d / nz))
    g = O.Geometry(s)
    M = 2 * math.sin(g.dphi / 2) / g.dphi
    st = np.zeros((O.N_STATE, nr, nphi, nz), complex)
    if mode == "TM":
        f = lambda k: sp.jv(M, k * a) * sp.yv(M, k * b) - sp.jv(M, k * b) * sp.yv(M, k * a)
        kr = _first_root(f, 0.5, 20)
        R = lambda r: sp.jv(M, kr * r) * sp.yv(M, kr * a) - sp.jv(M, kr * a) * sp.yv(M, kr * r)
        prof = R(g.r_n[:nr])
        prof[0] = 0
        st[2] = prof[:, None, None] * np.exp(1j * g.phi_n)[None, :, None] * np.ones((1, 1, nz))
        w2, comp, site = kr ** 2, 2, (nr // 3, 0, 0)
    else:
        f = lambda k: sp.jvp(M, k * a) * sp.yvp(M, k * b) - sp.jvp(M, k * b) * sp.yvp(M, k * a)
        kr = _first_root(f, 0.5, 20)
        R = lambda r: sp.jv(M, kr * r) * sp.yvp(M, kr * a) - sp.jvp(M, kr * a) * sp.yv(M, kr * r)
        kz = 2 / s.dz * math.sin(math.pi * s.dz / (2 * d))
        sz = np.sin(math.pi * s.dz * np.arange(nz) / d)[None, None, :]
        Rh = R(g.r_h)
        dR = np.zeros(nr)
        dR[1:] = (Rh[1:] - Rh[:-1]) / dr
        # divergence-free transverse E of the TE mode
        st[0] = (1j * M / g.r_h * Rh)[:, None, None] * np.exp(1j * g.phi_n)[None, :, None] * sz
        st[1] = (-dR)[:, None, None] * np.exp(1j * g.phi_h)[None, :, None] * sz
        w2, comp, site = kr ** 2 + kz ** 2, 1, (nr // 3, 0, nz // 2)
    eps = [np.ones((nr, nphi, nz))] * 3
    sig = np.empty(n_steps, complex)
    for n in range(n_steps):
        _, _, st = O.run(s, g, eps, n_steps=1, pml=O.no_pml(s), state=st)
        sig[n] = st[comp][site]
    # s[n+1] + s[n-1] = 2 cos(w dt) s[n] + const  =>  wt^2 = (2 - 2 cos(w dt)) / dt^2
    A = np.stack([sig[1:-1], np.ones(n_steps - 2)], axis=1)
    c = np.linalg.lstsq(A, sig[2:] + sig[:-2], rcond=None)[0][0].real
    return ((2 - c) / g.dt ** 2 - w2) / w2


@pytest.mark.parametrize("mode", ["TM", "TE"])
def test_T1_cavity_resonances_converge_to_bessel_zeros(mode):
    e1 = _cavity_error(0.05, mode)
    e2 = _cavity_error(0.025, mode)
    assert abs(e1) < 5e-3, e1                       # lambda/20
    assert 3.5 < e1 / e2 < 4.5, (e1, e2)            # second order in dr


# ---------------------------------------------------------------- T2
def test_T2_energy_conserved_with_pec_walls_and_bloch_phase():
    s = _pec_spec(r_lo=5.0, n_r=12, n_phi=6, n_z=10, n_fold=40, dr=0.1, dz=0.1)
    g = O.Geometry(s)
    rng = np.random.default_rng(0)
    eps = O.site_eps(s, g, rng.random((s.n_r_design, s.n_phi)))
    eps = tuple(e + 1.5 * rng.random(e.shape) for e in eps)      # inhomogeneous
    st = np.zeros((O.N_STATE, s.n_r, s.n_phi, s.n_z), complex)
    sh = (6, s.n_r, s.n_phi, s.n_z)
    st[:6] = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    st = _enforce_pec(st)
    VE, VH = _volumes(s, g)
    W = []
    for n in range(400):
        E, Hm = st[:3].copy(), st[3:6].copy()
        _, _, st = O.run(s, g, eps, n_steps=1, pml=O.no_pml(s), state=st)
        W.append(sum((eps[c] * VE[c] * abs(E[c]) ** 2).sum() for c in range(3))
                 + sum((VH[c] * np.real(np.conj(Hm[c]) * st[3 + c])).sum() for c in range(3)))
    W = np.array(W)
    assert np.abs(W / W[0] - 1).max() < 1e-12


# ---------------------------------------------------------------- T3 / T5
def _tem_run(dz, eps1, eps2, lam=1.0, L=10.0):
    """Coaxial TEM pulse (m = 0, E_r ~ 1/r, an exact discrete mode) launched
    in eps1 towards an interface with eps2; returns the DFT of r E_r at
    planes inside medium 2 and the time step."""
    nz = int(round(L / dz))
    pz = int(round(0.5 / dz))
    k_i = nz // 2
    s = ZoneSpec(r_lo=5.0, n_r=int(round(1 / dz)), n_phi=2, n_z=nz, n_fold=40, dr=dz, dz=dz, m=0,
                 pml_r_in=0, pml_r_out=0, pml_z=pz, layer_k0=(0, k_i), layer_eps=(eps1, eps2),
                 design_k0=k_i + nz // 10, design_k1=k_i + nz // 10 + nz // 5, courant=0.5,
                 wavelengths=(lam,), pulse_sigma=1.0, pulse_t0=6.0, n_steps=0)
    g = O.Geometry(s)
    T = int((12.0 + 2 * L * math.sqrt(max(eps1, eps2)) + 10) / g.dt)
    lay = np.where(np.arange(nz) < k_i, eps1, eps2)
    cells = np.broadcast_to(lay, (s.n_r, s.n_phi, nz)).copy()
    er = 0.5 * (cells + O._sh(cells, 2, -1, False))
    pat = np.zeros((1, 2, s.n_r, s.n_phi), complex)
    pat[0, 0] = (1 / g.r_h)[:, None]
    src = O.pulse(s, g.dt * (np.arange(T) + 0.5))[:, None].astype(complex)
    _, des, _ = O.run(s, g, (er, er.copy(), cells), n_steps=T, src_pat=pat, src_time=src,
                      src_k=pz + nz // 20, twiddle=O.twiddles(g, T), mon_k=-1)
    i = s.n_r // 2
    return des[0, 0, :, i, 0] * g.r_h[i], g


@pytest.mark.parametrize("eps", [1.0, 2.1])
def test_T3_numerical_dispersion_matches_yee_relation(eps):
    dz = 0.05
    E, g = _tem_run(dz, eps, eps)
    k = np.angle(E[1:] / E[:-1]).mean() / dz
    lhs = math.sin(g.omega[0] * g.dt / 2) / g.dt
    rhs = math.sin(k * dz / 2) / dz / math.sqrt(eps)
    assert abs(rhs / lhs - 1) < 1e-5
    # and the continuous relation is off by the expected O((k dz)^2) amount
    assert abs(k / (g.omega[0] * math.sqrt(eps)) - 1) > 1e-5


def test_T5_interface_transmission_converges_to_fresnel():
    n1, n2 = math.sqrt(2.1), 1.0
    t_exact = 2 * n1 / (n1 + n2)
    errs = []
    for dz in (0.05, 0.025):
        Ei, _ = _tem_run(dz, 2.1, 2.1)
        Et, _ = _tem_run(dz, 2.1, 1.0)
        assert np.abs(Et).std() / np.abs(Et).mean() < 1e-3        # no standing wave
        errs.append(np.abs(Et).mean() / np.abs(Ei).mean() / t_exact - 1)
    assert abs(errs[0]) < 1e-2, errs
    assert 3.5 < errs[0] / errs[1] < 4.6, errs


# ---------------------------------------------------------------- T4
def test_T4_wedge_equals_first_wedge_of_larger_domains():
    """An n-fold wedge run equals the first wedge of the n/k-fold run with
    k times more phi cells (same dphi) when eps repeats every 2pi/n."""
    rng = np.random.default_rng(3)
    base = dict(r_lo=3.0, n_r=14, n_z=24, dr=0.1, dz=0.1, pml_r_in=3, pml_r_out=3, pml_z=4,
                layer_k0=(0, 10, 14), layer_eps=(2.1, 1.0, 1.0), design_k0=10, design_k1=14,
                eps_lo=1.0, eps_hi=5.76, source_k=6, monitor_k=18, n_steps=150)
    rho = rng.random((8, 6))
    outs = []
    for n_fold, reps in ((8, 1), (2, 4), (1, 8)):
        s = ZoneSpec(n_phi=6 * reps, n_fold=n_fold, **base)
        g = O.Geometry(s)
        eps = O.site_eps(s, g, np.tile(rho, (1, reps)))
        t = g.dt * (np.arange(s.n_steps) + 0.5)
        mon, _, st = O.run(s, g, eps, src_pat=O.plane_wave_pattern(s, g),
                           src_time=O.pulse(s, t)[:, None].astype(complex),
                           twiddle=O.twiddles(g, s.n_steps), design=False,
                           state=np.zeros((O.N_STATE, s.n_r, s.n_phi, s.n_z), complex))
        outs.append((st[:6, :, :6], mon[:, :, :, :6]))
    for st, mon in outs[1:]:
        scale = np.abs(outs[0][0]).max()
        assert np.abs(st - outs[0][0]).max() < 1e-11 * scale
        assert np.abs(mon - outs[0][1]).max() < 1e-11 * np.abs(outs[0][1]).max()


# ---------------------------------------------------------------- T6
def test_T6_discrete_curls_are_weighted_adjoints():
    """<y, C_E x>_{V_H} = <C_H y, x>_{V_E} with the Bloch phase: the H
    update of a random E gives -dt C_E x and the E update of a random H
    (eps = 1) gives dt C_H y."""
    s = _pec_spec(r_lo=4.0, n_r=9, n_phi=5, n_z=7, n_fold=30, dr=0.1, dz=0.1)
    g = O.Geometry(s)
    rng = np.random.default_rng(5)
    sh = (3, s.n_r, s.n_phi, s.n_z)
    x = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    y = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    st = np.zeros((O.N_STATE, s.n_r, s.n_phi, s.n_z), complex)
    st[:3] = x
    st = _enforce_pec(st)
    x = st[:3].copy()
    ones = [np.ones((s.n_r, s.n_phi, s.n_z))] * 3
    _, _, a = O.run(s, g, ones, n_steps=1, pml=O.no_pml(s), state=st)
    CEx = -a[3:6] / g.dt
    st = np.zeros_like(st)
    st[3:6] = y
    st = _enforce_pec(st)
    y = st[3:6].copy()
    _, _, b = O.run(s, g, ones, n_steps=1, pml=O.no_pml(s), state=st)
    CHy = b[:3] / g.dt
    CHy = _enforce_pec(np.concatenate([CHy, np.zeros((11,) + CHy.shape[1:])]))[:3]
    VE, VH = _volumes(s, g)
    lhs = sum((VH[c] * np.conj(y[c]) * CEx[c]).sum() for c in range(3))
    rhs = sum((VE[c] * np.conj(CHy[c]) * x[c]).sum() for c in range(3))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------- T8
def _annulus_closed_form(z, r0, r1, k):
    R0, R1 = math.hypot(z, r0), math.hypot(z, r1)
    return z * np.exp(1j * k * R0) / R0 - z * np.exp(1j * k * R1) / R1


@pytest.mark.parametrize("which", ["E_r", "E_phi"])
def test_T8_rayleigh_sommerfeld_annulus_closed_form(which):
    """A uniform m = +1 field (E_x = U0 / 2 everywhere on the monitor) gives
    the on-axis RS-I field (U0/2) [z e^{ikR0}/R0 - z e^{ikR1}/R1]; each
    component is checked on its own (u_r - i u_phi = U0 from either)."""
    errs = []
    for dr in (0.05, 0.025):
        s = zone_tiny(r_lo=5.0, n_r=int(round(4 / dr)), dr=dr, pml_r_in=int(round(0.5 / dr)),
                      pml_r_out=int(round(0.5 / dr)), n_phi=12, n_fold=40, wavelengths=(0.9, 1.2),
                      focal=7.0)
        g = O.Geometry(s)
        U0 = 0.7 - 0.3j
        mon = np.zeros((g.n_freq, 2, s.n_r, s.n_phi), complex)
        if which == "E_r":
            mon[:, 0] = U0 * np.exp(1j * g.phi_n)[None, None, :]
        else:
            mon[:, 1] = 1j * U0 * np.exp(1j * g.phi_h)[None, None, :]
        S = O.focal_phasors(s, g, mon)
        _, _, zf = O.focal_weights(s, g)
        e = []
        for q in range(g.n_freq):
            k = 2 * math.pi / s.wavelengths[q % g.n_lambda]
            cf = _annulus_closed_form(zf, g.r0, g.r1, k) / 2
            want = U0 * cf if q < g.n_lambda else U0 * np.conj(cf)
            e.append(abs(S[q] - want) / abs(want))
        errs.append(max(e))
    assert errs[0] < 1e-2, errs                   # k dr ~ 0.35 at lambda/20
    assert 3.5 < errs[0] / errs[1] < 4.5, errs    # midpoint / trapezoid: O(dr^2)


def test_plane_wave_pattern_is_x_polarised():
    """m = +1 source plus its conjugate (the m = -1 part) is a uniform x-hat
    current: J_r = cos(phi), J_phi = -sin(phi) at the sites."""
    s = zone_tiny()
    g = O.Geometry(s)
    p = O.plane_wave_pattern(s, g)[0] * s.dz
    assert np.allclose(2 * p[0].real, np.cos(g.phi_n)[None, :])
    assert np.allclose(2 * p[1].real, -np.sin(g.phi_h)[None, :])


# ---------------------------------------------------------------- T9
def _filter_spec():
    return zone_tiny(n_r=30, pml_r_in=4, pml_r_out=4, n_phi=16, dr=0.05, filter_radius=0.17,
                     beta=6.0, eta=0.5)


def test_T9_conic_filter_identities():
    s = _filter_spec()
    g = O.Geometry(s)
    rng = np.random.default_rng(2)
    c = np.full((s.n_r_design, s.n_phi), 0.37)
    assert np.allclose(O.conic_filter(s, g, c), 0.37, atol=1e-15)          # constants kept
    x = rng.random((s.n_r_design, s.n_phi))
    y = rng.random((s.n_r_design, s.n_phi))
    lhs = (O.conic_filter(s, g, x) * y).sum()
    rhs = (x * O.conic_filter_T(s, g, y)).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # one pixel spreads over a cone: the weight falls linearly with distance
    d = np.zeros_like(x)
    d[10, 5] = 1.0
    fd = O.conic_filter(s, g, d)
    assert fd[10, 5] > fd[9, 5] > 0 and fd[10, 5] > fd[10, 4] > 0
    assert fd[10, 5 + 8] == 0.0
    # phi wraps: a pixel at the wedge edge feeds the other edge
    d = np.zeros_like(x)
    d[10, 0] = 1.0
    assert O.conic_filter(s, g, d)[10, -1] > 0


def test_T9_projection_limits_and_gradient():
    s = _filter_spec()
    x = np.linspace(0, 1, 11)
    p = O.project(s, x)
    assert abs(p[0]) < 1e-15 and abs(p[-1] - 1) < 1e-15 and abs(p[5] - 0.5) < 1e-15
    lin = O.project(s.replace(beta=1e-5), x)
    assert np.allclose(lin, x, atol=1e-9)                                   # beta -> 0
    h = 1e-6
    fd = (O.project(s, x + h) - O.project(s, x - h)) / (2 * h)
    assert np.allclose(O.project_grad(s, x), fd, rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------------- T7
def _fd_spec():
    # low-contrast layer (eps_hi = substrate eps): no guided modes, so the
    # fields decay and the frequency-domain adjoint is exact up to decay.
    return zone_tiny(n_steps=3200, courant=0.9, filter_radius=0.25, beta=4.0,
                     wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6, eps_hi=2.1)


def _fd_errors(spec, pixels, h=1e-4):
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 7, mode="minmax")
    _, grad, _, _ = O.gradient(spec, rho)
    errs = []
    for i, j in pixels:
        rp, rm = rho.copy(), rho.copy()
        rp[i, j] += h
        rm[i, j] -= h
        fd = (O.forward(spec, rp)["I"] - O.forward(spec, rm)["I"]) / (2 * h)
        errs.append(abs(grad[i, j] - fd))
    return np.array(errs) / np.abs(grad).max()


def _directional_error(spec, h=1e-3):
    """Relative error of the derivative along v = g / |g| (largest signal)."""
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 7, mode="minmax")
    _, grad, _, _ = O.gradient(spec, rho)
    v = grad / np.linalg.norm(grad)
    fd = (O.forward(spec, rho + h * v)["I"] - O.forward(spec, rho - h * v)["I"]) / (2 * h)
    return abs(fd / np.linalg.norm(grad) - 1)


_FD_PIXELS = [(0, 0), (0, 7), (3, 2), (5, 5), (7, 4), (8, 1), (10, 6), (12, 7), (15, 0), (15, 3)]


def test_T7_adjoint_gradient_matches_central_differences():
    errs = _fd_errors(_fd_spec(), _FD_PIXELS)
    assert errs.max() < 2e-3, errs
    assert _directional_error(_fd_spec()) < 1e-3


# ---------------------------------------------------------------- decay rule, high contrast
def _hc_spec(n_steps):
    # TiO2 (eps 5.76) design layer on SiO2 (eps 2.1): the high-contrast stack of
    # the single-zone and wide-zone workloads, which supports guided modes
    return zone_tiny(n_steps=n_steps, courant=0.9, filter_radius=0.25, beta=4.0,
                     wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6, eps_hi=5.76)


def test_field_energy_closed_form():
    """W of E_r = 1 everywhere (eps 1): sum of r_{i+1/2} dr dphi dz over the
    wedge = tau (r_hi^2 - r_lo^2) / 2 * n_z dz (the midpoint rule is exact)."""
    s = zone_tiny()
    g = O.Geometry(s)
    st = np.zeros((O.N_STATE, s.n_r, s.n_phi, s.n_z), complex)
    st[0] = 1.0
    ones = np.ones((s.n_r, s.n_phi, s.n_z))
    r1 = s.r_lo + s.n_r * s.dr
    want = g.tau * (r1 ** 2 - s.r_lo ** 2) / 2 * s.n_z * s.dz
    assert abs(O.field_energy(s, g, (ones, ones, ones), st) / want - 1) < 1e-12
    st[0] = 0.0
    st[4] = 2.0                                  # H_phi at r_{i+1/2}: 4 x the same sum
    assert abs(O.field_energy(s, g, (ones, ones, ones), st) / (4 * want) - 1) < 1e-12


def test_decay_rule_on_high_contrast_zone():
    """The decay measure Wdot (energy of the one-step difference) falls below
    1e-8 of its peak within the run, while W keeps the static field of the
    source's nonzero time integral (a plateau above 1e-3 of its peak)."""
    s = _hc_spec(10000)
    rho = smoothed_rho(s.n_r_design, s.n_phi, 7, mode="minmax")
    st, w, wd = O.energy_trace(s, rho, 10000, 250)
    T = O.decay_steps(st, wd)
    assert T is not None and 2000 < T < 10000, T
    assert w[-1] / w.max() > 1e-3                # static field: no decay of W
    assert O.decay_steps(st, w) is None
    assert np.all(wd[st >= T] <= 2e-8 * wd.max())


def test_T7_high_contrast_gradient_matches_central_differences():
    """FD check of the adjoint on the high-contrast (TiO2 on SiO2) stack, run
    for the decay rule's T (Wdot <= 1e-8 of its peak): per pixel <= 2e-3 of
    max abs(g), directional <= 1e-3 (measured 4e-4 and 2e-5)."""
    probe = _hc_spec(12000)
    rho = smoothed_rho(probe.n_r_design, probe.n_phi, 7, mode="minmax")
    st, _, wd = O.energy_trace(probe, rho, 12000, 250)
    s = probe.replace(n_steps=O.decay_steps(st, wd))
    errs = _fd_errors(s, _FD_PIXELS)
    assert errs.max() < 2e-3, errs
    assert _directional_error(s) < 1e-3


def test_T7_pin_detects_continuous_omega(monkeypatch):
    """Planted mistake: using w instead of wt = (2/dt) sin(w dt/2) in the
    adjoint (a ~0.5 % scaling at this dt) must break the directional check."""
    monkeypatch.setattr(O.Geometry, "omega_tilde", lambda self: self.omega)
    assert _directional_error(_fd_spec()) > 1e-3


# ---------------------------------------------------------------- paper numbers
def test_paper_focal_lengths_and_pixel_count():
    gold = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    for e in gold["focal_lengths"]:
        assert abs(focal_from_na(e["radius_lambda"], e["na"]) - e["focal_lambda"]) < e["tol_lambda"], e
    p = gold["pixel_count"]
    n = math.pi * p["radius_lambda"] ** 2 / p["pixel_lambda"] ** 2
    assert abs(n / p["pixels"] - 1) < p["rel_tol"]


def test_paper_dof_ratio_and_zone_tiling():
    """The wedge zones of the paper's lenses: with r dphi <= the grid step at
    each zone's outer radius (zone_lwir, zone_visible), the LWIR lens has
    ~10x the design degrees of freedom of its continuously axisymmetric
    twin (zone 1 continuous, zones 2..16 with n_phi pixels per radial pixel);
    the visible lenses' 32 zones tile their printed diameters."""
    from zda_inputs import zone_lwir, zone_visible
    gold = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    g = gold["dof_ratio"]
    zones = [zone_lwir(l, 10) for l in range(2, g["zones"] + 1)]
    nrd = zones[0].n_r_design
    assert nrd * zones[0].dr == pytest.approx(g["zone_width_lambda"])
    dof_ring = nrd + sum(z.n_r_design * z.n_phi for z in zones)      # zone 1: one pixel per radius
    ratio = dof_ring / (g["zones"] * nrd)
    assert abs(ratio / g["ratio"] - 1) < g["rel_tol"], ratio
    v = gold["visible_zone_counts"]
    for lens in ("rgb", "poly"):
        z = zone_visible(v[lens]["zones"], lens, 10)
        outer = z.r_lo + (z.n_r - z.pml_r_out) * z.dr
        assert abs(2 * outer / v[lens]["diameter_lambda"] - 1) < v["rel_tol"], (lens, outer)
        assert z.n_r_design * z.dr == pytest.approx(v[lens]["zone_width_lambda"], rel=1e-3)


def test_cfg1_geometry():
    """The single-zone workload: r dphi and the Courant step of the smallest
    azimuthal spacing; the r_lo * dphi bound must be the binding one."""
    s = zone_cfg1()
    g = O.Geometry(s)
    assert abs(s.r_lo * g.dphi - 2 * math.pi / 96 / 48 * 10) < 1e-15
    assert abs(g.dt - 0.5 / math.sqrt(2 / 0.05 ** 2 + 1 / (10 * g.dphi) ** 2)) < 1e-15
    assert abs(g.dt - 6.361e-3) < 1e-6


# ---------------------------------------------------------------- axis zone (continuous axisymmetry)
def _cylinder_error(dr, mode, a=1.0, d=1.0, n_steps=2500):
    """Full PEC cylinder r in [0, a] in the continuous-axisymmetry (axis
    zone) mode, m = 1: lowest TM_{1,1,0} (J_1 zero) / TE_{1,1,1} (J_1' zero)."""
    nr = int(round(a / dr))
    nz = 2 if mode == "TM" else int(round(d / dr))
    s = _pec_spec(r_lo=0.0, n_r=nr, n_phi=1, n_z=nz, n_fold=0, dr=dr, dz=(dr if mode == "TM" else d / nz))
    g = O.Geometry(s)
    st = np.zeros((O.N_STATE, nr, 1, nz), complex)
    if mode == "TM":
        k = sp.jn_zeros(1, 1)[0] / a
        prof = sp.jv(1, k * g.r_n[:nr])
        prof[0] = 0
        st[2] = prof[:, None, None] * np.ones((1, 1, nz))
        w2, comp, site = k * k, 2, (nr // 3, 0, 0)
    else:
        k = sp.jnp_zeros(1, 1)[0] / a
        kz = 2 / s.dz * math.sin(math.pi * s.dz / (2 * d))
        sz = np.sin(math.pi * s.dz * np.arange(nz) / d)[None, None, :]
        Rh = sp.jv(1, k * g.r_h)
        dR = np.zeros(nr)
        dR[1:] = (Rh[1:] - Rh[:-1]) / dr
        st[0] = (1j / g.r_h * Rh)[:, None, None] * sz
        st[1] = (-dR)[:, None, None] * sz
        w2, comp, site = k * k + kz * kz, 1, (nr // 3, 0, nz // 2)
    eps = [np.ones((nr, 1, nz))] * 3
    sig = np.empty(n_steps, complex)
    for n in range(n_steps):
        _, _, st = O.run(s, g, eps, n_steps=1, pml=O.no_pml(s), state=st)
        sig[n] = st[comp][site]
    A = np.stack([sig[1:-1], np.ones(n_steps - 2)], axis=1)
    c = np.linalg.lstsq(A, sig[2:] + sig[:-2], rcond=None)[0][0].real
    return ((2 - c) / g.dt ** 2 - w2) / w2


def test_axis_zone_cylinder_resonances():
    e1, e2 = _cylinder_error(0.05, "TM"), _cylinder_error(0.025, "TM")
    assert abs(e1) < 3e-3 and 3.5 < e1 / e2 < 4.5, (e1, e2)
    assert abs(_cylinder_error(0.05, "TE")) < 1e-4


def test_axis_zone_energy_conserved():
    """Axis zone with PEC walls: leap-frog energy with the r-weighted volumes
    (the on-axis sites weigh zero) is conserved."""
    s = _pec_spec(r_lo=0.0, n_r=12, n_phi=1, n_z=10, n_fold=0, dr=0.1, dz=0.1)
    g = O.Geometry(s)
    rng = np.random.default_rng(1)
    sh = (6, s.n_r, 1, s.n_z)
    st = np.zeros((O.N_STATE, s.n_r, 1, s.n_z), complex)
    st[:6] = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    st = _enforce_pec(st)
    eps = tuple(1.0 + rng.random((s.n_r, 1, s.n_z)) for _ in range(3))
    VE, VH = _volumes(s, g)
    W = []
    for n in range(300):
        E, Hm = st[:3].copy(), st[3:6].copy()
        _, _, st = O.run(s, g, eps, n_steps=1, pml=O.no_pml(s), state=st)
        W.append(sum((eps[c] * VE[c] * abs(E[c]) ** 2).sum() for c in range(3))
                 + sum((VH[c] * np.real(np.conj(Hm[c]) * st[3 + c])).sum() for c in range(3)))
    W = np.array(W)
    assert np.abs(W / W[0] - 1).max() < 1e-12


def test_axis_zone_adjoint_matches_central_differences():
    """The hybrid adjoint in the axis zone (continuous axisymmetry, r_lo = 0):
    directional derivative along the gradient and a few pixels."""
    spec = zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_steps=2400, courant=0.9,
                     filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1), pulse_sigma=0.4,
                     pulse_t0=1.6, eps_hi=2.1)
    assert _directional_error(spec) < 1e-3
    errs = _fd_errors(spec, [(0, 0), (3, 0), (9, 0), (15, 0)])
    assert errs.max() < 2e-3, errs


def test_focal_plane_on_axis_equals_on_axis_transform():
    """The brute-force focal-plane field at the axis equals the on-axis
    transform: (E_x, E_y) = c+ (1, i) + c- (1, -i), c+ = S(+w), c- = conj(S(-w))."""
    spec = zone_tiny(n_steps=500, wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6, focal=8.0)
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 3, mode="binary")
    f = O.forward(spec, rho)
    g = f["geom"]
    ex, ey = O.focal_plane_bruteforce(spec, g, f["mon"], [(0.0, 0.0)])
    nl = g.n_lambda
    cp, cm = f["S"][:nl], np.conj(f["S"][nl:])
    assert np.allclose(ex[:, 0], cp + cm, rtol=1e-10, atol=1e-14)
    assert np.allclose(ey[:, 0], 1j * (cp - cm), rtol=1e-10, atol=1e-14)


def test_field_off_the_focal_plane_matches_the_annulus_closed_form():
    """The brute-force field at (0, 0, h) above the focal plane of a uniform
    m = +1 annulus field (as in T8, E_r part) equals Re(U0) times the RS-I
    closed form at distance zf + h, converging at second order in dr."""
    hs = (-3.0, -1.0, 0.0, 2.5)
    errs = []
    for dr in (0.05, 0.025):
        s = zone_tiny(r_lo=5.0, n_r=int(round(4 / dr)), dr=dr, pml_r_in=int(round(0.5 / dr)),
                      pml_r_out=int(round(0.5 / dr)), n_phi=12, n_fold=40, wavelengths=(0.9,), focal=7.0)
        g = O.Geometry(s)
        U0 = 0.7 - 0.3j
        mon = np.zeros((g.n_freq, 2, s.n_r, s.n_phi), complex)
        mon[:, 0] = U0 * np.exp(1j * g.phi_n)[None, None, :]
        _, _, zf = O.focal_weights(s, g)
        ex, ey = O.focal_plane_bruteforce(s, g, mon, [(0.0, 0.0, h) for h in hs])
        k = 2 * math.pi / 0.9
        want = np.array([U0.real * _annulus_closed_form(zf + h, g.r0, g.r1, k) for h in hs])
        wy = np.array([-U0.imag * _annulus_closed_form(zf + h, g.r0, g.r1, k) for h in hs])
        errs.append(max(np.max(np.abs(ex[0] - want) / np.abs(want)), np.max(np.abs(ey[0] - wy) / np.abs(wy))))
    assert errs[0] < 1e-2, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs

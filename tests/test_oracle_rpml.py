"""Pins of the oracle's stretched-coordinate r-PML (section "Differentiable
FDTD in cylindrical coordinates": the stretched radius r' = r + i zeta_r / w
appears explicitly in the equations, and the r-PML must be regularised).

* the split of (1/r) d/dr (r .) into derivative + metric parts is the same
  operator as the unsplit one when nothing is stretched (one step, exact);
* the metric recursion realises 1/r~ with r~ = r + Omega / (alpha - i w),
  Omega recomputed here by quadrature of sigma;
* the stretched form reflects far less than the plain CPML (measured against
  a radially larger domain whose own walls are out of reach in the window);
* the regularisation: r~ in the inner (concave) slab makes the wedge's
  non-propagating azimuthal orders grow, the regularised form stays bounded.
"""
import math

import numpy as np

import oracle as O
from zda_inputs import ZoneSpec


def _ring_spec(r_face, n_r, n_fold, n_phi=4, n_z=64, pml_in=8, pml_out=8):
    dr = 0.05
    return ZoneSpec(r_lo=r_face - pml_in * dr, n_r=n_r, n_phi=n_phi, n_z=n_z, n_fold=n_fold, dr=dr, dz=dr,
                    pml_r_in=pml_in, pml_r_out=pml_out, pml_z=8, layer_k0=(0,), layer_eps=(1.0,),
                    source_k=n_z // 2, monitor_k=n_z // 2 + 8, n_steps=10, courant=0.5)


def _ring_source(spec, geom, i_src):
    pat = O.plane_wave_pattern(spec, geom)
    mask = np.zeros(spec.n_r)
    mask[i_src] = 1.0
    return pat * mask[None, None, :, None]


def _run_ring(spec, geom, pml, i_src, n_steps, twiddle=None, state=None, n0=0):
    eps = [np.ones((spec.n_r, spec.n_phi, spec.n_z)) for _ in range(3)]
    t = (np.arange(n0, n0 + n_steps) + 0.5) * geom.dt
    stime = O.pulse(spec, t).astype(np.complex128)[:, None]
    if state is None:
        state = np.zeros((O.N_STATE, spec.n_r, spec.n_phi, spec.n_z), complex)
    return O.run(spec, geom, eps, n_steps=n_steps, pml=pml, src_pat=_ring_source(spec, geom, i_src),
                 src_time=stime, src_k=spec.source_k, twiddle=twiddle, design=False, state=state)


def test_split_form_is_the_unsplit_operator():
    """rpml_metric = 1 with the PML switched on but nothing stretched
    (b != 0 selects the split form, c = bm = cm = 0) must reproduce one
    rpml_metric = 0 step from a random state to rounding: the split
    (F(i+1) - F(i)) / dr + (F(i+1) + F(i)) / (2 r) of the z-curls is an
    identity of (r_{i+1} F(i+1) - r_i F(i)) / (r dr)."""
    spec = _ring_spec(3.0, 24, 24, n_z=24)
    g = O.Geometry(spec)
    rng = np.random.default_rng(3)
    st = rng.standard_normal((O.N_STATE, spec.n_r, spec.n_phi, spec.n_z)) \
        + 1j * rng.standard_normal((O.N_STATE, spec.n_r, spec.n_phi, spec.n_z))
    st[6:] = 0.0
    base = O.no_pml(spec)
    base["br_n"] = np.full(spec.n_r + 1, 0.5)
    base["br_h"] = np.full(spec.n_r, 0.5)
    eps = [np.ones((spec.n_r, spec.n_phi, spec.n_z)) for _ in range(3)]
    _, _, a = O.run(spec, g, eps, n_steps=1, pml=base, state=st.copy(), design=False)
    split = dict(base, metric=1, bm_n=np.zeros(spec.n_r + 1), cm_n=np.zeros(spec.n_r + 1),
                 bm_h=np.zeros(spec.n_r), cm_h=np.zeros(spec.n_r))
    _, _, b = O.run(spec, g, eps, n_steps=1, pml=split, state=st.copy(), design=False)
    scale = np.abs(a[:6]).max()
    assert np.abs(a[:6] - b[:6]).max() < 1e-12 * scale
    # the step moves the fields, so the comparison is not vacuous
    assert np.abs(a[:6] - st[:6]).max() > 1e-3 * scale


def test_metric_recursion_is_one_over_stretched_radius():
    """Steady-state response of psi <- bm psi + cm X at the outer slab's
    deepest half node: (X + psi) / X = r / r~(w) with
    r~ = r + Omega / (alpha_max - i w), Omega = int sigma dr' by quadrature of
    sigma = sigma_max x^3 (sigma_max = -4 ln(1e-8) / (2 d))."""
    spec = _ring_spec(10.0, 56, 96)
    g = O.Geometry(spec)
    pml = O.cpml_coefficients(spec, g, metric=True)
    i = spec.n_r - 1                                     # deepest half node of the outer slab
    d = spec.pml_r_out * spec.dr
    face = spec.r_lo + (spec.n_r - spec.pml_r_out) * spec.dr
    r = g.r_h[i]
    xs = np.linspace(face, r, 4001)
    sig = (-4.0 * math.log(1e-8) / (2.0 * d)) * ((xs - face) / d) ** 3
    omega_int = np.trapezoid(sig, xs)
    alpha = 0.05 * 2.0 * math.pi * spec.pulse_f0
    for w in (2.0 * math.pi, -2.0 * math.pi, 0.5 * math.pi):
        n = np.arange(20000)
        X = np.exp(-1j * w * n * g.dt)
        psi = 0.0
        for x in X[:-1]:
            psi = pml["bm_h"][i] * psi + pml["cm_h"][i] * x
        psi = pml["bm_h"][i] * psi + pml["cm_h"][i] * X[-1]
        got = (X[-1] + psi) / X[-1]
        want = r / (r + omega_int / (alpha - 1j * w))
        # recursive convolution vs the continuous factor: relative error
        # O(w dt) of the metric effect 1 - r / r~ (a sign error in Omega
        # would miss it by twice its size)
        assert abs(got - want) < 0.1 * abs(1 - want), (w, got, want)
        assert abs(1 - want) > 0.05
    # the inner slab keeps the real radius (the regularisation)
    inner = g.r_h < spec.r_lo + spec.pml_r_in * spec.dr
    assert np.all(pml["bm_h"][inner] == 0) and np.all(pml["cm_h"][inner] == 0)


def _reflection(pml_kw, r_face=10.0, n_fold=96, W=40, L_in=100, L_out=200, T=10.0):
    """Relative difference of the +w monitor DFT over the interior between a
    zone and the same zone extended radially by L_in / L_out cells (whose own
    walls cannot be reached within T): the r-PML's reflection."""
    dr = 0.05
    test = _ring_spec(r_face, W + 16, n_fold)
    ref = _ring_spec(r_face - L_in * dr, W + 16 + L_in + L_out, n_fold)
    gt, gr = O.Geometry(test), O.Geometry(ref)
    gt.dt = gr.dt = min(gt.dt, gr.dt)
    n = int(round(T / gt.dt))
    nl = gt.n_lambda
    mr, _, _ = _run_ring(ref, gr, O.cpml_coefficients(ref, gr), 8 + W // 2 + L_in, n, O.twiddles(gr, n))
    mt, _, _ = _run_ring(test, gt, O.cpml_coefficients(test, gt, **pml_kw), 8 + W // 2, n, O.twiddles(gt, n))
    a = mt[:nl, :, 8:8 + W]
    b = mr[:nl, :, 8 + L_in:8 + L_in + W]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_stretched_r_pml_reflects_less_than_plain_cpml():
    plain = _reflection({})
    stretched = _reflection(dict(metric=True))
    assert plain > 1e-3                  # 1.9e-3 at r = 10 lambda
    assert stretched < 1.5e-4            # 5.3e-5: the 8-cell grading's own floor
    assert stretched < plain / 10


def _energy(spec, pml_kw, T, nseg=4):
    g = O.Geometry(spec)
    pml = O.cpml_coefficients(spec, g, **pml_kw)
    n = int(round(T / g.dt)) // nseg
    st, out = None, []
    for s in range(nseg):
        _, _, st = _run_ring(spec, g, pml, spec.n_r // 2, n, state=st, n0=s * n)
        out.append(float(np.sum(np.abs(st[:6]) ** 2)))
    return out


def test_regularisation_inner_slab_keeps_the_real_radius():
    """Wedge zone at r = 5 lambda (orders 1 + 48 k present): r~ in the inner
    slab grows without bound; the regularised form stays bounded, and so does
    the inner r~ with continuous axisymmetry (order 1 alone)."""
    spec = _ring_spec(5.0, 56, 48)
    grow = _energy(spec, dict(metric=True, metric_inner=True), 80.0)
    assert grow[-1] > 1e3 * grow[0]
    keep = _energy(spec, dict(metric=True), 80.0)
    assert keep[-1] < 1.01 * keep[1]
    bor = ZoneSpec(r_lo=4.6, n_r=56, n_phi=1, n_z=64, n_fold=0, dr=0.05, dz=0.05, pml_r_in=8, pml_r_out=8,
                   pml_z=8, source_k=32, monitor_k=40, n_steps=10, courant=0.5)
    axis = _energy(bor, dict(metric=True, metric_inner=True), 80.0)
    assert axis[-1] < 1.01 * axis[1]


def test_adjoint_gradient_with_the_stretched_form_matches_central_differences():
    """The adjoint run uses the same stepper with the stretched r-PML: its
    gradient must still match central differences of the form-1 objective
    (low-contrast layer so that the fields decay, as in the default form's
    FD pin).  The design pixels never sit in the r-PML, so only the decay
    and the PML's non-transposed discretisation limit the agreement."""
    from zda_inputs import smoothed_rho, zone_tiny
    spec = zone_tiny(n_steps=3200, courant=0.9, filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1),
                     pulse_sigma=0.4, pulse_t0=1.6, eps_hi=2.1)
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 7, mode="minmax")
    _, grad, _, _ = O.gradient(spec, rho, pml_form=1)
    _, grad0, _, _ = O.gradient(spec, rho)
    assert np.linalg.norm(grad - grad0) > 1e-4 * np.linalg.norm(grad0)    # the forms differ
    h = 1e-4
    errs = []
    for i, j in [(0, 0), (3, 2), (7, 4), (12, 7), (15, 3)]:
        rp, rm = rho.copy(), rho.copy()
        rp[i, j] += h
        rm[i, j] -= h
        fd = (O.forward(spec, rp, pml_form=1)["I"] - O.forward(spec, rm, pml_form=1)["I"]) / (2 * h)
        errs.append(abs(grad[i, j] - fd))
    assert max(errs) / np.abs(grad).max() < 2e-3, errs
    v = grad / np.linalg.norm(grad)
    hd = 1e-3
    fd = (O.forward(spec, rho + hd * v, pml_form=1)["I"] - O.forward(spec, rho - hd * v, pml_form=1)["I"]) / (2 * hd)
    assert abs(fd / np.linalg.norm(grad) - 1) < 1e-3

"""Max-min over wavelengths in epigraph form (Eqs. 7-8) with the CCSA
optimiser, on CPU: problems with closed-form optima, a linear program
against scipy's, the per-wavelength adjoint gradient against finite
differences, and an epigraph run on the oracle's zone."""
import numpy as np
import pytest

import oracle as O
from paper_2501_07979_gb300.topopt import (CCSA, Epigraph, wavelength_intensities,
                                             wavelength_sensitivity)
from zda_inputs import smoothed_rho, zone_tiny


def test_max_min_of_two_concave_quadratics_reaches_the_midpoint():
    """max_p min(1 - |p - a|^2, 1 - |p - b|^2): the optimum is the midpoint of a
    and b with value 1 - |a - b|^2 / 4 (both constraints active)."""
    a = np.array([0.2, 0.3])
    b = np.array([0.8, 0.7])

    def objectives(p, need_grad=True):
        I = np.array([1 - np.sum((p - a) ** 2), 1 - np.sum((p - b) ** 2)])
        if not need_grad:
            return I
        return I, [-2 * (p - a), -2 * (p - b)]

    ep = Epigraph(objectives, np.array([0.1, 0.9]), q_max=2.0)
    ep.run(40)
    assert np.allclose(ep.rho, (a + b) / 2, atol=2e-3)
    assert abs(ep.q - (1 - np.sum((a - b) ** 2) / 4)) < 2e-3
    mins = [h["min_I"] for h in ep.history]
    assert mins[-1] >= max(mins) - 1e-6


def test_ccsa_solves_a_linear_program_like_scipy():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    n, m = 6, 3
    c = rng.standard_normal(n)
    A = rng.uniform(0, 1, (m, n))
    bvec = A.sum(axis=1) * 0.4
    ref = scipy_opt.linprog(c, A_ub=A, b_ub=bvec, bounds=[(0, 1)] * n, method="highs")

    def values(x):
        return np.concatenate([[c @ x], A @ x - bvec])

    opt = CCSA(np.zeros(n), np.ones(n), m)
    x = np.full(n, 0.1)                                  # feasible start
    for _ in range(200):
        x, _, _ = opt.step(x, values(x), np.vstack([c, A]), values)
    assert np.all(A @ x - bvec <= 1e-6)
    assert abs(c @ x - ref.fun) < 1e-4 * max(1.0, abs(ref.fun))


def test_every_accepted_ccsa_step_is_conservative():
    """The accepted point satisfies f_i <= g_i for each approximation (the
    property that makes CCSA globally convergent)."""
    f0 = lambda x: float(np.sum(np.cos(3 * x)))                 # noqa: E731
    f1 = lambda x: float(np.sum(x ** 2)) - 1.0                  # noqa: E731
    x = np.full(4, 0.3)
    opt = CCSA(np.full(4, -1.0), np.full(4, 1.0), 1)
    values = lambda z: np.array([f0(z), f1(z)])                # noqa: E731
    prev = f0(x)
    for _ in range(15):
        g = np.vstack([-3 * np.sin(3 * x), 2 * x])
        xn, fn, _ = opt.step(x, values(x), g, values)
        assert fn[1] <= 1e-6                                      # stays feasible (dual-solve tolerance)
        assert fn[0] <= prev + 1e-6                               # objective never increases (up to the dual solve)
        prev, x = fn[0], xn


SPEC = zone_tiny(n_steps=700, filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1), eps_hi=2.1,
                 pulse_sigma=0.4, pulse_t0=1.6)


def _oracle_objectives(spec):
    def objectives(rho, need_grad=True):
        rho = np.asarray(rho, dtype=np.float64)
        fwd = O.forward(spec, rho)
        I = wavelength_intensities(fwd["S"], len(spec.wavelengths))
        if not need_grad:
            return I
        fwd["rho"] = rho
        geom = fwd["geom"]
        rbar = O.conic_filter(spec, geom, rho)
        grads = []
        for l in range(len(spec.wavelengths)):
            adj = O.adjoint(spec, fwd, wavelength_sensitivity(fwd["S"], len(spec.wavelengths), l))
            grads.append(O.conic_filter_T(spec, geom, adj["grad_rho_tilde"] * O.project_grad(spec, rbar)))
        return I, grads
    return objectives


def test_per_wavelength_adjoint_gradient_matches_finite_differences():
    obj = _oracle_objectives(SPEC)
    rho = smoothed_rho(SPEC.n_r_design, SPEC.n_phi, 21, mode="minmax")
    I, grads = obj(rho)
    d = np.random.default_rng(4).standard_normal(rho.shape)
    h = 1e-4
    Ip = obj(rho + h * d, False)
    Im = obj(rho - h * d, False)
    for l in range(2):
        fd = (Ip[l] - Im[l]) / (2 * h)
        assert abs(fd - np.sum(grads[l] * d)) < 1e-3 * max(abs(fd), 1e-12), (l, fd, np.sum(grads[l] * d))
    assert np.isclose(np.sum(I), O.intensity(O.forward(SPEC, rho)["S"]), rtol=1e-12)


def test_epigraph_raises_the_weakest_wavelength_on_the_oracle_zone():
    obj = _oracle_objectives(SPEC)
    rho0 = np.full((SPEC.n_r_design, SPEC.n_phi), 0.5)
    ep = Epigraph(obj, rho0)
    I0 = obj(rho0, False)
    ep.run(4)
    assert ep.history[-1]["min_I"] > 1.5 * float(np.min(I0))
    assert all(h["q"] <= h["min_I"] * (1 + 1e-6) + 1e-12 for h in ep.history)   # feasible epigraph variable

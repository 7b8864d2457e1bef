"""The oracle's focal-spot evaluation pinned on CPU: encircled power of
closed-form spots, FWHM of a Gaussian, and the evaluation (PSF, FWHM,
focusing efficiencies, Strehl ratio of Eq. 9) of an ideal Airy spot.  The
library's evaluation (zda_lens_evaluate) is held to this oracle on the GPU."""
import math

import numpy as np

import oracle as O


def test_encircled_power_of_a_uniform_disk_and_a_gaussian():
    r = np.linspace(0, 2, 2001)
    P = O.encircled_power(r, np.where(r <= 1.0, 1.0, 0.0))
    assert abs(P[-1] - math.pi) < 5e-3                       # pi * 1^2 (edge sampled at dr = 1e-3)
    s = 0.3
    Pg = O.encircled_power(r, np.exp(-r ** 2 / (2 * s * s)))
    exact = 2 * math.pi * s * s * (1 - np.exp(-r ** 2 / (2 * s * s)))
    assert np.max(np.abs(Pg - exact)) < 1e-6


def test_fwhm_of_a_gaussian():
    xs = np.linspace(0, 2, 2001)                  # profile from the peak outwards
    s = 0.25
    assert abs(O.fwhm(xs, np.exp(-xs ** 2 / (2 * s * s))) - 2 * math.sqrt(2 * math.log(2)) * s) < 1e-5


class _AiryLens:
    """Stand-in for a lens after its forward run: the paraxial focal field of
    a uniformly lit aperture of radius a at focal distance F carrying power P
    per wavelength, I(rho) = I0 (2 J1(v) / v)^2, v = 2 pi a rho / (lambda F),
    I0 = P pi a^2 / (lambda^2 F^2)."""

    def __init__(self, lams, a, F, P):
        import types
        self.zones = [types.SimpleNamespace(spec=types.SimpleNamespace(wavelengths=tuple(lams)))]
        self.lams, self.a, self.F, self.P = np.asarray(lams), a, F, np.asarray(P)

    def intensity(self, l, rho):
        from scipy.special import j1
        lam = self.lams[l]
        v = 2 * math.pi * self.a * np.asarray(rho) / (lam * self.F)
        amp = np.where(v == 0, 1.0, 2 * j1(np.where(v == 0, 1.0, v)) / np.where(v == 0, 1.0, v))
        return self.P[l] * math.pi * self.a ** 2 / (lam * self.F) ** 2 * amp ** 2

    def focal_plane(self, pts):
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
        rho = np.hypot(pts[:, 0], pts[:, 1])
        ex = np.array([np.sqrt(2 * self.intensity(l, rho)) for l in range(len(self.lams))], dtype=complex)
        return ex, np.zeros_like(ex), self.P.copy()


def test_evaluate_spot_on_an_airy_spot():
    """FWHM = 1.029 lambda F / (2 a); the power within 3 FWHM is the Airy
    encircled energy 1 - J0(v)^2 - J1(v)^2; transmittance = P / (I_inc A);
    Strehl = 1 for the ideal spot (Eq. 9: I lambda^2 F^2 / (P A))."""
    import pytest
    special = pytest.importorskip("scipy.special")
    lams, a, F = (0.9, 1.0), 100.0, 200.0
    P = (3.0, 2.0)
    lens = _AiryLens(lams, a, F, P)
    inc = np.array([1.0 / (math.pi * a * a), 0.5 / (math.pi * a * a)])       # incident powers 1 and 0.5
    res, xs, I = O.evaluate_spot(lens.focal_plane, lams, a, F, inc, n_line=4 * 96, n_rad=96, n_ang=4)
    for l, r in enumerate(res):
        lam = lams[l]
        assert abs(r["fwhm"] - 1.0290 * lam * F / (2 * a)) < 2e-3 * r["fwhm"]
        v = 2 * math.pi * a * 3 * r["fwhm"] / (lam * F)
        ee = 1 - special.j0(v) ** 2 - special.j1(v) ** 2
        assert abs(r["relative_efficiency"] - ee) < 2e-3, (r["relative_efficiency"], ee)
        assert abs(r["transmittance"] - P[l] / (inc[l] * math.pi * a * a)) < 1e-12
        assert abs(r["strehl"] - 1.0) < 1e-9


def test_fwhm_edge_cases_and_disc_samples():
    """A profile that never falls below half has no FWHM (NaN, as the
    library returns); the crossing is interpolated between the samples that
    bracket it; the disc samples sit at (k + 1/2) 3 w / n_rad, n_ang angles."""
    xs = np.linspace(0, 1, 11)
    assert math.isnan(O.fwhm(xs, np.ones(11)))
    I = np.array([1.0, 0.8, 0.4, 0.1])
    # half = 0.5 between x = 1 (0.8) and x = 2 (0.4): 1 + 0.3 / 0.4 = 1.75
    assert abs(O.fwhm(np.arange(4.0), I) - 3.5) < 1e-15
    rr, pts = O.disc_points(0.2, 4, 3)
    assert np.allclose(rr, (np.arange(4) + 0.5) * 0.6 / 4)
    assert pts.shape == (12, 2)
    assert np.allclose(np.hypot(pts[:, 0], pts[:, 1]).reshape(4, 3), rr[:, None])

"""Focal-spot evaluation of a lens ("Centimeter-scale metalens at long-wave
infrared": PSF and FWHM, absolute focusing efficiency = power within 3 FWHM
of the focal spot / incident power, relative efficiency = the same /
transmitted power; Eq. 9: Strehl ratio SR = I lambda^2 F^2 / (P_trans A))."""
import math

import numpy as np


def incident_intensity(spec, device=0):
    """Plane-wave intensity (n/2)|E|^2 of the source in the substrate, per
    wavelength, from a reference run of the zone with every layer and the
    design layer made of the substrate (no interface, no lens): the m = +1
    run's phi-mean of u_r at the monitor is half the plane-wave amplitude."""
    import torch
    from .zone import Zone
    eps_sub = float(spec.layer_eps[0])
    ref = spec.replace(layer_eps=tuple(eps_sub for _ in spec.layer_eps), eps_lo=eps_sub, eps_hi=eps_sub,
                       filter_radius=0.0, beta=0.0)
    z = Zone(ref, device=device)
    z.forward(torch.zeros((z.n_r_design, ref.n_phi), dtype=torch.float32, device=z.device))
    mon = z.monitor_dft().cpu().numpy()
    nl = z.n_freq // 2
    i0, i1 = ref.pml_r_in, ref.n_r - ref.pml_r_out
    if ref.n_fold == 0:
        ph = np.ones(ref.n_phi)
    else:
        dphi = 2 * math.pi / ref.n_fold / ref.n_phi
        ph = np.exp(-1j * dphi * np.arange(ref.n_phi))
    out = np.zeros(nl)
    for l in range(nl):
        u = (mon[l, 0, i0:i1] * ph[None, :]).mean()
        out[l] = 0.5 * math.sqrt(eps_sub) * abs(2 * u) ** 2
    return out


def intensity(ex, ey, n_top=1.0):
    return 0.5 * n_top * (np.abs(ex) ** 2 + np.abs(ey) ** 2)


def fwhm(xs, I):
    """Full width at half maximum of a centred profile I(xs), xs >= 0 from the
    peak at xs[0]; linear interpolation of the half-maximum crossing."""
    I = np.asarray(I, dtype=np.float64)
    half = 0.5 * I[0]
    below = np.nonzero(I < half)[0]
    if below.size == 0:
        return float("nan")
    j = below[0]
    x0, x1, y0, y1 = xs[j - 1], xs[j], I[j - 1], I[j]
    return 2.0 * (x0 + (half - y0) * (x1 - x0) / (y1 - y0))


def evaluate_lens(lens, lens_radius, focal, incident, n_top=1.0, n_rad=48, n_ang=8, n_phi_samples=128):
    """PSF line, FWHM, focal intensity, focusing efficiency (absolute and
    relative) and Strehl ratio per wavelength after lens.forward(...)."""
    lam = np.asarray(lens.zones[0].spec.wavelengths, dtype=np.float64)
    nl = lam.size
    # PSF along x out to 4 lambda
    xs = np.linspace(0.0, 4.0 * lam.max(), 4 * n_rad)
    ex, ey, p_trans = lens.focal_plane(np.stack([xs, np.zeros_like(xs)], 1), n_phi_samples)
    I_line = intensity(ex, ey, n_top)
    res = []
    for l in range(nl):
        w = fwhm(xs, I_line[l])
        rmax = 3.0 * w
        rr = (np.arange(n_rad) + 0.5) * rmax / n_rad
        aa = 2 * math.pi * np.arange(n_ang) / n_ang
        pts = np.array([(r * math.cos(a), r * math.sin(a)) for r in rr for a in aa])
        fx, fy, _ = lens.focal_plane(pts, n_phi_samples)
        Id = intensity(fx[l], fy[l], n_top).reshape(n_rad, n_ang)
        p_disc = float(np.sum(Id.mean(axis=1) * 2 * math.pi * rr) * (rmax / n_rad))
        area = math.pi * lens_radius ** 2
        p_inc = incident[l] * area
        I0 = I_line[l, 0]
        res.append({"lambda": float(lam[l]), "fwhm": w, "focal_intensity": float(I0),
                    "focusing_efficiency": p_disc / p_inc, "relative_efficiency": p_disc / p_trans[l],
                    "transmittance": p_trans[l] / p_inc,
                    "strehl": float(I0 * lam[l] ** 2 * focal ** 2 / (p_trans[l] * area)),
                    "order_bound": lens.order_bound(pts)})
    return res, xs, I_line


def xz_map(lens, xs, hs, n_top=1.0, n_phi_samples=128):
    """Intensity (n/2)(|E_x|^2 + |E_y|^2) on the xz plane through the axis:
    [n_lambda][len(hs)][len(xs)], h = height above the focal plane."""
    X, Hh = np.meshgrid(np.asarray(xs, dtype=np.float64), np.asarray(hs, dtype=np.float64))
    pts = np.stack([X.ravel(), np.zeros(X.size), Hh.ravel()], axis=1)
    ex, ey = lens.field_points(pts, n_phi_samples=n_phi_samples)
    return intensity(ex, ey, n_top).reshape(ex.shape[0], len(hs), len(xs))


def encircled_power(radii, I_of_r):
    """Encircled power P(rho) = int_0^rho I(r) 2 pi r dr of a radially
    symmetric focal spot sampled at increasing radii (trapezoid rule)."""
    r = np.asarray(radii, dtype=np.float64)
    f = np.asarray(I_of_r, dtype=np.float64) * 2 * math.pi * r
    out = np.zeros_like(r)
    out[1:] = np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(r))
    return out

"""Focal-spot evaluation of a lens ("Centimeter-scale metalens at long-wave
infrared": PSF and FWHM, absolute focusing efficiency = power within 3 FWHM
of the focal spot / incident power, relative efficiency = the same /
transmitted power; Eq. 9: Strehl ratio SR = I lambda^2 F^2 / (P_trans A)).
Every quantity is computed by the library (zda_lens_evaluate,
zda_zone_incident_intensity, zda_field_intensity, zda_encircled_power in
include/zda.h); this module marshals arguments and results."""
import ctypes
import math
import warnings

import numpy as np

from . import _lib
from ._lib import check
from .lens import ORDER_BOUND_TOL


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def incident_intensity(spec, device=0):
    """Plane-wave intensity (n/2)|E|^2 of the source in the substrate, per
    wavelength, from a reference run of the zone with every layer and the
    design layer made of the substrate (no interface, no lens)
    (zda_zone_incident_intensity)."""
    import torch
    from .zone import Zone
    eps_sub = float(spec.layer_eps[0])
    ref = spec.replace(layer_eps=tuple(eps_sub for _ in spec.layer_eps), eps_lo=eps_sub, eps_hi=eps_sub,
                       filter_radius=0.0, beta=0.0)
    z = Zone(ref, device=device)
    z.forward(torch.zeros((z.n_r_design, ref.n_phi), dtype=torch.float32, device=z.device))
    out = torch.empty(z.n_freq // 2, dtype=torch.float64, device=z.device)
    check(_lib.lib().zda_zone_incident_intensity(z.handle, _dptr(out), _stream()))
    return out.cpu().numpy()


def evaluate_lens(lens, lens_radius, focal, incident, n_top=1.0, n_rad=48, n_ang=8, n_phi_samples=128):
    """PSF line, FWHM, focal intensity, focusing efficiency (absolute and
    relative), transmittance and Strehl ratio per wavelength after
    lens.forward(...) (zda_lens_evaluate: a PSF line of 4 n_rad samples over
    [0, 4 lambda_max], discs of n_rad x n_ang samples within 3 FWHM).
    Returns (list of dicts, xs, I_line)."""
    import torch
    lam = np.asarray(lens.zones[0].spec.wavelengths, dtype=np.float64)
    nl = lam.size
    n_line, x_max = 4 * n_rad, 4.0 * float(lam.max())
    inc = np.ascontiguousarray(np.asarray(incident, dtype=np.float64).ravel()[:nl])
    if inc.size != nl:
        raise ValueError("incident: one intensity per wavelength (%d) expected" % nl)
    dev = lens.zones[0].device
    line = torch.empty((nl, n_line), dtype=torch.float64, device=dev)
    nb = ctypes.c_size_t()
    check(_lib.lib().zda_lens_evaluate_scratch_bytes(lens.handle, int(n_line), int(n_rad), int(n_ang),
                                                     ctypes.byref(nb)))
    scratch = torch.empty(nb.value + 256, dtype=torch.uint8, device=dev)
    base = (scratch.data_ptr() + 255) // 256 * 256           # 256-byte aligned start
    out = (ctypes.c_double * (8 * nl))()
    check(_lib.lib().zda_lens_evaluate(lens.handle, float(lens_radius), float(focal),
                                       inc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(n_top), int(n_line),
                                       x_max, int(n_rad), int(n_ang), int(n_phi_samples), ctypes.c_void_p(base),
                                       nb.value, out, _dptr(line), _stream()))
    xs = np.linspace(0.0, x_max, n_line)              # the sample positions the library used
    o = np.array(out[:]).reshape(nl, 8)
    b_line = lens.order_bound(np.stack([xs, 0 * xs], 1))
    res = []
    for l in range(nl):
        w = o[l, 0]
        rr = (np.arange(n_rad) + 0.5) * 3.0 * w / n_rad
        aa = 2 * math.pi * np.arange(n_ang) / n_ang
        pts = np.array([(q * math.cos(a), q * math.sin(a)) for q in rr for a in aa]) if np.isfinite(w) else \
            np.zeros((1, 2))
        bound = lens.order_bound(pts)
        if max(bound, b_line) > ORDER_BOUND_TOL:
            warnings.warn("lens field: the neglected azimuthal orders may reach %.2g of the kept ones at these "
                          "points (zones with small n far off axis)" % max(bound, b_line), RuntimeWarning,
                          stacklevel=2)
        res.append({"lambda": float(lam[l]), "fwhm": float(w), "focal_intensity": float(o[l, 1]),
                    "focusing_efficiency": float(o[l, 2]), "relative_efficiency": float(o[l, 3]),
                    "transmittance": float(o[l, 4]), "strehl": float(o[l, 5]), "disc_power": float(o[l, 6]),
                    "transmitted_power": float(o[l, 7]), "order_bound": bound})
    return res, xs, line.cpu().numpy()


def xz_map(lens, xs, hs, n_top=1.0, n_phi_samples=128):
    """Intensity (n/2)(|E_x|^2 + |E_y|^2) on the xz plane through the axis:
    [n_lambda][len(hs)][len(xs)], h = height above the focal plane
    (zda_lens_field_points, zda_field_intensity)."""
    import torch
    X, Hh = np.meshgrid(np.asarray(xs, dtype=np.float64), np.asarray(hs, dtype=np.float64))
    pts_h = np.stack([X.ravel(), np.zeros(X.size), Hh.ravel()], axis=1)
    dev = lens.zones[0].device
    pts = torch.tensor(pts_h, dtype=torch.float64, device=dev)
    n = pts.shape[0]
    nl = lens.n_freq // 2
    field = torch.empty((2, nl, n, 2), dtype=torch.float64, device=dev)
    check(_lib.lib().zda_lens_field_points(lens.handle, _dptr(pts), int(n), int(n_phi_samples), _dptr(field),
                                           _stream()))
    lens._check_orders(pts_h)
    I = torch.empty((nl, n), dtype=torch.float64, device=dev)
    check(_lib.lib().zda_field_intensity(_dptr(field), int(nl), int(n), float(n_top), _dptr(I), _stream()))
    return I.cpu().numpy().reshape(nl, len(hs), len(xs))


def encircled_power(radii, I_of_r, device=0):
    """Encircled power P(rho) = int_0^rho I(r) 2 pi r dr of radially symmetric
    spots sampled at increasing radii (trapezoid rule; zda_encircled_power).
    I_of_r: one profile [n] or several [n_prof][n]."""
    import torch
    r = torch.tensor(np.asarray(radii, dtype=np.float64), device="cuda:%d" % device)
    I = np.asarray(I_of_r, dtype=np.float64)
    one = I.ndim == 1
    It = torch.tensor(I.reshape(-1, r.numel()), device=r.device)
    out = torch.empty_like(It)
    check(_lib.lib().zda_encircled_power(_dptr(r), _dptr(It), int(It.shape[0]), int(r.numel()), _dptr(out),
                                         _stream()))
    o = out.cpu().numpy()
    return o[0] if one else o

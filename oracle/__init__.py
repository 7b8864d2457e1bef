"""ORACLE -- test infrastructure, not the product.

A plain, slow, FP64 CPU statement of the zoned-discrete-axisymmetry (ZDA)
zone solve: geometry, density -> permittivity (conic filter, tanh projection,
Eq. 6), the cylindrical Yee time loop with CPML, plane-wave source and
running DFTs (C file `fdtd_ref.c`), the on-axis near-to-far focal transform,
the focal-intensity objective and the hybrid time/frequency adjoint gradient
(section "Differentiable FDTD in cylindrical coordinates"; "Results and
Discussion", Eqs. 6-8).  It shares no code with the CUDA library and never
imports it.  Only tests/, the smoke check and the benchmark's CPU-baseline
leg may use it.

Every function names the passage it follows.  Where the paper is silent the
reading used is stated in the docstring; the CUDA path implements the same
readings independently.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


# --------------------------------------------------------------------------
# C time loop: build + load
# --------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile fdtd_ref.c into oracle/_build/liborc.so with gcc (-fopenmp)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liborc.so")
    src = os.path.join(_HERE, "fdtd_ref.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fcx-limited-range", "-fopenmp", "-shared",
                               "-fPIC", "-std=c11", src, "-o", tmp, "-lm"])
        os.replace(tmp, so)
    return so


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int), ("nphi", ctypes.c_int), ("nz", ctypes.c_int),
        ("n_steps", ctypes.c_int),
        ("r_lo", ctypes.c_double), ("dr", ctypes.c_double), ("dz", ctypes.c_double),
        ("dphi", ctypes.c_double), ("dt", ctypes.c_double),
        ("bloch_re", ctypes.c_double), ("bloch_im", ctypes.c_double),
        ("eps_r", ctypes.c_void_p), ("eps_p", ctypes.c_void_p), ("eps_z", ctypes.c_void_p),
        ("br_n", ctypes.c_void_p), ("cr_n", ctypes.c_void_p),
        ("br_h", ctypes.c_void_p), ("cr_h", ctypes.c_void_p),
        ("bz_n", ctypes.c_void_p), ("cz_n", ctypes.c_void_p),
        ("bz_h", ctypes.c_void_p), ("cz_h", ctypes.c_void_p),
        ("src_k", ctypes.c_int), ("n_src", ctypes.c_int),
        ("src_pat", ctypes.c_void_p), ("src_time", ctypes.c_void_p),
        ("n_freq", ctypes.c_int), ("twiddle", ctypes.c_void_p),
        ("bor", ctypes.c_int), ("m", ctypes.c_int),
        ("mon_k", ctypes.c_int), ("mon_dft", ctypes.c_void_p),
        ("des_k0", ctypes.c_int), ("des_nk", ctypes.c_int), ("des_dft", ctypes.c_void_p),
        ("state", ctypes.c_void_p), ("nthreads", ctypes.c_int),
        ("rpml_metric", ctypes.c_int),
        ("bm_n", ctypes.c_void_p), ("cm_n", ctypes.c_void_p),
        ("bm_h", ctypes.c_void_p), ("cm_h", ctypes.c_void_p),
    ]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = ctypes.CDLL(build())
            _LIB.orc_run.argtypes = [ctypes.POINTER(_Problem)]
            _LIB.orc_run.restype = ctypes.c_int
        return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data


N_STATE = 18   # E_r, E_phi, E_z, H_r, H_phi, H_z, 8 CPML and 4 metric auxiliaries


# --------------------------------------------------------------------------
# a1: zone geometry
# --------------------------------------------------------------------------
class Geometry:
    """Zone geometry (section "Zoned discrete axisymmetry"; Eqs. 1-2).

    tau = 2 pi / n is the wedge's azimuthal period and dphi = tau / n_phi.
    The time step is courant * dt_cyl with
    dt_cyl = 1 / sqrt(1/dr^2 + 1/(r_min dphi)^2 + 1/dz^2), r_min = r_lo: the
    Courant-Friedrichs-Lewy bound of the section "Centimeter-scale metalens"
    with the smallest azimuthal spacing of the wedge."""

    def __init__(self, spec):
        self.spec = spec
        s = spec
        self.bor = s.n_fold == 0
        if self.bor:
            # continuous axisymmetry (the axis zone): one phi cell, d/dphi -> i m
            if s.n_phi != 1 or s.r_lo < 0:
                raise ValueError("continuous axisymmetry needs n_phi = 1 and r_lo >= 0")
        elif s.n_fold < 0 or s.r_lo <= 0:
            raise ValueError("annular wedge zones need n_fold > 0 and r_lo > 0")
        self.nr, self.nphi, self.nz = s.n_r, s.n_phi, s.n_z
        self.dr, self.dz = s.dr, s.dz
        self.tau = 2.0 * math.pi / (1 if self.bor else s.n_fold)
        self.dphi = self.tau / s.n_phi
        self.r_n = s.r_lo + s.dr * np.arange(s.n_r + 1)          # r_i
        self.r_h = s.r_lo + s.dr * (np.arange(s.n_r) + 0.5)       # r_{i+1/2}
        if self.bor:
            # the im/r terms act at r >= r_lo + dr/2 (no phi-difference): the
            # smallest radius plays the part of r dphi in the Courant bound
            r_min = s.r_lo if s.r_lo > 0 else 0.5 * s.dr
            self.dt = s.courant / math.sqrt(1.0 / s.dr ** 2 + (s.m / r_min) ** 2 + 1.0 / s.dz ** 2)
        else:
            r_min = s.r_lo
            self.dt = s.courant / math.sqrt(1.0 / s.dr ** 2 + 1.0 / (r_min * self.dphi) ** 2
                                            + 1.0 / s.dz ** 2)
        self.bloch = complex(math.cos(s.m * self.tau), math.sin(s.m * self.tau))
        self.i_d0 = s.pml_r_in
        self.i_d1 = s.n_r - s.pml_r_out
        self.r0 = s.r_lo + self.i_d0 * s.dr          # design / monitor annulus
        self.r1 = s.r_lo + self.i_d1 * s.dr
        if self.bor:                                              # u-form: no phase
            self.phi_n = np.zeros(1)
            self.phi_h = np.zeros(1)
        else:
            self.phi_n = self.dphi * np.arange(s.n_phi)           # phi_j
            self.phi_h = self.dphi * (np.arange(s.n_phi) + 0.5)   # phi_{j+1/2}
        lam = np.asarray(s.wavelengths, dtype=np.float64)
        w = 2.0 * math.pi / lam
        self.omega = np.concatenate([w, -w])        # signed frequency list, +w first
        self.n_lambda = lam.size
        self.n_freq = 2 * lam.size
        self.des_k0 = s.design_k0
        self.des_nk = s.design_k1 - s.design_k0 + 1

    def omega_tilde(self):
        """Discrete-time frequency (2/dt) sin(w dt / 2) of the leap-frog scheme."""
        return 2.0 * np.sin(self.omega * self.dt / 2.0) / self.dt


# --------------------------------------------------------------------------
# CPML profiles (stretched-coordinate PML in r and z)
# --------------------------------------------------------------------------
def cpml_coefficients(spec, geom, R0: float = 1e-8, grade: int = 3, metric: bool = False,
                      outer_stretch: bool = True, metric_inner: bool = False, margin: float = 2.0):
    """Convolutional PML coefficients b, c at r nodes, r half nodes, z nodes and
    z half nodes (section "Differentiable FDTD": stretched-coordinate PMLs in
    (r, z)).  Reading: kappa = 1, sigma(x) = sigma_max x^grade with
    sigma_max = -(grade+1) ln(R0) / (2 d), alpha(x) = alpha_max (1 - x) with
    alpha_max = 0.05 * 2 pi f0, x = depth / d in [0, 1];
    b = exp(-(sigma + alpha) dt), c = sigma / (sigma + alpha) (b - 1).

    metric=True: inside the r-PML the metric factors use the stretched
    radius (the same section: r' = r + i zeta_r / w appears in the equations
    themselves).  (1/r~) d/dr~ (r~ F) = (1/s_r) dF/dr + F / r~, so only the
    derivative part of (1/r) d/dr (r .) carries the CPML stretch, and the
    metric parts are divided by r~.  Outer slab: r~ = r + Omega(r) /
    (alpha_max - i w), Omega(r) = int sigma dr' from the slab's interior face,
    with the same constant alpha_max in s_r so that dr~/dr = s_r exactly;
    1/r~ = (1/r) / (1 + sigma_m / (alpha_max - i w)), sigma_m = Omega / r >= 0,
    is one more recursive convolution: bm = exp(-(sigma_m + alpha) dt),
    cm = sigma_m / (sigma_m + alpha) (bm - 1).  outer_stretch=False keeps
    r~ = r there too (bm = cm = 0).

    The regularisation (the same section warns that the r-PML must be
    regularised against divergence): the inner slab's metric keeps the real
    radius (bm = cm = 0).  There Omega < 0, so Im r~ < 0, and a field of
    azimuthal order M with M / r >> k (the wedge's non-propagating orders
    m + k n) gains at a rate ~ -sigma_m instead of decaying.
    metric_inner=True builds that unregularised inner slab anyway
    (alpha_s = max(alpha_max, margin max(-sigma_m)) in it keeps its own pole
    stable) so that a test can show the growth."""
    s = spec
    dt = geom.dt
    a_max = 0.05 * 2.0 * math.pi * s.pulse_f0

    def depth(pos, lo, hi, n_in, n_out, h):
        """(x in [0, 1], sign: -1 inner PML, +1 outer PML, 0 interior, d)."""
        pos = np.asarray(pos, dtype=np.float64)
        x = np.zeros_like(pos)
        sgn = np.zeros_like(pos)
        if n_in > 0:
            d = n_in * h
            inner = pos < lo + d
            x = np.where(inner, (lo + d - pos) / d, x)
            sgn = np.where(inner, -1.0, sgn)
        if n_out > 0:
            d = n_out * h
            outer = pos > hi - d
            x = np.where(outer, (pos - (hi - d)) / d, x)
            sgn = np.where(outer, 1.0, sgn)
        d = np.where(sgn < 0, max(n_in, 1) * h, max(n_out, 1) * h)
        return np.clip(x, 0.0, 1.0), sgn, d

    def recursion(sig, alp):
        b = np.exp(-(sig + alp) * dt)
        c = np.where(sig != 0, sig / np.where(sig != 0, sig + alp, 1.0) * (b - 1.0), 0.0)
        return np.where(sig != 0, b, 0.0), c

    def coeffs(pos, lo, hi, n_in, n_out, h):
        x, sgn, d = depth(pos, lo, hi, n_in, n_out, h)
        smax = -(grade + 1) * math.log(R0) / (2.0 * d)
        return recursion(smax * x ** grade, a_max * (1.0 - x))

    r_lo, r_hi = s.r_lo, s.r_lo + s.n_r * s.dr
    z_lo, z_hi = 0.0, s.n_z * s.dz
    br_n, cr_n = coeffs(geom.r_n, r_lo, r_hi, s.pml_r_in, s.pml_r_out, s.dr)
    br_h, cr_h = coeffs(geom.r_h, r_lo, r_hi, s.pml_r_in, s.pml_r_out, s.dr)
    zn = s.dz * np.arange(s.n_z + 1)
    zh = s.dz * (np.arange(s.n_z) + 0.5)
    bz_n, cz_n = coeffs(zn, z_lo, z_hi, s.pml_z, s.pml_z, s.dz)
    bz_h, cz_h = coeffs(zh, z_lo, z_hi, s.pml_z, s.pml_z, s.dz)
    out = dict(br_n=br_n, cr_n=cr_n, br_h=br_h, cr_h=cr_h,
               bz_n=bz_n, cz_n=cz_n, bz_h=bz_h, cz_h=cz_h)
    if not metric:
        return out

    def stretch(pos):
        x, sgn, d = depth(pos, r_lo, r_hi, s.pml_r_in, s.pml_r_out, s.dr)
        smax = -(grade + 1) * math.log(R0) / (2.0 * d)
        omega_int = sgn * smax * d * x ** (grade + 1) / (grade + 1)     # int sigma dr' from the face
        pos = np.asarray(pos, dtype=np.float64)
        sig_m = np.where(pos > 0, omega_int / np.where(pos > 0, pos, 1.0), 0.0)
        return smax * x ** grade, sig_m, sgn

    a_in = a_max
    parts = {}
    for key, pos in (("n", geom.r_n), ("h", geom.r_h)):
        parts[key] = stretch(pos)
        if metric_inner:
            a_in = max(a_in, margin * max(0.0, float(-parts[key][1].min())))
    for key, (sig, sig_m, sgn) in parts.items():
        stretched = ((sgn > 0) & outer_stretch) | ((sgn < 0) & metric_inner)
        alp = np.where(sgn < 0, a_in, a_max)
        b, c = recursion(np.where(stretched, sig, 0.0), alp)
        out["br_" + key] = np.where(stretched, b, out["br_" + key])
        out["cr_" + key] = np.where(stretched, c, out["cr_" + key])
        out["bm_" + key], out["cm_" + key] = recursion(np.where(stretched, sig_m, 0.0), alp)
    out["metric"] = 1
    out["alpha_s"] = (a_in, a_max)
    return out


def no_pml(spec):
    z = lambda n: np.zeros(n)
    return dict(br_n=z(spec.n_r + 1), cr_n=z(spec.n_r + 1), br_h=z(spec.n_r), cr_h=z(spec.n_r),
                bz_n=z(spec.n_z + 1), cz_n=z(spec.n_z + 1), bz_h=z(spec.n_z), cz_h=z(spec.n_z))


# --------------------------------------------------------------------------
# a2: density -> permittivity (conic filter, tanh projection, Eq. 6)
# --------------------------------------------------------------------------
def _filter_offsets(spec, geom):
    R = spec.filter_radius
    di_max = int(math.floor(R / spec.dr))
    r_c = geom.r_h[geom.i_d0:geom.i_d1]                       # pixel-centre radii
    dj_max = int(math.floor(R / (float(r_c.min()) * geom.dphi)))
    return R, di_max, dj_max, r_c


def conic_filter(spec, geom, rho):
    """Conic filter on the curvilinear wedge ("Results and Discussion", last
    paragraph: standard conic filter).  Reading: weight max(0, 1 - d/R) with
    d^2 = (di dr)^2 + (r_c dj dphi)^2, r_c the output pixel's radius; the
    density wraps periodically in phi (it repeats every wedge); pixels beyond
    the design's r-edges are dropped and the weights renormalised."""
    if spec.filter_radius <= 0:
        return rho.copy()
    R, di_max, dj_max, r_c = _filter_offsets(spec, geom)
    nrd, nphi = rho.shape
    out = np.zeros_like(rho)
    norm = np.zeros(nrd)
    for di in range(-di_max, di_max + 1):
        lo, hi = max(0, -di), min(nrd, nrd - di)      # output rows with a valid input row
        for dj in range(-dj_max, dj_max + 1):
            d = np.sqrt((di * spec.dr) ** 2 + (r_c[lo:hi] * dj * geom.dphi) ** 2)
            w = np.maximum(0.0, 1.0 - d / R)
            out[lo:hi] += w[:, None] * np.roll(rho, -dj, axis=1)[lo + di:hi + di]
            norm[lo:hi] += w
    return out / norm[:, None]


def conic_filter_T(spec, geom, g):
    """Transpose of conic_filter (for the chain rule back to rho)."""
    if spec.filter_radius <= 0:
        return g.copy()
    R, di_max, dj_max, r_c = _filter_offsets(spec, geom)
    nrd, nphi = g.shape
    norm = np.zeros(nrd)
    for di in range(-di_max, di_max + 1):
        lo, hi = max(0, -di), min(nrd, nrd - di)
        for dj in range(-dj_max, dj_max + 1):
            d = np.sqrt((di * spec.dr) ** 2 + (r_c[lo:hi] * dj * geom.dphi) ** 2)
            norm[lo:hi] += np.maximum(0.0, 1.0 - d / R)
    gn = g / norm[:, None]
    out = np.zeros_like(g)
    for di in range(-di_max, di_max + 1):
        lo, hi = max(0, -di), min(nrd, nrd - di)
        for dj in range(-dj_max, dj_max + 1):
            d = np.sqrt((di * spec.dr) ** 2 + (r_c[lo:hi] * dj * geom.dphi) ** 2)
            w = np.maximum(0.0, 1.0 - d / R)
            contrib = np.zeros_like(g)
            contrib[lo + di:hi + di] = w[:, None] * gn[lo:hi]
            out += np.roll(contrib, dj, axis=1)
    return out


def project(spec, x):
    """Binarising tanh projection ("Results and Discussion": standard
    binarization filter).  Reading: [tanh(b e) + tanh(b (x - e))] /
    [tanh(b e) + tanh(b (1 - e))]; beta <= 0 means no projection."""
    b, e = spec.beta, spec.eta
    if b <= 0:
        return x.copy()
    return (math.tanh(b * e) + np.tanh(b * (x - e))) / (math.tanh(b * e) + math.tanh(b * (1 - e)))


def project_grad(spec, x):
    b, e = spec.beta, spec.eta
    if b <= 0:
        return np.ones_like(x)
    return b / np.cosh(b * (x - e)) ** 2 / (math.tanh(b * e) + math.tanh(b * (1 - e)))


def rho_tilde(spec, geom, rho):
    return project(spec, conic_filter(spec, geom, rho))


def cell_eps(spec, geom, rt):
    """Per-cell permittivity [nr][nphi][nz]: the layer table outside the design
    layer; inside it Eq. 6, eps = eps_lo + rho~ (eps_hi - eps_lo) over the
    design annulus.  Reading: the design layer's cells inside the r-PMLs hold
    the background eps_lo, so no density-dependent site lies in a PML (the
    PML's discrete operator is not self-transposed, and the adjoint gradient
    would be wrong there)."""
    s = spec
    k = np.arange(s.n_z)
    layer = np.searchsorted(np.asarray(s.layer_k0), k, side="right") - 1
    eps_k = np.asarray(s.layer_eps, dtype=np.float64)[layer]
    cells = np.broadcast_to(eps_k, (s.n_r, s.n_phi, s.n_z)).copy()
    cells[:, :, s.design_k0:s.design_k1] = s.eps_lo
    eps_d = s.eps_lo + rt * (s.eps_hi - s.eps_lo)                        # (nrd, nphi)
    cells[geom.i_d0:geom.i_d1, :, s.design_k0:s.design_k1] = eps_d[:, :, None]
    return cells


def _sh(a, axis, d, wrap):
    """a shifted so that out[idx] = a[idx + d] along axis; clamp or wrap."""
    n = a.shape[axis]
    idx = np.arange(n) + d
    idx = idx % n if wrap else np.clip(idx, 0, n - 1)
    return np.take(a, idx, axis=axis)


def site_eps(spec, geom, rt):
    """Permittivity at the E sites (reading: arithmetic mean of the cells
    sharing the site -- E_r: 2 phi-neighbours x 2 z-neighbours; E_phi:
    2 r-neighbours x 2 z-neighbours; E_z: 2 r x 2 phi neighbours; phi wraps,
    r and z clamp at the domain edge)."""
    c = cell_eps(spec, geom, rt)
    er = 0.25 * sum(_sh(_sh(c, 1, dj, True), 2, dk, False) for dj in (-1, 0) for dk in (-1, 0))
    ep = 0.25 * sum(_sh(_sh(c, 0, di, False), 2, dk, False) for di in (-1, 0) for dk in (-1, 0))
    ez = 0.25 * sum(_sh(_sh(c, 0, di, False), 1, dj, True) for di in (-1, 0) for dj in (-1, 0))
    return er, ep, ez


def _sh_T(g, axis, d, wrap):
    """Transpose of _sh."""
    n = g.shape[axis]
    idx = np.arange(n) + d
    idx = idx % n if wrap else np.clip(idx, 0, n - 1)
    out = np.zeros_like(g)
    moved = np.moveaxis(out, axis, 0)
    np.add.at(moved, idx, np.moveaxis(g, axis, 0))
    return out


def site_eps_T(spec, geom, g_er, g_ep, g_ez):
    """Chain rule of site_eps and cell_eps: d/d rho~ from d/d eps at the sites."""
    s = spec
    gc = 0.25 * sum(_sh_T(_sh_T(g_er, 2, dk, False), 1, dj, True) for dj in (-1, 0) for dk in (-1, 0))
    gc += 0.25 * sum(_sh_T(_sh_T(g_ep, 2, dk, False), 0, di, False) for di in (-1, 0) for dk in (-1, 0))
    gc += 0.25 * sum(_sh_T(_sh_T(g_ez, 1, dj, True), 0, di, False) for di in (-1, 0) for dj in (-1, 0))
    gcol = gc[:, :, s.design_k0:s.design_k1].sum(axis=2) * (s.eps_hi - s.eps_lo)   # (nr, nphi)
    return gcol[geom.i_d0:geom.i_d1].copy()


# --------------------------------------------------------------------------
# a4/a5: source and DFT tables
# --------------------------------------------------------------------------
def pulse(spec, t):
    """Gaussian pulse centred at f0 (reading: cos(2 pi f0 (t - t0))
    exp(-(t - t0)^2 / (2 sigma^2)))."""
    u = t - spec.pulse_t0
    return np.cos(2 * math.pi * spec.pulse_f0 * u) * np.exp(-u * u / (2 * spec.pulse_sigma ** 2))


def plane_wave_pattern(spec, geom):
    """Normally incident x-polarised plane wave, m = +1 part ("Results and
    Discussion": a normally incident plane wave splits into m = +-1).
    x-hat = (cos phi, -sin phi) in (r, phi) has m = +1 part
    (1/2, i/2) e^{i phi}; the sheet current per cell is that / dz."""
    s = spec
    pr = 0.5 * np.exp(1j * s.m * geom.phi_n)[None, :] * np.ones((s.n_r, 1)) / s.dz
    pp = 0.5j * np.exp(1j * s.m * geom.phi_h)[None, :] * np.ones((s.n_r, 1)) / s.dz
    return np.stack([pr, pp])[None].astype(np.complex128)      # [1][2][nr][nphi]


def twiddles(geom, n_steps):
    """DFT weights e^{i w t_{n+1}} dt for the signed frequency list (reading:
    e^{-i w t} phasors, X(w) = sum_n E^n e^{i w n dt} dt)."""
    t = geom.dt * (np.arange(n_steps) + 1.0)
    return (np.exp(1j * np.outer(t, geom.omega)) * geom.dt).astype(np.complex128)


# --------------------------------------------------------------------------
# time loop driver (C)
# --------------------------------------------------------------------------
def run(spec, geom, eps, n_steps=None, pml=None, src_pat=None, src_time=None, src_k=None,
        twiddle=None, mon_k=None, design=True, state=None, nthreads=0, bloch=None):
    """Run the Yee time loop (fdtd_ref.c).  Returns (mon_dft, des_dft, state)."""
    s = spec
    n_steps = s.n_steps if n_steps is None else int(n_steps)
    pml = cpml_coefficients(s, geom) if pml is None else pml
    er, ep, ez = [np.ascontiguousarray(a, dtype=np.float64) for a in eps]
    nf = 0 if twiddle is None else twiddle.shape[1]
    mon = None
    des = None
    if twiddle is not None:
        twiddle = np.ascontiguousarray(twiddle, dtype=np.complex128)
        if mon_k is None:
            mon_k = s.monitor_k
        if mon_k >= 0:
            mon = np.zeros((nf, 2, s.n_r, s.n_phi), np.complex128)
        if design:
            des = np.zeros((nf, 3, geom.des_nk, s.n_r, s.n_phi), np.complex128)
    n_src = 0
    if src_pat is not None:
        src_pat = np.ascontiguousarray(src_pat, dtype=np.complex128)
        src_time = np.ascontiguousarray(src_time, dtype=np.complex128)
        n_src = src_pat.shape[0]
        assert src_time.shape == (n_steps, n_src)
    if state is not None:
        state = np.ascontiguousarray(state, dtype=np.complex128)
        assert state.shape == (N_STATE, s.n_r, s.n_phi, s.n_z)
    metric = int(pml.get("metric", 0))
    pm = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in pml.items()
          if k not in ("metric", "alpha_s")}
    if metric:
        mt = {k: _ptr(pm[k]) for k in ("bm_n", "cm_n", "bm_h", "cm_h")}
    else:
        mt = dict(bm_n=None, cm_n=None, bm_h=None, cm_h=None)
    b = geom.bloch if bloch is None else bloch
    P = _Problem(
        nr=s.n_r, nphi=s.n_phi, nz=s.n_z, n_steps=n_steps,
        r_lo=s.r_lo, dr=s.dr, dz=s.dz, dphi=geom.dphi, dt=geom.dt,
        bloch_re=b.real, bloch_im=b.imag,
        eps_r=_ptr(er), eps_p=_ptr(ep), eps_z=_ptr(ez),
        br_n=_ptr(pm["br_n"]), cr_n=_ptr(pm["cr_n"]), br_h=_ptr(pm["br_h"]), cr_h=_ptr(pm["cr_h"]),
        bz_n=_ptr(pm["bz_n"]), cz_n=_ptr(pm["cz_n"]), bz_h=_ptr(pm["bz_h"]), cz_h=_ptr(pm["cz_h"]),
        src_k=(s.source_k if src_k is None else src_k), n_src=n_src,
        src_pat=_ptr(src_pat), src_time=_ptr(src_time),
        n_freq=nf, twiddle=_ptr(twiddle),
        mon_k=(mon_k if mon is not None else -1), mon_dft=_ptr(mon),
        des_k0=geom.des_k0, des_nk=(geom.des_nk if des is not None else 0), des_dft=_ptr(des),
        state=_ptr(state), nthreads=int(nthreads), bor=int(geom.bor), m=int(s.m),
        rpml_metric=metric, **mt)
    rc = _lib().orc_run(ctypes.byref(P))
    if rc != 0:
        raise RuntimeError("oracle time loop failed: %d" % rc)
    return mon, des, state


# --------------------------------------------------------------------------
# decay rule: the time-domain fields must have died out by the end of the run
# --------------------------------------------------------------------------
def field_energy(spec, geom, eps, state):
    """Electromagnetic energy of a field state, sum over the Yee sites of
    eps_s abs(E_s)^2 V_s + abs(H_s)^2 V_s, V = r dr dphi dz with r at the
    site's radius (E_r, H_phi, H_z at r_{i+1/2}; E_phi, E_z, H_r at r_i).
    Section "Differentiable FDTD": the frequency-domain adjoint (all
    frequencies from one forward and one adjoint run) equals the gradient of
    the running-DFT objective only once the fields have decayed; this is the
    quantity whose decay is measured (the PML auxiliaries are not fields and
    are left out)."""
    s = spec
    vol_h = (geom.r_h * s.dr * geom.dphi * s.dz)[:, None, None]
    vol_n = (geom.r_n[:s.n_r] * s.dr * geom.dphi * s.dz)[:, None, None]
    er, ep, ez = eps
    a2 = lambda x: np.abs(x) ** 2
    w = np.sum(er * a2(state[0]) * vol_h) + np.sum(ep * a2(state[1]) * vol_n) + np.sum(ez * a2(state[2]) * vol_n)
    w += np.sum(a2(state[3]) * vol_n) + np.sum(a2(state[4]) * vol_h) + np.sum(a2(state[5]) * vol_h)
    return float(w)


def energy_trace(spec, rho, n_steps, every, nthreads=0, pml_form=0):
    """Field energy of the forward run (plane-wave source) after steps
    every, 2 every, ...: W of the state and Wdot of its one-step difference
    (E^{n+1} - E^n, H^{n+1/2} - H^{n-1/2}).  The run is cut into chunks that
    carry the full state (fields and PML auxiliaries), so the trace is that of
    one uninterrupted run.  Returns (steps, W, Wdot).

    Wdot is the decay measure.  The sheet source's pulse has a nonzero time
    integral, so the run leaves a static charge whose field never decays; a
    static field has no one-step difference and no component at the DFT
    frequencies +-w, while every oscillating field does."""
    geom = Geometry(spec)
    pml = cpml_coefficients(spec, geom, metric=bool(pml_form))
    rt = rho_tilde(spec, geom, np.asarray(rho, dtype=np.float64))
    eps = site_eps(spec, geom, rt)
    state = np.zeros((N_STATE, spec.n_r, spec.n_phi, spec.n_z), np.complex128)
    pat = plane_wave_pattern(spec, geom)

    def advance(n0, n1):
        t_half = geom.dt * (np.arange(n0, n1) + 0.5)
        src_t = pulse(spec, t_half)[:, None].astype(np.complex128)
        run(spec, geom, eps, n_steps=n1 - n0, pml=pml, src_pat=pat, src_time=src_t, state=state,
            nthreads=nthreads)

    steps, ws, wds = [], [], []
    n0 = 0
    while n0 + every <= n_steps:
        n1 = n0 + every
        if n1 - 1 > n0:
            advance(n0, n1 - 1)
        prev = state[:6].copy()
        advance(n1 - 1, n1)
        steps.append(n1)
        ws.append(field_energy(spec, geom, eps, state))
        wds.append(field_energy(spec, geom, eps, state[:6] - prev))
        n0 = n1
    return np.array(steps), np.array(ws), np.array(wds)


def decay_steps(steps, wdot, tol=1e-8):
    """The decay rule: the first sampled step after the peak of Wdot at which
    Wdot is at most tol times that peak (None if the trace never gets there)."""
    steps = np.asarray(steps)
    w = np.asarray(wdot)
    k = int(np.argmax(w))
    below = np.nonzero(w[k:] <= tol * w[k])[0]
    return int(steps[k + below[0]]) if below.size else None


# --------------------------------------------------------------------------
# a6/a7: near-to-far focal transform and objective
# --------------------------------------------------------------------------
def focal_weights(spec, geom):
    """Weights w_q on the monitor-plane E_r and E_phi sites so that the focal
    phasor is S_q = sum w_q E_q (readings of "Results and Discussion" +
    Eq. 9's focal intensity):

    * Rayleigh-Sommerfeld (first kind) propagation of each Cartesian E
      component from the monitor plane to the on-axis focal point,
      K(R) = (1/2pi) (z/R) (1/R - i k) e^{i k R} / R, z = f - (z_mon - z_top).
    * On the axis only the m = +-1 parts survive; the m = +1 part gives
      (E_x, E_y) = c+ (1, i) with c+ = (n/2) int K (u_r - i u_phi) r dr dphi,
      u = psi e^{-i phi} (the integral of the tau-periodic u over the full
      circle is n times its wedge integral).
    * The m = -1 field is the complex conjugate of the m = +1 run, so at
      +w it is conj(Psi(-w)); it gives c- (1, -i).  We report S(+w) = c+ and
      S(-w) = conj(c-); I = |E_x|^2 + |E_y|^2 = 2 (|S(+w)|^2 + |S(-w)|^2).
    * Quadrature over the design annulus [r0, r1]: midpoint at the E_r
      (half-node) radii, trapezoid at the E_phi (node) radii.
    """
    s = spec
    if s.m != 1:
        raise ValueError("the on-axis focal transform needs the m = 1 run")
    k_mon = s.monitor_k
    layer = np.searchsorted(np.asarray(s.layer_k0), k_mon, side="right") - 1
    n_top = math.sqrt(s.layer_eps[layer])
    z_top = s.design_k1 * s.dz
    zf = s.focal - (k_mon * s.dz - z_top)
    nq = geom.n_freq
    wr = np.zeros((nq, s.n_r, s.n_phi), np.complex128)
    wp = np.zeros((nq, s.n_r, s.n_phi), np.complex128)
    qr = np.zeros(s.n_r)
    qr[geom.i_d0:geom.i_d1] = s.dr
    qp = np.zeros(s.n_r + 1)
    qp[geom.i_d0:geom.i_d1 + 1] = s.dr
    qp[geom.i_d0] *= 0.5
    qp[geom.i_d1] *= 0.5
    qp = qp[:s.n_r]   # E_phi node i = n_r is the PEC wall (never inside the annulus)
    for q in range(nq):
        lam = s.wavelengths[q % geom.n_lambda]
        kk = 2 * math.pi * n_top / lam

        def G(r):
            R = np.sqrt(zf * zf + r * r)
            K = (1 / (2 * math.pi)) * (zf / R) * (1 / R - 1j * kk) * np.exp(1j * kk * R) / R
            return 0.5 * (1 if geom.bor else s.n_fold) * K * r * geom.dphi

        gr = G(geom.r_h) * qr
        gp = G(geom.r_n[:s.n_r]) * qp
        if q >= geom.n_lambda:
            gr, gp = np.conj(gr), np.conj(gp)
        wr[q] = gr[:, None] * np.exp(-1j * geom.phi_n)[None, :]
        wp[q] = -1j * gp[:, None] * np.exp(-1j * geom.phi_h)[None, :]
    return wr, wp, zf


def focal_phasors(spec, geom, mon):
    wr, wp, _ = focal_weights(spec, geom)
    return np.einsum("qij,qij->q", wr, mon[:, 0]) + np.einsum("qij,qij->q", wp, mon[:, 1])


def intensity(S):
    """Summed focal-spot intensity over wavelengths, I = 2 sum_q |S_q|^2."""
    return 2.0 * float(np.sum(np.abs(S) ** 2))


def intensity_grad(S):
    """d I / d(Re S) + i d I / d(Im S)."""
    return 4.0 * S


# --------------------------------------------------------------------------
# forward and adjoint (hybrid time/frequency adjoint)
# --------------------------------------------------------------------------
def forward(spec, rho, nthreads=0, n_steps=None, pml_form=0):
    """Forward zone solve: rho -> rho~ -> eps -> time loop with the plane-wave
    source -> monitor and design-volume DFTs -> focal phasors S -> I.
    pml_form 1: the stretched-coordinate r-PML (cpml_coefficients, metric)."""
    geom = Geometry(spec)
    pml = cpml_coefficients(spec, geom, metric=bool(pml_form))
    rt = rho_tilde(spec, geom, np.asarray(rho, dtype=np.float64))
    eps = site_eps(spec, geom, rt)
    n = spec.n_steps if n_steps is None else n_steps
    t_half = geom.dt * (np.arange(n) + 0.5)
    src_t = pulse(spec, t_half)[:, None].astype(np.complex128)
    mon, des, _ = run(spec, geom, eps, n_steps=n, pml=pml, src_pat=plane_wave_pattern(spec, geom),
                      src_time=src_t, twiddle=twiddles(geom, n), nthreads=nthreads)
    S = focal_phasors(spec, geom, mon)
    return dict(geom=geom, rho_tilde=rt, eps=eps, mon=mon, des=des, S=S, I=intensity(S), n_steps=n,
                pml=pml)


def adjoint_pulse_matrix(spec, geom, n_steps):
    """Time profiles k_q(t_{n+1/2}) of the broadband adjoint source (section
    "Differentiable FDTD": broadband adjoint sources built from temporal pulses
    so that every frequency is extracted from one run).  Reading:

    * basis pulses are first differences g_l[n] = p_l(t_{n+1}) - p_l(t_n) of
      p_l(t) = e^{+i w_l (t - t0a)} exp(-(t - t0a)^2 / (2 sigma^2)),
      t0a = 6 sigma, so each is centred at -w_l and sums to zero over the run
      (the adjoint patterns are not divergence-free: a DC component would
      leave static charge whose field never decays);
    * k_q = sum_l C_ql g_l with C the inverse of the discrete DFT matrix
      G'_lj = sum_n g_l[n] e^{-i w_j t_{n+1/2}} dt, so that the DFT of k_q
      at -w_j is exactly delta_qj.
    """
    t_half = geom.dt * (np.arange(n_steps) + 0.5)
    t_full = geom.dt * np.arange(n_steps + 1)
    t0a = 6.0 * spec.pulse_sigma
    u = t_full - t0a
    p = np.exp(1j * np.outer(u, geom.omega)) * np.exp(-u * u / (2 * spec.pulse_sigma ** 2))[:, None]
    g = p[1:] - p[:-1]                                               # [n][l]
    Gp = (g.T @ np.exp(-1j * np.outer(t_half, geom.omega))) * geom.dt   # [l][j]
    C = np.linalg.inv(Gp)                                            # C @ Gp = I
    return g @ C.T                                                   # [n][q]


def adjoint(spec, fwd, dI_dS, nthreads=0):
    """Adjoint gradient dI/drho (hybrid time/frequency adjoint, section
    "Differentiable FDTD").  Steps:

    1. a_q(x) = conj(g_q) w_q(x): the sensitivity of I to the monitor DFT,
       g_q = dI/dRe S_q + i dI/dIm S_q.
    2. The frequency-domain system of the Yee scheme is
       (curl curl - wt^2 eps) E = i wt J with wt = (2/dt) sin(w dt/2); its
       transpose in the Bloch-m space is V (Bloch -m operator) V^-1, and the
       Bloch -m run equals the conjugate of a Bloch +m run with conjugated
       sources.  So the adjoint is a +m run with source patterns
       b_q = i conj(a_q) / (wt_q V) on the monitor-plane sites and time
       profiles k_q whose DFT at -w_j is delta_qj, with a design-volume DFT.
    3. dI/deps_s = Re sum_q wt_q^2 V_s E_q(s) conj(A_{-q}(s)), A the adjoint
       run's DFT at -w_q.
    4. Chain rule through the site averaging, Eq. 6, the projection and the
       conic filter.
    """
    s = spec
    geom = fwd["geom"]
    n = fwd["n_steps"]
    g = np.asarray(dI_dS, dtype=np.complex128)
    wr, wp, _ = focal_weights(s, geom)
    wt = geom.omega_tilde()
    k = s.monitor_k
    Vr = (geom.r_h * s.dr * geom.dphi * s.dz)[:, None]
    Vp = (geom.r_n[:s.n_r] * s.dr * geom.dphi * s.dz)[:, None]
    a_r = np.conj(g)[:, None, None] * wr
    a_p = np.conj(g)[:, None, None] * wp
    b_r = 1j * np.conj(a_r) / (wt[:, None, None] * Vr[None])
    with np.errstate(invalid="ignore", divide="ignore"):       # V = 0 on the axis
        b_p = 1j * np.conj(a_p) / (wt[:, None, None] * Vp[None])
    b_p[:, 0, :] = 0.0                                 # E_phi on the PEC wall r_lo (or the axis)
    pat = np.stack([b_r, b_p], axis=1)                 # [q][2][nr][nphi]
    src_t = adjoint_pulse_matrix(s, geom, n)
    _, des_a, _ = run(s, geom, fwd["eps"], n_steps=n, pml=fwd.get("pml"), src_pat=pat, src_time=src_t, src_k=k,
                      twiddle=twiddles(geom, n), mon_k=-1, nthreads=nthreads)
    nl = geom.n_lambda
    qbar = (np.arange(geom.n_freq) + nl) % geom.n_freq
    des_f = fwd["des"]
    V = [(geom.r_h * s.dr * geom.dphi * s.dz)[:, None],
         (geom.r_n[:s.n_r] * s.dr * geom.dphi * s.dz)[:, None],
         (geom.r_n[:s.n_r] * s.dr * geom.dphi * s.dz)[:, None]]
    gsite = []
    for c in range(3):
        acc = np.zeros((geom.des_nk, s.n_r, s.n_phi))
        for q in range(geom.n_freq):
            acc += np.real(wt[q] ** 2 * des_f[q, c] * np.conj(des_a[qbar[q], c]))
        full = np.zeros((s.n_r, s.n_phi, s.n_z))
        full[:, :, geom.des_k0:geom.des_k0 + geom.des_nk] = np.moveaxis(acc, 0, 2) * V[c][:, :, None]
        gsite.append(full)
    g_rt = site_eps_T(s, geom, *gsite)
    return dict(grad_rho_tilde=g_rt, des_adj=des_a, site_grad=gsite)


def gradient(spec, rho, nthreads=0, n_steps=None, pml_form=0):
    """dI/drho for I = summed focal intensity: forward, adjoint, then the
    projection derivative and the transposed conic filter."""
    rho = np.asarray(rho, dtype=np.float64)
    fwd = forward(spec, rho, nthreads=nthreads, n_steps=n_steps, pml_form=pml_form)
    fwd["rho"] = rho
    adj = adjoint(spec, fwd, intensity_grad(fwd["S"]), nthreads=nthreads)
    geom = fwd["geom"]
    rbar = conic_filter(spec, geom, rho)
    g_rbar = adj["grad_rho_tilde"] * project_grad(spec, rbar)
    g_rho = conic_filter_T(spec, geom, g_rbar)
    return fwd["I"], g_rho, fwd, adj


# --------------------------------------------------------------------------
# a14: focal-plane field (off axis) and transmitted power
# --------------------------------------------------------------------------
def focal_plane_bruteforce(spec, geom, mon, pts):
    """Physical focal-plane field (E_x, E_y) [n_lambda][n_pts] of one zone by
    brute force: every wedge copy c of the monitor plane is rebuilt with its
    Bloch phase e^{i m c tau} (all azimuthal orders kept), the physical phasor
    at +w is Psi(+w) + conj(Psi(-w)) (m = +1 run plus its conjugate), and the
    Rayleigh-Sommerfeld (first kind) kernel is summed over every site of the
    full circle (midpoint radial weights at E_r, trapezoid at E_phi, the grid's
    dphi).  For continuous axisymmetry the circle is sampled with n_phi_bor
    points."""
    s = spec
    nl = geom.n_lambda
    layer = np.searchsorted(np.asarray(s.layer_k0), s.monitor_k, side="right") - 1
    n_top = math.sqrt(s.layer_eps[layer])
    zf = s.focal - (s.monitor_k * s.dz - s.design_k1 * s.dz)
    qr = np.zeros(s.n_r)
    qr[geom.i_d0:geom.i_d1] = s.dr
    qp = np.zeros(s.n_r + 1)
    qp[geom.i_d0:geom.i_d1 + 1] = s.dr
    qp[geom.i_d0] *= 0.5
    qp[geom.i_d1] *= 0.5
    qp = qp[:s.n_r]
    pts = np.asarray(pts, dtype=np.float64)
    pts = np.concatenate([pts, np.zeros((len(pts), 1))], axis=1) if pts.shape[-1] == 2 else pts.reshape(-1, 3)
    if geom.bor:
        ncopy, dphi, nphi = 1, 2 * math.pi / 256, 256
    else:
        ncopy, dphi, nphi = s.n_fold, geom.dphi, s.n_phi
    ex = np.zeros((nl, len(pts)), complex)
    ey = np.zeros((nl, len(pts)), complex)
    for l in range(nl):
        kk = 2 * math.pi * n_top / s.wavelengths[l]
        Er = mon[l, 0] + np.conj(mon[l + nl, 0])           # [nr][nphi] physical phasors
        Ep = mon[l, 1] + np.conj(mon[l + nl, 1])
        for comp in (0, 1):
            r = geom.r_h if comp == 0 else geom.r_n[:s.n_r]
            w = qr if comp == 0 else qp
            if geom.bor:
                # the axis zone stores u: the physical field is u e^{i phi} + conj(u(-w)) e^{-i phi}
                phis = dphi * np.arange(nphi)
                up = mon[l, comp][:, 0][:, None] * np.exp(1j * phis)[None, :]
                um = np.conj(mon[l + nl, comp][:, 0])[:, None] * np.exp(-1j * phis)[None, :]
                F = up + um
                ph = np.broadcast_to(phis, F.shape)
            else:
                base = geom.phi_n if comp == 0 else geom.phi_h
                F = []
                ph = []
                for c in range(ncopy):
                    # psi of copy c = e^{i m c tau} psi; its conjugate part gets the opposite phase
                    Pp = mon[l, comp] * np.exp(1j * s.m * c * geom.tau)
                    Pm = np.conj(mon[l + nl, comp] * np.exp(1j * s.m * c * geom.tau))
                    F.append(Pp + Pm)
                    ph.append(np.broadcast_to(base + c * geom.tau, Pp.shape))
                F = np.concatenate(F, axis=1)
                ph = np.concatenate(ph, axis=1)
            cs, sn = np.cos(ph), np.sin(ph)
            fx = F * cs if comp == 0 else -F * sn
            fy = F * sn if comp == 0 else F * cs
            X = r[:, None] * cs
            Y = r[:, None] * sn
            wt = (w * r)[:, None] * dphi
            for p, (x, y, h) in enumerate(pts):
                zp = zf + h
                R = np.sqrt(zp * zp + (x - X) ** 2 + (y - Y) ** 2)
                K = (1 / (2 * math.pi)) * (zp / R) * (1 / R - 1j * kk) * np.exp(1j * kk * R) / R
                ex[l, p] += np.sum(K * fx * wt)
                ey[l, p] += np.sum(K * fy * wt)
    return ex, ey


def transmitted_power(spec, geom, mon):
    """(n/2) |E_t|^2 over the monitor annulus of the whole circle per
    wavelength (plane-wave estimate of the transmitted flux, section
    "Results and Discussion": relative focusing efficiency).

    The physical +w field is E+ + E- with E+ = psi(+w) (order m = +1) and
    E- = conj(psi(-w)) (order -1).  Over the n wedge copies the cross term
    2 Re(E+ conj(E-)) turns by e^{2 i tau} per copy and sums to zero for
    n >= 3 (and over the circle for continuous axisymmetry), so the
    full-circle sum is n sum_wedge (|E+|^2 + |E-|^2); for n = 1, 2 every copy
    carries the same cross term and it stays."""
    s = spec
    nl = geom.n_lambda
    layer = np.searchsorted(np.asarray(s.layer_k0), s.monitor_k, side="right") - 1
    n_top = math.sqrt(s.layer_eps[layer])
    copies = 1.0 if geom.bor else float(s.n_fold)
    cross = (not geom.bor) and s.n_fold <= 2
    out = np.zeros(nl)
    for l in range(nl):
        if cross:
            Er = mon[l, 0] + np.conj(mon[l + nl, 0])
            Ep = mon[l, 1] + np.conj(mon[l + nl, 1])
            pw = (np.abs(Er) ** 2 + np.abs(Ep) ** 2).sum(axis=1)
        else:
            pw = (np.abs(mon[l]) ** 2 + np.abs(mon[l + nl]) ** 2).sum(axis=(0, 2))
        i0, i1 = geom.i_d0, geom.i_d1
        out[l] = 0.5 * n_top * np.sum(pw[i0:i1] * geom.r_h[i0:i1] * s.dr * geom.dphi) * copies
    return out


# ---------------------------------------------------------------- focal-spot evaluation
# Section "Centimeter-scale metalens at long-wave infrared": the PSF and its
# FWHM, the focusing efficiency as the power within 3 FWHM of the focus over
# the incident power (relative: over the transmitted power), and Eq. 9's
# Strehl ratio SR = I lambda^2 F^2 / (P_trans A).  Written out directly on the
# sampled fields; the sample positions follow the same rule as the library's
# evaluation (a PSF line on the x axis, discs of n_rad radii x n_ang angles).

def spot_intensity(ex, ey, n_top=1.0):
    """(n_top/2)(abs(E_x)^2 + abs(E_y)^2) of focal-plane field samples."""
    return 0.5 * n_top * (np.abs(ex) ** 2 + np.abs(ey) ** 2)


def fwhm(xs, I):
    """Full width at half maximum of a profile I(xs) sampled from its peak at
    xs[0] outwards: twice the half-maximum crossing, linearly interpolated
    between the first sample below half of I[0] and the one before; NaN if
    the profile never falls below half."""
    I = np.asarray(I, dtype=np.float64)
    half = 0.5 * I[0]
    below = np.nonzero(I < half)[0]
    below = below[below > 0]
    if below.size == 0:
        return float("nan")
    j = below[0]
    x0, x1, y0, y1 = xs[j - 1], xs[j], I[j - 1], I[j]
    return 2.0 * (x0 + (half - y0) * (x1 - x0) / (y1 - y0))


def encircled_power(radii, I_of_r):
    """P(rho_k) = integral of I(r) 2 pi r dr from radii[0] to radii[k] of a
    radially symmetric spot (trapezoid rule on the given samples)."""
    r = np.asarray(radii, dtype=np.float64)
    f = np.asarray(I_of_r, dtype=np.float64) * 2 * math.pi * r
    out = np.zeros_like(r)
    out[1:] = np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(r))
    return out


def disc_points(w, n_rad, n_ang):
    """Sample disc of radius 3 w: radii (k + 1/2) 3 w / n_rad, angles 2 pi a / n_ang
    ((x, y) rows, radius-major); (radii, points)."""
    rmax = 3.0 * w
    rr = (np.arange(n_rad) + 0.5) * rmax / n_rad
    aa = 2 * math.pi * np.arange(n_ang) / n_ang
    return rr, np.array([(q * math.cos(a), q * math.sin(a)) for q in rr for a in aa])


def evaluate_spot(focal_plane, lams, lens_radius, focal, incident, n_top=1.0, n_line=192, x_max=None, n_rad=48,
                  n_ang=8):
    """FWHM, I(0), FE, relative FE, transmittance and SR per wavelength of a
    lens whose focal-plane field is focal_plane(pts) -> (E_x, E_y, P_trans)
    ([n_lambda][n_pts] each, P_trans per wavelength).  Returns a list of dicts
    and the PSF line (xs, I_line)."""
    lams = np.asarray(lams, dtype=np.float64)
    if x_max is None:
        x_max = 4.0 * lams.max()
    xs = np.linspace(0.0, x_max, n_line)
    ex, ey, p_trans = focal_plane(np.stack([xs, np.zeros_like(xs)], 1))
    I_line = spot_intensity(ex, ey, n_top)
    area = math.pi * lens_radius ** 2
    out = []
    for l in range(lams.size):
        w = fwhm(xs, I_line[l])
        rr, pts = disc_points(w, n_rad, n_ang)
        fx, fy, _ = focal_plane(pts)
        Id = spot_intensity(fx[l], fy[l], n_top).reshape(n_rad, n_ang)
        p_disc = float(np.sum(Id.mean(axis=1) * 2 * math.pi * rr) * (3.0 * w / n_rad))
        p_inc = incident[l] * area
        I0 = float(I_line[l, 0])
        out.append({"lambda": float(lams[l]), "fwhm": w, "focal_intensity": I0,
                    "focusing_efficiency": p_disc / p_inc, "relative_efficiency": p_disc / p_trans[l],
                    "transmittance": p_trans[l] / p_inc,
                    "strehl": I0 * lams[l] ** 2 * focal ** 2 / (p_trans[l] * area)})
    return out, xs, I_line

"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds workload descriptions (plain numbers: grid sizes, layer
stacks, wavelengths, seeds) and the seeded density generator.  It contains
none of the method's arithmetic: time steps, PML profiles, filters,
projections, permittivity assembly, DFT twiddles and near-to-far weights are
derived independently by the oracle and by the CUDA library.

Units: c = eps0 = mu0 = 1 and the design wavelength lambda0 = 1, so lengths
are in lambda0 and times in lambda0 / c.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["ZoneSpec", "zone_cfg1", "zone_cfg2", "zone_tiny", "zone_lwir", "zone_visible", "smoothed_rho",
           "rho_for", "lens_zones", "focal_from_na"]


@dataclass(frozen=True)
class ZoneSpec:
    """One annular zone's n-fold wedge, simulated domain including its PMLs.

    The simulated radial span is [r_lo, r_lo + n_r*dr]; the design / monitor
    annulus is the interior [r_lo + pml_r_in*dr, r_lo + (n_r - pml_r_out)*dr].
    z runs over [0, n_z*dz].  Layer l covers z-cells k >= layer_k0[l] up to the
    next layer's start; cells in [design_k0, design_k1) are the design layer,
    whose permittivity is eps_lo + rho~ (eps_hi - eps_lo).
    """
    r_lo: float
    n_r: int
    n_phi: int
    n_z: int
    n_fold: int
    dr: float = 0.05
    dz: float = 0.05
    m: int = 1
    pml_r_in: int = 8
    pml_r_out: int = 8
    pml_z: int = 8
    layer_k0: tuple = (0,)
    layer_eps: tuple = (1.0,)
    design_k0: int = 0
    design_k1: int = 0
    eps_lo: float = 1.0
    eps_hi: float = 1.0
    source_k: int = 0
    monitor_k: int = 0
    courant: float = 0.5
    n_steps: int = 100
    filter_radius: float = 0.0     # <= 0: no conic filter
    beta: float = 0.0              # <= 0: no projection
    eta: float = 0.5
    wavelengths: tuple = (1.0,)
    pulse_f0: float = 1.0
    pulse_sigma: float = 0.5
    pulse_t0: float = 2.0
    focal: float = 10.0            # focal distance above the design top (lambda0)
    label: str = "zone"

    @property
    def n_r_design(self) -> int:
        return self.n_r - self.pml_r_in - self.pml_r_out

    @property
    def cells(self) -> int:
        return self.n_r * self.n_phi * self.n_z

    def replace(self, **kw) -> "ZoneSpec":
        return dataclasses.replace(self, **kw)

    def to_json(self) -> str:
        """The spec as a JSON object (tuples as lists)."""
        import json
        return json.dumps(dataclasses.asdict(self), sort_keys=True)

    @classmethod
    def from_json(cls, text: str) -> "ZoneSpec":
        import json
        d = json.loads(text)
        for f in dataclasses.fields(cls):
            if isinstance(d.get(f.name), list):
                d[f.name] = tuple(d[f.name])
        return cls(**d)


def zone_cfg1() -> ZoneSpec:
    """Single annular zone forward solve: r in [10, 12.4] (48 cells incl. 8-cell
    r-CPMLs), n = 96 with 48 phi cells, 64 z cells incl. 8-cell z-CPMLs.
    z-stack: SiO2 (eps 2.1) for cells 0..21 with the source sheet at k = 12,
    a 12-cell (0.6 lambda) TiO2/air design layer (eps 1 / 5.76) for 22..33,
    air above with the monitor plane at k = 44 (0.5 lambda above the layer).
    Gaussian pulse centred at lambda0, 1000 steps at Courant 0.5."""
    return ZoneSpec(
        r_lo=10.0, n_r=48, n_phi=48, n_z=64, n_fold=96,
        layer_k0=(0, 22, 34), layer_eps=(2.1, 1.0, 1.0),
        design_k0=22, design_k1=34, eps_lo=1.0, eps_hi=5.76,
        source_k=12, monitor_k=44, courant=0.5, n_steps=1000,
        filter_radius=0.0, beta=0.0,
        wavelengths=(1.0,), pulse_sigma=0.5, pulse_t0=2.0, focal=20.0,
        label="cfg1 single zone 48x48x64, n=96")


def zone_cfg2(n_steps: int = 20000) -> ZoneSpec:
    """Wide zone for forward + adjoint: r in [200, 215] (300 cells), n = 4000,
    320 phi cells, 160 z cells; SiO2 to k = 40, 12-cell design layer, air;
    monitor 0.5 lambda above the layer; three wavelengths 0.82/1.0/1.18;
    conic filter R = 0.08, tanh projection beta = 8; focal distance 300."""
    return ZoneSpec(
        r_lo=200.0, n_r=300, n_phi=320, n_z=160, n_fold=4000,
        layer_k0=(0, 40, 52), layer_eps=(2.1, 1.0, 1.0),
        design_k0=40, design_k1=52, eps_lo=1.0, eps_hi=5.76,
        source_k=12, monitor_k=62, courant=0.5, n_steps=n_steps,
        filter_radius=0.08, beta=8.0, eta=0.5,
        wavelengths=(0.82, 1.0, 1.18), pulse_sigma=0.4, pulse_t0=1.6,
        focal=300.0, label="cfg2 wide zone 300x320x160, n=4000, 3 wavelengths")


def zone_lwir(ell: int = 16, n_steps: int = 4000) -> ZoneSpec:
    """Zone l (2..16) of the paper's LWIR lens at its own discretisation
    (section "Centimeter-scale metalens at long-wave infrared"): 25 lambda
    wide, r in [25 (l - 1), 25 l], fold n = 720 l, dr = dz = lambda / 50,
    r dphi < 0.021 lambda (11 phi cells), silicon (n = 3.42) substrate and
    0.6 lambda design layer, NA 0.3 focus of the 800-lambda lens.  A
    throughput workload: the z stack (0.64 lambda of substrate below the
    layer, the monitor 0.5 lambda above it, 8-cell CPMLs) is this build's
    choice."""
    eps_si = 3.42 ** 2
    n_phi = int(np.ceil(25.0 * ell * 2 * np.pi / (720 * ell) / 0.021))
    return ZoneSpec(
        r_lo=25.0 * (ell - 1) - 8 * 0.02, n_r=1250 + 16, n_phi=n_phi, n_z=112, n_fold=720 * ell,
        dr=0.02, dz=0.02, pml_r_in=8, pml_r_out=8, pml_z=8,
        layer_k0=(0, 40, 70), layer_eps=(eps_si, 1.0, 1.0),
        design_k0=40, design_k1=70, eps_lo=1.0, eps_hi=eps_si,
        source_k=20, monitor_k=95, courant=0.5, n_steps=n_steps,
        filter_radius=0.08, beta=8.0, eta=0.5, wavelengths=(1.0,),
        pulse_sigma=0.5, pulse_t0=2.0, focal=focal_from_na(400.0, 0.3),
        label="LWIR zone %d: 25 lambda, lambda/50, n = %d" % (ell, 720 * ell))


def zone_visible(ell: int = 16, lens: str = "rgb", n_steps: int = 4000) -> ZoneSpec:
    """Zone l (2..32) of the paper's visible lenses at their lambda/36 grid
    (section "Millimeter-scale poly-achromatic metalenses in the visible"),
    lambda = the longest design wavelength:
    rgb:  25 lambda zones, fold n = 360 l, wavelengths 0.74 / 0.81 / 1.0,
          NA 0.8 (f = 600 lambda for the 800-lambda radius);
    poly: 47 lambda zones, fold n = 1440 l, six wavelengths 490..650 nm
          relative to 650 nm, NA 0.3.
    TiO2 (n = 2.4) one wavelength thick (658 nm) on fused silica (n = 1.46);
    conic filter radius 0.056 lambda; phi cells so that r dphi <= lambda/36 at
    the zone's outer radius.  A throughput workload: the z stack (0.64 lambda
    of substrate under the layer, the monitor 0.5 lambda above it, 8-cell
    CPMLs) is this build's choice, as for the LWIR zone."""
    if lens == "rgb":
        width, fold, lams, na = 25.0, 360 * ell, (0.74, 0.81, 1.0), 0.8
    elif lens == "poly":
        width, fold, lams, na = 47.0, 1440 * ell, tuple(round(w / 650.0, 4) for w in (490, 520, 540, 570, 610, 650)), 0.3
    else:
        raise ValueError("lens must be 'rgb' or 'poly'")
    h = 1.0 / 36.0
    n_phi = int(np.ceil(width * ell * 2 * np.pi / fold / h))
    k_layer, k_top = 8 + 23, 8 + 23 + 36
    return ZoneSpec(
        r_lo=width * (ell - 1) - 8 * h, n_r=int(round(width * 36)) + 16, n_phi=n_phi, n_z=k_top + 18 + 8 + 7,
        n_fold=fold, dr=h, dz=h, pml_r_in=8, pml_r_out=8, pml_z=8,
        layer_k0=(0, k_layer, k_top), layer_eps=(1.46 ** 2, 1.0, 1.0),
        design_k0=k_layer, design_k1=k_top, eps_lo=1.0, eps_hi=2.4 ** 2,
        source_k=14, monitor_k=k_top + 18, courant=0.5, n_steps=n_steps,
        filter_radius=0.056, beta=8.0, eta=0.5, wavelengths=lams,
        pulse_sigma=0.4, pulse_t0=1.6, focal=focal_from_na(32 * width, na),
        label="%s zone %d: %g lambda, lambda/36, n = %d" % (lens, ell, width, fold))


def zone_patch(r_mid: float = 200.0, n_steps: int = 830, n_design: int = 128, n_phi: int = 128,
               arc: float = 6.4) -> ZoneSpec:
    """A surrogate-sized zone: n_design x n_phi design pixels at lambda/20
    (6.4 x 6.4 lambda for 128 x 128) centred on radius r_mid, fold
    n = round(2 pi r_mid / arc) so the wedge arc at r_mid is ~arc; the wide
    zone's z stack (SiO2 substrate, 0.6 lambda TiO2 design layer, air, monitor
    0.5 lambda above), three wavelengths 0.82 / 1.0 / 1.18, conic filter
    R = 0.08, tanh projection beta = 8; 8-cell PMLs in r and z."""
    pml = 8
    dr = 0.05
    nf = max(1, int(round(2.0 * math.pi * r_mid / arc)))
    r_lo = r_mid - 0.5 * n_design * dr - pml * dr
    return ZoneSpec(
        r_lo=r_lo, n_r=n_design + 2 * pml, n_phi=n_phi, n_z=160, n_fold=nf, dr=dr, dz=dr,
        pml_r_in=pml, pml_r_out=pml, pml_z=pml,
        layer_k0=(0, 40, 52), layer_eps=(2.1, 1.0, 1.0),
        design_k0=40, design_k1=52, eps_lo=1.0, eps_hi=5.76,
        source_k=12, monitor_k=62, courant=0.5, n_steps=n_steps,
        filter_radius=0.08, beta=8.0, eta=0.5,
        wavelengths=(0.82, 1.0, 1.18), pulse_sigma=0.4, pulse_t0=1.6,
        focal=300.0, label="surrogate patch zone at r = %g lambda (%dx%d design pixels)" % (r_mid, n_design, n_phi))


def zone_tiny(**kw) -> ZoneSpec:
    """A small zone for oracle pins and quick parity cases (defaults: 24 r-cells
    with 4-cell PMLs, 8 phi cells, 40 z-cells, coarse lambda/10 grid)."""
    base = dict(
        r_lo=5.0, n_r=24, n_phi=8, n_z=40, n_fold=40, dr=0.1, dz=0.1,
        pml_r_in=4, pml_r_out=4, pml_z=6,
        layer_k0=(0, 16, 20), layer_eps=(2.1, 1.0, 1.0),
        design_k0=16, design_k1=20, eps_lo=1.0, eps_hi=5.76,
        source_k=9, monitor_k=24, courant=0.5, n_steps=600,
        filter_radius=0.0, beta=0.0, wavelengths=(1.0,),
        pulse_sigma=0.5, pulse_t0=2.0, focal=10.0, label="tiny zone")
    base.update(kw)
    return ZoneSpec(**base)


def smoothed_rho(n_rd: int, n_phi: int, seed: int, sigma: float = 2.0,
                 mode: str = "binary") -> np.ndarray:
    """Seeded design density on the (r, phi) design grid, shape (n_rd, n_phi).

    Uniform [0,1) noise from numpy's default_rng(seed), Gaussian-smoothed with
    sigma cells (reflecting in r, wrapping in phi because the density is
    periodic over the wedge), then either thresholded at 0.5 ("binary") or
    min-max normalised to [0, 1] ("minmax")."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    x = rng.random((n_rd, n_phi))
    y = gaussian_filter(x, sigma=sigma, mode=("reflect", "wrap"))
    if mode == "binary":
        return (y >= 0.5).astype(np.float64)
    lo, hi = float(y.min()), float(y.max())
    return (y - lo) / max(hi - lo, 1e-30)


def rho_for(spec: ZoneSpec, seed: int) -> np.ndarray:
    """The density used with a zone: binary for projection-free zones,
    min-max normalised when a projection (beta > 0) follows."""
    mode = "minmax" if spec.beta > 0 else "binary"
    return smoothed_rho(spec.n_r_design, spec.n_phi, seed, mode=mode)


def focal_from_na(radius: float, na: float) -> float:
    """Focal length of a lens of the given radius and numerical aperture,
    NA = sin(theta) with tan(theta) = R / f."""
    return radius * math.sqrt(1.0 - na * na) / na


def lens_zones(n_zones: int = 40, radius: float = 400.0, seed: int = 4,
               width_lo: float = 8.0, width_hi: float = 15.0, arc: float = 10.0,
               n_phi: int = 200, n_z: int = 160, n_steps: int = 2000,
               dr: float = 0.05, pml: int = 8) -> list:
    """Zones of one lens covering r in [0, radius]: widths ~ U[width_lo,
    width_hi] (seeded), rescaled to sum to the radius; fold n = round(2 pi r1
    / arc) so the wedge arc stays near `arc`; the innermost zone contains the
    axis (n_fold = 0: continuously axisymmetric, one phi cell).  Each zone's
    PMLs are added outside its design annulus, so neighbouring simulated
    domains overlap by the PML widths."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(width_lo, width_hi, n_zones)
    w *= radius / w.sum()
    edges = np.concatenate([[0.0], np.cumsum(w)])
    zones = []
    for z in range(n_zones):
        r0, r1 = float(edges[z]), float(edges[z + 1])
        nd = max(1, int(round((r1 - r0) / dr)))
        if z == 0:
            zones.append(ZoneSpec(
                r_lo=0.0, n_r=nd + pml, n_phi=1, n_z=n_z, n_fold=0, dr=dr, dz=dr,
                pml_r_in=0, pml_r_out=pml, pml_z=pml,
                layer_k0=(0, 40, 52), layer_eps=(2.1, 1.0, 1.0),
                design_k0=40, design_k1=52, eps_lo=1.0, eps_hi=5.76,
                source_k=12, monitor_k=62, n_steps=n_steps,
                wavelengths=(0.82, 1.0, 1.18), pulse_sigma=0.4, pulse_t0=1.6,
                label="lens zone 0 (axis)"))
            continue
        nf = max(1, int(round(2.0 * math.pi * r1 / arc)))
        zones.append(ZoneSpec(
            r_lo=r0 - pml * dr, n_r=nd + 2 * pml, n_phi=n_phi, n_z=n_z, n_fold=nf,
            dr=dr, dz=dr, pml_r_in=pml, pml_r_out=pml, pml_z=pml,
            layer_k0=(0, 40, 52), layer_eps=(2.1, 1.0, 1.0),
            design_k0=40, design_k1=52, eps_lo=1.0, eps_hi=5.76,
            source_k=12, monitor_k=62, n_steps=n_steps,
            wavelengths=(0.82, 1.0, 1.18), pulse_sigma=0.4, pulse_t0=1.6,
            label="lens zone %d" % z))
    return zones

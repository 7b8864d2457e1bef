"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-by-element comparisons on the same seeded inputs: filter and
projection, the focal transform, forward DFT fields / final fields / focal
phasors, the adjoint DFT and the gradient, on grids that span several tiles
with ragged tails, plus the full-size wide-zone workload checked against the
oracle through the phi-invariant (ring) reduction.
Tolerances: DFT fields relative L2 <= 1e-4, gradients <= 1e-3 (FP32 device
arithmetic against FP64).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from zda_inputs import zone_lwir, zone_visible, zone_cfg1, zone_cfg2, zone_tiny, smoothed_rho, rho_for

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4
GRAD_TOL = 1e-3


KERNELS = {"split": (0, 2, 0), "split_r4": (0, 4, 0), "split_r16": (0, 16, 0), "split_r32": (0, 32, 0),
           "split_e3": (0, 8, 3),
           "split1": (2, 2, 0),
           "fused2": (1, 2, 0), "fused4": (1, 4, 0),
           "fused2_ir3": (1, 2, 3), "tile8": (3, 8, 0), "tile4": (3, 4, 0), "tile16": (3, 16, 0),
           "tile8_r5": (3, 8, 5), "etile8": (4, 8, 0), "etile16": (4, 16, 0), "etile32": (4, 32, 0),
           "etile16_r7": (4, 16, 7), "htile8": (5, 8, 0), "htile16": (5, 16, 0), "htile32": (5, 32, 0),
           "htile16_r7": (5, 16, 7)}


def _zone(spec, kernel=None):
    from paper_2501_07979_gb300 import Zone
    if kernel is not None and KERNELS[kernel][0] == 1 and (spec.n_z % 2 or spec.n_fold == 0):
        pytest.skip("the fused step needs an even n_z and an annular zone")
    if kernel is not None and KERNELS[kernel][0] in (3, 4, 5) and (spec.n_z % 2 or spec.pml_z % 2 or spec.n_fold == 0):
        pytest.skip("the tile kernels need even n_z and pml_z and an annular zone")
    z = Zone(spec, device=0)
    if kernel is not None:
        z.set_kernel(*KERNELS[kernel])
    return z


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device="cuda:0")


def _oracle_forward_state(spec, rho):
    g = O.Geometry(spec)
    rt = O.rho_tilde(spec, g, rho)
    eps = O.site_eps(spec, g, rt)
    t = g.dt * (np.arange(spec.n_steps) + 0.5)
    mon, des, st = O.run(spec, g, eps, src_pat=O.plane_wave_pattern(spec, g),
                         src_time=O.pulse(spec, t)[:, None].astype(complex),
                         twiddle=O.twiddles(g, spec.n_steps),
                         state=np.zeros((O.N_STATE, spec.n_r, spec.n_phi, spec.n_z), complex))
    return mon, des, st, O.focal_phasors(spec, g, mon)


RAGGED = {
    "tiny": zone_tiny(n_steps=300),
    "ragged": zone_tiny(n_r=27, n_phi=7, n_z=45, pml_r_in=3, pml_r_out=5, pml_z=5, n_steps=250,
                        layer_k0=(0, 15, 19), design_k0=15, design_k1=19, source_k=8, monitor_k=26,
                        wavelengths=(0.85, 1.0, 1.2), filter_radius=0.2, beta=3.0, pulse_sigma=0.4,
                        pulse_t0=1.6),
    "ragged_even": zone_tiny(n_r=27, n_phi=7, n_z=46, pml_r_in=3, pml_r_out=5, pml_z=5, n_steps=250,
                             layer_k0=(0, 15, 19), design_k0=15, design_k1=19, source_k=8, monitor_k=26,
                             wavelengths=(0.85, 1.0, 1.2), filter_radius=0.2, beta=3.0, pulse_sigma=0.4,
                             pulse_t0=1.6),
    # several tiles of the tile step in every direction, each with a ragged tail (13 phi rows, 46
    # z-cells, 27 radii), odd r-PML widths
    "ragged_tile": zone_tiny(n_r=27, n_phi=13, n_z=46, pml_r_in=3, pml_r_out=5, pml_z=6, n_steps=250,
                             layer_k0=(0, 15, 19), design_k0=15, design_k1=19, source_k=8, monitor_k=26,
                             wavelengths=(0.85, 1.0, 1.2), filter_radius=0.2, beta=3.0, pulse_sigma=0.4,
                             pulse_t0=1.6),
    "one_phi_cell": zone_tiny(n_phi=1, n_fold=300, n_steps=200, r_lo=8.0),
    "no_inner_pml": zone_tiny(pml_r_in=0, n_steps=200),
    # a 1-lambda strip of the paper's LWIR zone 16: lambda/50 grid, silicon, 11 phi cells
    "lwir_strip": zone_lwir(16, 1500).replace(n_r=66, r_lo=395.0),
    # a 1-lambda strip of the paper's RGB zone 16: lambda/36, TiO2 on SiO2, three wavelengths
    "rgb_strip": zone_visible(16, "rgb", 900).replace(n_r=52, r_lo=395.0),
}


# ------------------------------------------------------------------ K6
@pytest.mark.parametrize("name", ["cfg2", "ragged"])
def test_filter_project_matches_oracle(name):
    spec = zone_cfg2(n_steps=10) if name == "cfg2" else RAGGED["ragged"]
    g = O.Geometry(spec)
    rho = rho_for(spec, 2)
    z = _zone(spec)
    got = z.filter_project(_dev(rho)).cpu().numpy()
    want = O.project(spec, O.conic_filter(spec, g, rho))
    assert np.abs(got - want).max() < 5e-6


@pytest.mark.parametrize("name", ["cfg2", "ragged"])
def test_filter_project_backward_matches_oracle(name):
    spec = zone_cfg2(n_steps=10) if name == "cfg2" else RAGGED["ragged"]
    g = O.Geometry(spec)
    rng = np.random.default_rng(9)
    rho = rho_for(spec, 2)
    gt = rng.standard_normal(rho.shape)
    z = _zone(spec)
    got = z.filter_project_backward(_dev(rho), _dev(gt)).cpu().numpy()
    want = O.conic_filter_T(spec, g, gt * O.project_grad(spec, O.conic_filter(spec, g, rho)))
    assert _rel(got, want) < 1e-5


# ------------------------------------------------------------------ K10
@pytest.mark.parametrize("name", ["cfg2", "ragged"])
def test_focal_transform_matches_oracle(name):
    spec = zone_cfg2(n_steps=10) if name == "cfg2" else RAGGED["ragged"]
    g = O.Geometry(spec)
    rng = np.random.default_rng(4)
    sh = (g.n_freq, 2, spec.n_r, spec.n_phi)
    mon = (rng.standard_normal(sh) + 1j * rng.standard_normal(sh)).astype(np.complex64)
    z = _zone(spec)
    got = z.focal_transform(torch.tensor(mon, device="cuda:0"))
    want = O.focal_phasors(spec, g, mon.astype(np.complex128))
    assert _rel(got, want) < 1e-6


# ------------------------------------------------------------------ forward
@pytest.mark.parametrize("kernel", list(KERNELS))
@pytest.mark.parametrize("name", ["cfg1"] + list(RAGGED))
def test_forward_matches_oracle(name, kernel):
    spec = zone_cfg1() if name == "cfg1" else RAGGED[name]
    rho = rho_for(spec, 1)
    z = _zone(spec, kernel)
    S = z.forward(_dev(rho))
    mon, des, st, S_ref = _oracle_forward_state(spec, rho)
    assert _rel(z.monitor_dft().cpu().numpy(), mon) < FIELD_TOL
    got_des = np.moveaxis(z.design_dft(0).cpu().numpy(), 4, 2)        # -> [q][c][k][i][j]
    assert _rel(got_des, des) < FIELD_TOL
    assert _rel(z.fields().cpu().numpy(), st[:6]) < FIELD_TOL
    assert _rel(S, S_ref) < FIELD_TOL


@pytest.mark.parametrize("value", [0.0, 1.0])
def test_forward_uniform_density(value):
    """Degenerate designs: rho = 0 (air layer) and rho = 1 (solid TiO2)."""
    spec = RAGGED["tiny"]
    rho = np.full((spec.n_r_design, spec.n_phi), value)
    z = _zone(spec)
    S = z.forward(_dev(rho))
    _, _, _, S_ref = _oracle_forward_state(spec, rho)
    assert _rel(S, S_ref) < FIELD_TOL


@pytest.mark.parametrize("kernel", ["fused2", "fused4", "split1", "tile4", "tile8", "tile16", "etile8", "etile16",
                                    "etile32", "htile8", "htile16", "htile32"])
def test_fused_step_equals_split_step(kernel):
    """The fused single-launch step and the split H/E launches compute the
    same scheme: fields and DFTs agree to FP32 rounding on the wide-zone grid
    (400 steps, all CTAs, CPML slabs, phi wrap, ragged radius ranges)."""
    spec = zone_cfg2(n_steps=400).replace(pulse_t0=0.05, source_k=38, monitor_k=54)
    rho = _dev(rho_for(spec, 2))
    a = _zone(spec, "split")
    b = _zone(spec, kernel)
    Sa, Sb = a.forward(rho), b.forward(rho)
    assert np.abs(a.fields().cpu().numpy()).max() > 0
    assert _rel(b.fields().cpu().numpy(), a.fields().cpu().numpy()) < 1e-6
    assert _rel(b.design_dft(0).cpu().numpy(), a.design_dft(0).cpu().numpy()) < 1e-6
    assert _rel(Sb, Sa) < 1e-6


def test_forward_is_deterministic():
    spec = RAGGED["ragged"]
    z = _zone(spec)
    r = _dev(rho_for(spec, 3))
    a = z.forward(r)
    fa = z.fields().cpu()
    b = z.forward(r)
    assert np.array_equal(a, b) and torch.equal(fa, z.fields().cpu())


@pytest.mark.parametrize("kernel", ["split", "split1", "fused2"])
def test_event_timing_samples_each_launch_of_a_step(kernel):
    spec = RAGGED["ragged_even"]
    z = _zone(spec, kernel)
    z.set_timing(10)
    z.forward(_dev(rho_for(spec, 3)))
    ms, n = z.timing()
    z.set_timing(0)
    assert n == (spec.n_steps + 9) // 10
    used = {"split": [0, 1, 2], "split1": [0, 1], "fused2": [0, 2]}[kernel]   # launches of a step
    assert all(ms[u] > 0 for u in used)
    assert z.timing() == ([0.0, 0.0, 0.0], 0)             # reset by the read


# ------------------------------------------------------------------ adjoint
GRAD_SPECS = {
    "tiny2": zone_tiny(n_steps=700, filter_radius=0.25, beta=4.0, wavelengths=(0.9, 1.1),
                       pulse_sigma=0.4, pulse_t0=1.6),
    "ragged3": RAGGED["ragged_even"].replace(n_steps=500),
    "ragged_tile3": RAGGED["ragged_tile"].replace(n_steps=500),
}


@pytest.mark.parametrize("kernel", ["split", "split1", "fused2", "fused4", "tile8", "tile4", "tile8_r5", "etile16",
                                    "etile8", "etile16_r7", "htile16", "htile8", "htile16_r7"])
@pytest.mark.parametrize("name", list(GRAD_SPECS))
def test_gradient_matches_oracle(name, kernel):
    spec = GRAD_SPECS[name]
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 5, mode="minmax")
    z = _zone(spec, kernel)
    S = z.forward(_dev(rho))
    grad = z.adjoint(4.0 * S).cpu().numpy()
    I_ref, g_ref, fwd, adj = O.gradient(spec, rho)
    assert _rel(S, fwd["S"]) < FIELD_TOL
    got_adj = np.moveaxis(z.design_dft(1).cpu().numpy(), 4, 2)
    assert _rel(got_adj, adj["des_adj"]) < GRAD_TOL
    assert _rel(grad, g_ref) < GRAD_TOL


def test_autograd_function_and_iteration_agree():
    from paper_2501_07979_gb300 import zone_focal
    spec = GRAD_SPECS["tiny2"]
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 5, mode="minmax")
    z = _zone(spec)
    r = _dev(rho).requires_grad_(True)
    S = zone_focal(r, z)
    I = 2.0 * (S ** 2).sum()
    I.backward()
    I_it, g_it = z.iteration(_dev(rho))
    I_h, g_h = z.iteration(torch.tensor(rho, dtype=torch.float32), host=True)
    I_ref, g_ref, _, _ = O.gradient(spec, rho)
    assert abs(I.item() - I_ref) / I_ref < FIELD_TOL
    assert abs(I_it - I_ref) / I_ref < FIELD_TOL and I_h == I_it
    assert _rel(r.grad.cpu().numpy(), g_ref) < GRAD_TOL
    assert torch.equal(g_it.cpu(), r.grad.cpu()) and torch.equal(g_h, g_it.cpu())


def test_objective_of_phasors_other_than_intensity():
    """The backward accepts any dI/dS: here f = |S_0|^2 only."""
    from paper_2501_07979_gb300 import zone_focal
    spec = GRAD_SPECS["tiny2"]
    rho = smoothed_rho(spec.n_r_design, spec.n_phi, 6, mode="minmax")
    z = _zone(spec)
    r = _dev(rho).requires_grad_(True)
    S = zone_focal(r, z)
    (S[0] ** 2).sum().backward()
    fwd = O.forward(spec, rho)
    fwd["rho"] = rho
    g = np.zeros(fwd["S"].shape, complex)
    g[0] = 2 * fwd["S"][0]
    adj = O.adjoint(spec, fwd, g)
    geom = fwd["geom"]
    rbar = O.conic_filter(spec, geom, rho)
    g_ref = O.conic_filter_T(spec, geom, adj["grad_rho_tilde"] * O.project_grad(spec, rbar))
    assert _rel(r.grad.cpu().numpy(), g_ref) < GRAD_TOL


# ------------------------------------------------------------------ full size
def _rings(spec, seed):
    """Seeded axisymmetric (phi-invariant) density: smoothed random rings."""
    from scipy.ndimage import gaussian_filter1d
    rng = np.random.default_rng(seed)
    f = gaussian_filter1d(rng.random(spec.n_r_design), 2.0, mode="reflect")
    f = (f - f.min()) / (f.max() - f.min())
    return np.repeat(f[:, None], spec.n_phi, axis=1)


@pytest.mark.parametrize("n_steps", [20000])
def test_wide_zone_full_size_against_one_cell_wedge(n_steps):
    """Full-size wide zone (300x320x160, 3 wavelengths, filter + projection,
    the benchmark's launch configuration and step count) with a
    phi-invariant ring density.  Its solution is the single Bloch mode
    e^{i phi}: the 320-cell wedge equals a 1-cell wedge of the same dphi
    (n_fold = 4000 * 320), which the oracle runs in full.  Compared element
    by element: monitor and design DFTs (times e^{i phi_j}), focal phasors,
    and the gradient (the 1-cell pixel gradient is the sum over the 320
    pixels of a ring, each equal by symmetry)."""
    spec = zone_cfg2(n_steps=n_steps)
    rho = _rings(spec, 12)
    z = _zone(spec)
    S = z.forward(_dev(rho))
    mon = z.monitor_dft().cpu().numpy()
    des = np.moveaxis(z.design_dft(0).cpu().numpy(), 4, 2)
    grad = z.adjoint(4.0 * S).cpu().numpy()
    one = spec.replace(n_phi=1, n_fold=spec.n_fold * spec.n_phi)
    I1, g1, f1, _ = O.gradient(one, rho[:, :1])
    g = O.Geometry(spec)
    shift = np.exp(1j * g.phi_n)          # cell j is cell 0 rotated by j dphi
    mon_ref = f1["mon"] * shift
    assert _rel(mon, mon_ref) < FIELD_TOL
    des_ref = f1["des"] * shift
    assert _rel(des, des_ref) < FIELD_TOL
    assert _rel(S, f1["S"]) < FIELD_TOL
    assert _rel(grad, np.repeat(g1 / spec.n_phi, spec.n_phi, axis=1)) < GRAD_TOL


@pytest.mark.parametrize("kernel", ["split", "tile4", "etile16", "htile16"])
def test_wide_zone_full_size_phi_varying_against_oracle(kernel):
    """The full 300x320x160 wide-zone grid with its seeded, phi-varying
    density (filter + projection, 3 wavelengths), 300 steps with the sheet
    source two cells below the design layer and the monitor inside it (so
    that the fields reach both within the run): final fields, monitor and
    design-volume DFTs and focal phasors element by element against the FP64
    oracle.  Every phi-coupling path at full size is exercised: the Bloch
    wrap of the 320th row, phi-neighbour loads, filter taps across the wrap."""
    spec = zone_cfg2(n_steps=300).replace(pulse_t0=0.05, source_k=38, monitor_k=42)
    rho = rho_for(spec, 2)
    z = _zone(spec, kernel)
    S = z.forward(_dev(rho))
    mon, des, st, S_ref = _oracle_forward_state(spec, rho)
    assert np.abs(mon).max() > 0 and np.abs(des).max() > 0
    assert _rel(z.monitor_dft().cpu().numpy(), mon) < FIELD_TOL
    got_des = np.moveaxis(z.design_dft(0).cpu().numpy(), 4, 2)
    assert _rel(got_des, des) < FIELD_TOL
    f = z.fields().cpu().numpy()
    num = sum(float(np.linalg.norm((f[c] - st[c]).ravel())) ** 2 for c in range(6))
    den = sum(float(np.linalg.norm(st[c].ravel())) ** 2 for c in range(6))
    assert (num / den) ** 0.5 < FIELD_TOL                # the six components together, as the other forward checks
    assert _rel(S, S_ref) < FIELD_TOL


# ------------------------------------------------------------------ axis zone
AXIS = zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_steps=700, filter_radius=0.25, beta=4.0,
                 wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6)


def test_axis_zone_forward_and_gradient_match_oracle():
    """Continuous axisymmetry with the axis inside (the innermost zone of a
    lens): forward DFTs, fields, phasors and the adjoint gradient."""
    spec = AXIS
    rho = smoothed_rho(spec.n_r_design, 1, 8, mode="minmax")
    z = _zone(spec)
    assert z.get_kernel()[0] == 0                      # split step
    S = z.forward(_dev(rho))
    mon, des, st, S_ref = _oracle_forward_state(spec, rho)
    assert _rel(z.monitor_dft().cpu().numpy(), mon) < FIELD_TOL
    assert _rel(np.moveaxis(z.design_dft(0).cpu().numpy(), 4, 2), des) < FIELD_TOL
    assert _rel(z.fields().cpu().numpy(), st[:6]) < FIELD_TOL
    assert _rel(S, S_ref) < FIELD_TOL
    grad = z.adjoint(4.0 * S).cpu().numpy()
    _, g_ref, _, _ = O.gradient(spec, rho)
    assert _rel(grad, g_ref) < GRAD_TOL


# ------------------------------------------------------------------ errors
def test_adjoint_before_forward_is_a_state_error():
    from paper_2501_07979_gb300 import ZdaError
    spec = RAGGED["tiny"]
    z = _zone(spec)
    with pytest.raises(ZdaError, match="ZDA_ERR_STATE"):
        z.adjoint(np.ones(z.n_freq, complex))


@pytest.mark.parametrize("kernel,name", [("fused2", "tiny"), ("tile4", "ragged_tile"), ("etile16", "ragged_tile"),
                                         ("htile16", "ragged_tile")])
def test_fused_wait_timeout_is_reported_and_context_survives(kernel, name):
    """The fused and tiled steps' barrier waits are bounded: with a barrier
    that nothing completes and a short limit the call returns ZDA_ERR_TIMEOUT
    instead of hanging, and the same zone then runs normally."""
    from paper_2501_07979_gb300 import ZdaError
    spec = RAGGED[name].replace(n_steps=3)
    z = _zone(spec, kernel)
    r = _dev(rho_for(spec, 1))
    z.set_wait_limit(200, inject_timeout=True)
    with pytest.raises(ZdaError, match="ZDA_ERR_TIMEOUT"):
        z.forward(r)
    z.set_wait_limit(1 << 22, inject_timeout=False)
    S = z.forward(r)
    _, _, _, S_ref = _oracle_forward_state(spec, rho_for(spec, 1))
    assert np.all(np.isfinite(S)) and _rel(S, S_ref) < FIELD_TOL


def test_divergent_run_reports_nonfinite():
    """A near-zero permittivity makes the explicit scheme overflow: the run
    ends with ZDA_ERR_NONFINITE instead of returning garbage."""
    from paper_2501_07979_gb300 import ZdaError
    spec = RAGGED["tiny"].replace(layer_eps=(1e-9, 1e-9, 1e-9), n_steps=400)
    z = _zone(spec)
    with pytest.raises(ZdaError, match="ZDA_ERR_NONFINITE"):
        z.forward(_dev(np.zeros((spec.n_r_design, spec.n_phi))))


@pytest.mark.parametrize("which", ["wide", "lwir16"])
def test_autotuner_times_candidates_and_applies_the_fastest(tmp_path, which):
    from paper_2501_07979_gb300.autotune import tune_zone, candidates
    spec = zone_cfg2(n_steps=100) if which == "wide" else zone_lwir(16, 100)
    z = _zone(spec)
    cache = str(tmp_path / "tiles.json")
    choice, times = tune_zone(z, steps=8, cache_path=cache)
    print("tile tuner ms per 8 steps:", {c: round(t, 3) for c, t in times.items()})
    assert len(times) == len(candidates(spec)) and times[choice] == min(times.values())
    v, tj, _ = z.get_kernel()
    assert (v, tj) == choice[:2]
    z2 = _zone(spec)
    again, t2 = tune_zone(z2, cache_path=cache)           # cached: no timing
    assert again == choice and t2 == {}


# ------------------------------------------------------------------ lens (all zones, one graph)
def _lens_specs(n_zones=3):
    """An axis zone and annular zones of uneven width and fold (n_zones = 3
    or 8)."""
    base = dict(n_steps=500, filter_radius=0.2, beta=3.0, wavelengths=(0.9, 1.1), pulse_sigma=0.4,
                pulse_t0=1.6, focal=12.0)
    if n_zones == 3:
        return [zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_r=20, **base),
                zone_tiny(r_lo=1.2, n_fold=12, n_phi=6, n_r=24, **base),
                zone_tiny(r_lo=3.2, n_fold=24, n_phi=8, n_r=28, **base)]
    # interior widths 12, 16, 10, 22, 14, 18, 11, 20 cells (dr = 0.1), folds growing with radius
    widths = (12, 16, 10, 22, 14, 18, 11, 20)
    folds = (0, 12, 20, 27, 40, 44, 60, 66)
    phis = (1, 6, 4, 8, 5, 8, 6, 7)
    out, r = [], 0.0
    for w, n, p in zip(widths, folds, phis):
        if n == 0:
            out.append(zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_r=w + 4, **base))
        else:
            out.append(zone_tiny(r_lo=r - 0.4, n_fold=n, n_phi=p, n_r=w + 8, **base))
        r += 0.1 * w
    return out


@pytest.mark.parametrize("n_zones", [3, 8])
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("kernel", ["split", "fused2"])
def test_lens_equals_sum_of_zones_and_oracle(use_graph, kernel, n_zones):
    from paper_2501_07979_gb300.lens import Lens
    specs = _lens_specs(n_zones)
    rhos = [smoothed_rho(s.n_r_design, s.n_phi, 30 + z, mode="minmax") for z, s in enumerate(specs)]
    zones = [_zone(s) for s in specs]
    if kernel == "fused2":
        for z in zones[1:]:
            z.set_kernel(*KERNELS["fused2"])
    lens = Lens(zones, use_graph=use_graph)
    S = lens.forward([_dev(r) for r in rhos])
    per_zone = [lens.zone_focal(z) for z in range(len(zones))]
    assert _rel(S, sum(per_zone)) < 1e-12
    refs = [O.gradient(s, r) for s, r in zip(specs, rhos)]           # (I, g, fwd, adj) per zone
    S_ref = sum(f[2]["S"] for f in refs)
    assert _rel(S, S_ref) < FIELD_TOL
    g = 4.0 * S
    grads = lens.adjoint(g)
    for z, (s, r) in enumerate(zip(specs, rhos)):
        f = dict(refs[z][2])
        f["rho"] = r
        adj = O.adjoint(s, f, g)
        gm = f["geom"]
        g_ref = O.conic_filter_T(s, gm, adj["grad_rho_tilde"] * O.project_grad(s, O.conic_filter(s, gm, r)))
        assert _rel(grads[z].cpu().numpy(), g_ref) < GRAD_TOL
    # a second iteration replays the same graph with new densities
    n0 = lens.launches
    S2 = lens.forward([_dev(1.0 - r) for r in rhos])
    assert lens.launches == n0 + 1 and _rel(S2, S) > 1e-3
    assert _rel(S2, sum(lens.zone_focal(z) for z in range(len(zones)))) < 1e-12


def test_lens_focal_plane_matches_bruteforce_oracle():
    """Off-axis focal-plane field of a lens (axis zone + two wedge zones):
    the GPU's azimuthal-order +-1 quadrature against the oracle's brute-force
    sum over every site of the full circle; transmitted power likewise."""
    from paper_2501_07979_gb300.lens import Lens
    specs = _lens_specs()
    rhos = [smoothed_rho(s.n_r_design, s.n_phi, 40 + z, mode="minmax") for z, s in enumerate(specs)]
    zones = [_zone(s) for s in specs]
    lens = Lens(zones)
    lens.forward([_dev(r) for r in rhos])
    pts = [(0.0, 0.0), (0.4, 0.0), (0.0, 0.7), (1.1, -0.5), (2.0, 1.0)]
    ex, ey, pt = lens.focal_plane(pts, n_phi_samples=256)
    rx = ry = 0
    p_ref = 0
    for s, r in zip(specs, rhos):
        f = O.forward(s, r)
        a, b = O.focal_plane_bruteforce(s, f["geom"], f["mon"], pts)
        rx, ry = rx + a, ry + b
        p_ref = p_ref + O.transmitted_power(s, f["geom"], f["mon"])
    assert _rel(ex, rx) < 1e-4 and _rel(ey, ry) < 1e-4
    assert _rel(pt, p_ref) < 1e-4
    # off the focal plane (x, y, h): the xz-map path
    pts3 = [(0.0, 0.0, -2.0), (0.5, 0.0, 1.5), (1.0, 0.3, -0.5)]
    ex3, ey3 = lens.field_points(pts3, n_phi_samples=256)
    rx3 = ry3 = 0
    for s, r in zip(specs, rhos):
        f = O.forward(s, r)
        a, b = O.focal_plane_bruteforce(s, f["geom"], f["mon"], pts3)
        rx3, ry3 = rx3 + a, ry3 + b
    assert _rel(ex3, rx3) < 1e-4 and _rel(ey3, ry3) < 1e-4
    # the xz map (x, h grid through the axis) = the oracle's intensity of the brute-force field
    from paper_2501_07979_gb300.evaluate import xz_map
    xs, hs = [0.0, 0.6, 1.2], [-1.0, 0.8]
    M = xz_map(lens, xs, hs, n_top=1.2, n_phi_samples=256)
    grid = [(x, 0.0, h) for h in hs for x in xs]
    gx = gy = 0
    for s, r in zip(specs, rhos):
        f = O.forward(s, r)
        a, b = O.focal_plane_bruteforce(s, f["geom"], f["mon"], grid)
        gx, gy = gx + a, gy + b
    assert _rel(M, O.spot_intensity(gx, gy, 1.2).reshape(M.shape)) < 2e-4


def test_topopt_on_a_zone_increases_focal_intensity():
    from paper_2501_07979_gb300.topopt import TopOpt
    spec = GRAD_SPECS["tiny2"]
    z = _zone(spec)
    rho0 = smoothed_rho(spec.n_r_design, spec.n_phi, 5, mode="minmax")

    def vg(rhos):
        I, g = z.iteration(_dev(rhos[0]))
        return I, [g.cpu().numpy()]

    opt = TopOpt(vg, [rho0], lr=0.05, set_beta=z.set_projection, schedule=lambda it: 4.0)
    hist = opt.run(6)
    assert hist[-1]["objective"] > 1.2 * hist[0]["objective"]


def _eval_specs():
    """Three zones of a small lens whose folds keep the azimuthal orders the
    focal-plane transform neglects below 1e-3 at every evaluated point (an
    axis zone, then n = 64 and n = 128 wedges), each run for ~12 lambda/c."""
    base = dict(filter_radius=0.2, beta=3.0, wavelengths=(0.9, 1.1), pulse_sigma=0.4, pulse_t0=1.6,
                focal=12.0)
    specs = [zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_r=20, **base),
             zone_tiny(r_lo=1.2, n_fold=64, n_phi=6, n_r=24, **base),
             zone_tiny(r_lo=3.2, n_fold=128, n_phi=8, n_r=28, **base)]
    return [s.replace(n_steps=int(math.ceil(12.0 / O.Geometry(s).dt))) for s in specs]


def _oracle_evaluation(specs, rhos, lens_radius, xs, pts_disc, inc):
    """FE, relative FE, transmittance and Strehl built from the oracle's
    brute-force focal-plane field (every site of every wedge copy, all
    azimuthal orders) and its transmitted power, with the same quadrature as
    the library's evaluation."""
    fw = [O.forward(s, r) for s, r in zip(specs, rhos)]
    line = [O.focal_plane_bruteforce(s, f["geom"], f["mon"], np.stack([xs, 0 * xs], 1)) for s, f in zip(specs, fw)]
    ex = sum(a for a, _ in line)
    ey = sum(b for _, b in line)
    pt = sum(O.transmitted_power(s, f["geom"], f["mon"]) for s, f in zip(specs, fw))
    I_line = O.spot_intensity(ex, ey)
    lam = np.asarray(specs[0].wavelengths)
    out = []
    for l, (rr, pts) in enumerate(pts_disc):
        d = [O.focal_plane_bruteforce(s, f["geom"], f["mon"], pts) for s, f in zip(specs, fw)]
        Id = O.spot_intensity(sum(a for a, _ in d)[l], sum(b for _, b in d)[l]).reshape(len(rr), -1)
        p_disc = float(np.sum(Id.mean(axis=1) * 2 * math.pi * rr) * (rr[1] - rr[0]))
        area = math.pi * lens_radius ** 2
        out.append({"fwhm": O.fwhm(xs, I_line[l]), "focusing_efficiency": p_disc / (inc[l] * area),
                    "relative_efficiency": p_disc / pt[l], "transmittance": pt[l] / (inc[l] * area),
                    "strehl": float(I_line[l, 0] * lam[l] ** 2 * specs[0].focal ** 2 / (pt[l] * area))})
    return out


def test_field_intensity_and_encircled_power_match_oracle():
    """The library's intensity of field samples and its encircled power
    (trapezoid rule) against the oracle's on seeded random inputs."""
    import ctypes
    from paper_2501_07979_gb300 import _lib
    from paper_2501_07979_gb300.evaluate import encircled_power
    rng = np.random.default_rng(7)
    nl, n = 3, 257
    f = rng.standard_normal((2, nl, n, 2))
    field = torch.tensor(f, dtype=torch.float64, device="cuda:0")
    out = torch.empty((nl, n), dtype=torch.float64, device="cuda:0")
    rc = _lib.lib().zda_field_intensity(ctypes.c_void_p(field.data_ptr()), nl, n, 1.5, ctypes.c_void_p(out.data_ptr()),
                                        None)
    assert rc == 0
    ex, ey = f[0, ..., 0] + 1j * f[0, ..., 1], f[1, ..., 0] + 1j * f[1, ..., 1]
    assert np.allclose(out.cpu().numpy(), O.spot_intensity(ex, ey, 1.5), rtol=1e-14, atol=0)
    r = np.sort(rng.uniform(0, 3, 101))
    I = rng.uniform(0, 1, (4, 101))
    got = encircled_power(r, I)
    want = np.array([O.encircled_power(r, I[q]) for q in range(4)])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-14)
    assert np.allclose(encircled_power(r, I[1]), want[1], rtol=1e-12, atol=1e-14)


def test_lens_evaluation_matches_bruteforce_oracle():
    """Focusing efficiency (absolute, relative), transmittance, FWHM and the
    Strehl ratio (Eq. 9) of a three-zone lens against the same quantities
    built from the oracle's brute-force focal-plane field, on zones whose
    neglected azimuthal orders stay below 1e-3 of the kept ones (checked)."""
    import warnings
    from paper_2501_07979_gb300.evaluate import evaluate_lens, incident_intensity
    from paper_2501_07979_gb300.lens import Lens
    specs = _eval_specs()
    rhos = [smoothed_rho(s.n_r_design, s.n_phi, 50 + z, mode="minmax") for z, s in enumerate(specs)]
    lens = Lens([_zone(s) for s in specs])
    lens.forward([_dev(r) for r in rhos])
    inc = incident_intensity(specs[1])
    R = specs[-1].r_lo + (specs[-1].n_r - specs[-1].pml_r_out) * specs[-1].dr
    with warnings.catch_warnings():
        warnings.simplefilter("error")                 # no order-bound warning may be raised
        res, xs, I = evaluate_lens(lens, R, specs[0].focal, inc, n_rad=16, n_ang=4)
    n_rad, n_ang = 16, 4
    discs = []
    for r in res:
        assert r["order_bound"] < 1e-3, r["order_bound"]
        rmax = 3.0 * r["fwhm"]
        rr = (np.arange(n_rad) + 0.5) * rmax / n_rad
        aa = 2 * math.pi * np.arange(n_ang) / n_ang
        discs.append((rr, np.array([(q * math.cos(a), q * math.sin(a)) for q in rr for a in aa])))
    # incident plane-wave intensity: the oracle's reference run (substrate everywhere)
    s1 = specs[1]
    es = float(s1.layer_eps[0])
    ref_spec = s1.replace(layer_eps=tuple(es for _ in s1.layer_eps), eps_lo=es, eps_hi=es, filter_radius=0.0,
                          beta=0.0)
    f_inc = O.forward(ref_spec, np.zeros((ref_spec.n_r_design, ref_spec.n_phi)))
    g1 = f_inc["geom"]
    nl = g1.n_lambda
    i0, i1 = ref_spec.pml_r_in, ref_spec.n_r - ref_spec.pml_r_out
    inc_ref = np.array([0.5 * math.sqrt(es) * abs(2 * (f_inc["mon"][l, 0, i0:i1] * np.exp(-1j * g1.phi_n)[None, :]).mean()) ** 2
                        for l in range(nl)])
    assert _rel(inc, inc_ref) < 1e-4
    ref = _oracle_evaluation(specs, rhos, R, xs, discs, inc_ref)
    for got, want in zip(res, ref):
        assert abs(got["fwhm"] / want["fwhm"] - 1) < 1e-3
        for key in ("focusing_efficiency", "relative_efficiency", "transmittance", "strehl"):
            assert abs(got[key] / want[key] - 1) < 1e-3, (key, got[key], want[key])
        assert abs(got["focusing_efficiency"] - got["transmittance"] * got["relative_efficiency"]) < 1e-12
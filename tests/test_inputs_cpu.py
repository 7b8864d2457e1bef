"""The workload descriptions: JSON round trip of every zone factory, and the
seeded density generator's determinism and range."""
import numpy as np

from zda_inputs import (ZoneSpec, zone_cfg1, zone_cfg2, zone_lwir, zone_tiny, zone_visible, smoothed_rho,
                        lens_zones)


def test_zone_specs_round_trip_through_json():
    specs = [zone_cfg1(), zone_cfg2(100), zone_tiny(), zone_lwir(16, 100), zone_visible(16, "rgb", 100),
             zone_visible(16, "poly", 100)] + list(lens_zones()[:3])
    for s in specs:
        back = ZoneSpec.from_json(s.to_json())
        assert back == s
        assert hash(back) == hash(s)


def test_smoothed_density_is_seeded_and_in_range():
    a = smoothed_rho(20, 12, 5, mode="minmax")
    b = smoothed_rho(20, 12, 5, mode="minmax")
    c = smoothed_rho(20, 12, 6, mode="minmax")
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() == 0.0 and a.max() == 1.0
    d = smoothed_rho(20, 12, 5, mode="binary")
    assert set(np.unique(d)) <= {0.0, 1.0}


def test_bench_whole_step_fractions():
    """bench.py's whole-step roofline figures: 96 B per cell-update against
    the peak, and the step kernels' bytes over their time (the DFT flush
    counted once per 32 steps)."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    kernels = [("k_tile_e", 1.2e9, 0.2), ("k_update_h_pair", 1.2e9, 0.2), ("k_dft_flush", 3.2e9, 0.4)]
    per_step = {"k_tile_e": 0.2, "k_update_h_pair": 0.2, "k_dft_flush": 0.4 / 32}
    w = bench.whole_step(40.0, 6000.0, kernels, per_step)
    assert abs(w["frac_96B"] - 40.0 * 96 / 6000.0) < 1e-15
    assert abs(w["algorithmic_bytes_per_step"] - (2.4e9 + 1e8)) < 1.0
    assert abs(w["kernel_ms_per_step"] - 0.4125) < 1e-12
    assert abs(w["frac_step_bytes"] - 2.5e9 / 0.4125e-3 / 1e9 / 6000.0) < 1e-12


def test_tuner_candidates_follow_the_kernels_constraints():
    """The tile kernels (variants 3-5) are offered only where they run
    (annular zone, even n_z and z-PML); the split step's block shapes never
    exceed twice the phi cells; the wide zone gets every family."""
    from paper_2501_07979_gb300.autotune import candidates
    from zda_inputs import zone_cfg2, zone_tiny
    wide = candidates(zone_cfg2(n_steps=10))
    fams = {v for v, _, _ in wide}
    assert fams == {0, 1, 2, 3, 4, 5}
    assert {(4, 16, 0), (5, 16, 0), (3, 4, 0)} <= set(wide)
    axis = candidates(zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0))
    assert all(v in (0, 2) for v, _, _ in axis)
    odd = candidates(zone_tiny(n_z=45))
    assert all(v not in (3, 4, 5) for v, _, _ in odd)
    narrow = candidates(zone_tiny(n_phi=3))
    assert all(t <= 6 for v, t, _ in narrow if v in (0, 3, 4, 5))

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

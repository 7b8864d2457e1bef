"""zda_zone_order_bound (host only): the estimate of the azimuthal orders that
the off-axis lens-field transform neglects (reading: only the orders +-1 of
each zone's near field are propagated; the wedge's orders m + j n reach a
point through J_L(k r rho / z_f) with abs(L) >= n - 2).  Checked against
scipy's Bessel functions, which the bound must dominate, and its limits."""
import math

import numpy as np
import pytest

from zda_inputs import zone_tiny, zone_lwir

scipy_special = pytest.importorskip("scipy.special")


def _x(spec, rho, h=0.0):
    k = 2 * math.pi * math.sqrt(spec.layer_eps[-1]) / min(spec.wavelengths)
    r_hi = spec.r_lo + spec.n_r * spec.dr
    zf = spec.focal - (spec.monitor_k - spec.design_k1) * spec.dz + h
    return k * r_hi * rho / zf


@pytest.mark.parametrize("n_fold", [6, 12, 24, 40])
def test_bound_dominates_the_bessel_function(n_fold):
    from paper_2501_07979_gb300.lens import order_bound
    spec = zone_tiny(n_fold=n_fold, r_lo=1.2, focal=12.0)
    nu = n_fold - 2
    for rho in (0.1, 0.5, 1.0, 2.0, 4.0):
        b = order_bound(spec, [(rho / math.sqrt(2), rho / math.sqrt(2))])
        x = _x(spec, rho)
        assert b >= abs(scipy_special.jv(nu, x)) * (1 - 1e-12)
        assert b == pytest.approx((x / 2) ** nu / math.gamma(nu + 1), rel=1e-9)


def test_bound_limits():
    from paper_2501_07979_gb300.lens import order_bound
    spec = zone_tiny(n_fold=24, r_lo=3.2, focal=12.0)
    assert order_bound(spec, [(0.0, 0.0)]) == 0.0                       # on the axis: nothing neglected
    axis = zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0)
    assert order_bound(axis, [(3.0, 1.0)]) == 0.0                       # continuous axisymmetry
    zf = spec.focal - (spec.monitor_k - spec.design_k1) * spec.dz
    assert math.isinf(order_bound(spec, [(0.5, 0.0, -zf - 0.1)]))       # below the monitor plane
    far = order_bound(spec, [(1.0, 0.0), (3.0, 0.0)])
    assert far == order_bound(spec, [(3.0, 0.0)]) > order_bound(spec, [(1.0, 0.0)])   # max over points
    # closer to the focal plane from above: larger z_f, smaller bound
    assert order_bound(spec, [(1.0, 0.0, 2.0)]) < order_bound(spec, [(1.0, 0.0, 0.0)])


def test_paper_zones_neglect_nothing_measurable():
    """LWIR zone 2 (n = 1440, the smallest fold of the wedge zones) at 10
    lambda off axis in the focal plane: the bound underflows to 0."""
    from paper_2501_07979_gb300.lens import order_bound
    assert order_bound(zone_lwir(2, 10), [(10.0, 0.0)]) < 1e-300

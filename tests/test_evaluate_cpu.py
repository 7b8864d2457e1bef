"""Focal-spot analysis helpers on CPU: encircled power of closed-form
spots, FWHM of a Gaussian."""
import math

import numpy as np

from paper_2501_07979_gb300.evaluate import encircled_power, fwhm


def test_encircled_power_of_a_uniform_disk_and_a_gaussian():
    r = np.linspace(0, 2, 2001)
    P = encircled_power(r, np.where(r <= 1.0, 1.0, 0.0))
    assert abs(P[-1] - math.pi) < 5e-3                       # pi * 1^2 (edge sampled at dr = 1e-3)
    s = 0.3
    Pg = encircled_power(r, np.exp(-r ** 2 / (2 * s * s)))
    exact = 2 * math.pi * s * s * (1 - np.exp(-r ** 2 / (2 * s * s)))
    assert np.max(np.abs(Pg - exact)) < 1e-6


def test_fwhm_of_a_gaussian():
    xs = np.linspace(0, 2, 2001)                  # profile from the peak outwards
    s = 0.25
    assert abs(fwhm(xs, np.exp(-xs ** 2 / (2 * s * s))) - 2 * math.sqrt(2 * math.log(2)) * s) < 1e-5

"""Pins of the jet's evaluation quantities (Section 3.3) computed by the
oracle from time-averaged fields: exact fields with known widths."""
import math

import numpy as np
import pytest

from oracle.jetstats import jet_fit, radial_profile

N = 96                 # cross-section of level 0 (cells)
Y0 = Z0 = 48.3         # axis off the cell lattice (no ring-boundary ties)


def field(fn, nx=4):
    y = np.arange(N) + 0.5
    r = np.sqrt((y[None, :] - Y0) ** 2 + (y[:, None] - Z0) ** 2)
    m = fn(r)
    return np.repeat(m[:, :, None], nx, axis=2)


def test_gaussian_profile_gives_its_width_and_unit_fit():
    """u = U exp(-(r / b)^2): the half width at u_m / e is b, and the
    Gaussian fit returns a = 1, c = 1 (up to the averaging over rings one
    cell wide)."""
    U, b = 0.05, 9.0
    mean = field(lambda r: U * np.exp(-(r / b) ** 2))
    var = np.zeros_like(mean)
    pm, pv, pc = radial_profile(mean, var, 0, Y0, Z0, 1.0, 40, [1.5])
    um, be, ti, a, c = jet_fit(pm[0], pv[0], pc[0], 1.0)
    assert abs(um - U) <= 0.01 * U              # ring 0 averages r < 1
    assert abs(be - b) <= 0.01 * b
    assert ti == 0.0
    assert abs(a - 1.0) <= 0.02 and abs(c - 1.0) <= 0.03


def test_parabolic_profile_half_width_closed_form():
    """u = U (1 - r^2 / R^2): u = U / e at r = R sqrt(1 - 1/e)."""
    U, R = 0.04, 30.0
    mean = field(lambda r: np.where(r < R, U * (1 - (r / R) ** 2), 0.0))
    pm, pv, pc = radial_profile(mean, np.zeros_like(mean), 0, Y0, Z0, 0.5, 80, [0.2])
    _, be, _, _, _ = jet_fit(pm[0], pv[0], pc[0], 0.5)
    assert abs(be - R * math.sqrt(1 - 1 / math.e)) <= 0.01 * R


def test_uniform_field_rings_counts_and_intensity():
    """A uniform mean and variance: every ring holds them; the ring counts add
    up to the cells within nbins * dr; tI = sqrt(var) / u."""
    mean = field(lambda r: np.full_like(r, 0.03))
    var = field(lambda r: np.full_like(r, 4e-6))
    mean[:, :5, :] = np.nan                      # cells without a value are skipped
    pm, pv, pc = radial_profile(mean, var, 0, Y0, Z0, 1.3, 20, [0.5, 2.7])
    y = np.arange(N) + 0.5
    r = np.sqrt((y[None, :] - Y0) ** 2 + (y[:, None] - Z0) ** 2)
    for s in range(2):
        ok = pc[s] > 0
        assert np.allclose(pm[s][ok], 0.03, rtol=0, atol=1e-15)
        # the NaN rows are y < 5 in the field above (axis order z, y)
        expect = int(((r < 20 * 1.3) & (np.arange(N)[None, :] >= 5)).sum())
        assert int(pc[s].sum()) == expect
        um, be, ti, a, c = jet_fit(pm[s], pv[s], pc[s], 1.3)
        assert abs(ti - math.sqrt(4e-6) / 0.03) <= 1e-12
        assert math.isnan(be)

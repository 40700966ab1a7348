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


def test_levels_profile_reduces_to_one_level_and_weights_by_area():
    """Over all levels: rings that lie in one level's active cells give that
    level's plain average; a uniform field gives the uniform value
    everywhere; a field 1 on level-0 cells and 3 on level-1 cells gives, in
    a ring whose cells are all on one level, 1 or 3, and in between the
    area-weighted value (level-1 cells count a quarter)."""
    from oracle.jetstats import radial_profile_levels
    N0 = 32
    act0 = np.ones((N0, N0, 4), dtype=bool)
    act0[8:24, 8:24, :] = False                      # refined square in the middle
    act1 = np.zeros((2 * N0, 2 * N0, 8), dtype=bool)
    act1[16:48, 16:48, :] = True
    one = lambda a, v: np.where(a, v, np.nan)
    lv = [(one(act0, 1.0), one(act0, 0.0), act0), (one(act1, 3.0), one(act1, 0.0), act1)]
    y0 = z0 = 16.2
    pm, pv, pc = radial_profile_levels(lv, y0, z0, 1.0, 22, [1.3])
    inner = np.arange(22) < 7          # r < 7: only fine cells (square of half side 8)
    outer = np.arange(22) >= 12        # r >= 12 (> 8 sqrt 2): only coarse cells
    ok = pc[0] > 0
    assert np.allclose(pm[0][inner & ok], 3.0, atol=1e-15)
    assert np.allclose(pm[0][outer & ok], 1.0, atol=1e-15)
    mid = ok & ~inner & ~outer
    assert ((pm[0][mid] > 1.0) & (pm[0][mid] < 3.0)).any()
    # mixed rings: (n0 * 1 + n1 / 4 * 3) / (n0 + n1 / 4) with n_l the active
    # cells of level l whose centre lies in the ring (counted on the grids)
    c0 = np.arange(N0) + 0.5
    c1 = (np.arange(2 * N0) + 0.5) / 2
    r0 = np.sqrt((c0[None, :] - y0) ** 2 + (c0[:, None] - z0) ** 2)
    r1 = np.sqrt((c1[None, :] - y0) ** 2 + (c1[:, None] - z0) ** 2)
    for b in np.nonzero(mid)[0]:
        n0 = int((act0[:, :, 1] & (np.floor(r0) == b)).sum())
        n1 = int((act1[:, :, 2] & (np.floor(r1) == b)).sum())
        assert abs(pm[0][b] - (n0 + 0.75 * n1) / (n0 + 0.25 * n1)) <= 1e-14
    # the same rings from the fine level alone (plain averages) where it holds them
    pf, _, cf = radial_profile(one(act1, 3.0), one(act1, 0.0), 1, y0, z0, 1.0, 22, [1.3])
    assert np.array_equal(cf[0][inner], pc[0][inner])
    # a uniform field is uniform whatever the split
    lu = [(one(act0, 0.02), one(act0, 1e-6), act0), (one(act1, 0.02), one(act1, 1e-6), act1)]
    um, uv, uc = radial_profile_levels(lu, y0, z0, 1.0, 22, [1.3])
    assert np.allclose(um[0][uc[0] > 0], 0.02, rtol=1e-14)
    assert np.allclose(uv[0][uc[0] > 0], 1e-6, rtol=1e-12)

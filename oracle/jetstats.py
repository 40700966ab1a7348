"""The jet's evaluation quantities of Section 3.3 from time-averaged fields:
radial profiles on cross-sections, the centreline velocity u_m, the
spreading (half) width where the mean axial velocity falls to u_m / e
(0.368 u_m, the isoline the paper's spreading function uses), the
turbulence intensity sqrt(<u_x'^2>) / u_m on the axis and a Gaussian fit of
the radial profile (the paper compares with u_x / u_m = 0.938 exp(-0.944
(r / r_e)^2)).

Test infrastructure: the plain statement the CUDA path is checked against.

Reading (the paper gives the quantities, not how they are sampled):
* ring b of a station holds the cells of the level-l layer containing x
  (coarse units) whose centre lies at r in [b dr, (b + 1) dr) from the axis
  (y0, z0); its values are plain averages over those cells of the time mean
  of u_x and of the time variance of u_x;
* over all levels of a nested grid, the unrefined (active) cells of every
  level in its layer containing x enter, each weighted by its cross-section
  area 4^-l (the active cells of all levels tile the plane x = const), and
  a ring's values are area-weighted averages;
* u_m is the value of ring 0; the half width b_e interpolates linearly
  between the centres (b + 1/2) dr of the first ring (b >= 1) at or below
  u_m / e and the ring before it;
* tI = sqrt(max(var_0, 0)) / u_m;
* the Gaussian fit is the least-squares line through (X, Y) = ((r_b / b_e)^2,
  ln(u_b / u_m)) over the rings with cells, u_b >= 0.05 u_m and r_b <= 2 b_e:
  u / u_m = a exp(-c (r / b_e)^2).
"""
import math

import numpy as np


def _rings(parts, y0, z0, dr, nbins, x_stations):
    """Weighted ring sums over parts = [(level, mean, var, use, weight)]:
    mean, var (NZ, NY, NX) of that level, use a boolean mask of the cells
    that enter."""
    ns = len(x_stations)
    sm = np.zeros((ns, nbins))
    sv = np.zeros((ns, nbins))
    sw = np.zeros((ns, nbins))
    cnt = np.zeros((ns, nbins), dtype=np.int64)
    for level, mean_ux, var_ux, use, w in parts:
        s = 2.0 ** -level
        NZ, NY, NX = mean_ux.shape
        for si, xs in enumerate(x_stations):
            X = int(math.floor(xs * 2 ** level))
            if not 0 <= X < NX:
                raise ValueError("station outside the level")
            for z in range(NZ):
                for y in range(NY):
                    if not use[z, y, X]:
                        continue
                    dy = (y + 0.5) * s - y0
                    dz = (z + 0.5) * s - z0
                    b = int(math.floor(math.sqrt(dy * dy + dz * dz) / dr))
                    if b >= nbins:
                        continue
                    sm[si, b] += w * mean_ux[z, y, X]
                    sv[si, b] += w * var_ux[z, y, X]
                    sw[si, b] += w
                    cnt[si, b] += 1
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(cnt > 0, sm / sw, np.nan), np.where(cnt > 0, sv / sw, np.nan), cnt


def radial_profile(mean_ux, var_ux, level, y0, z0, dr, nbins, x_stations):
    """Ring averages of the time mean and variance of u_x on one level.

    mean_ux, var_ux: (NZ, NY, NX) of level `level`, NaN where the level holds
    no value.  Returns (mean[s][b], var[s][b], counts[s][b]); NaN for empty
    rings."""
    return _rings([(level, mean_ux, var_ux, ~np.isnan(mean_ux), 1.0)], y0, z0, dr, nbins, x_stations)


def radial_profile_levels(levels, y0, z0, dr, nbins, x_stations):
    """Area-weighted ring averages over every level of a nested grid.

    levels: [(mean_ux, var_ux, active)] per level l = 0, 1, ..., with active
    the (NZ, NY, NX) mask of the level's unrefined cells."""
    parts = [(l, m, v, a, 4.0 ** -l) for l, (m, v, a) in enumerate(levels)]
    return _rings(parts, y0, z0, dr, nbins, x_stations)


def jet_fit(mean, var, counts, dr):
    """(u_m, b_e, tI, a, c) of one station's ring profile (module docstring);
    NaN where a quantity is undefined."""
    nan = float("nan")
    if counts[0] == 0 or not mean[0] > 0:
        return (nan,) * 5
    um = float(mean[0])
    ti = math.sqrt(max(float(var[0]), 0.0)) / um
    level = um / math.e
    be = nan
    for b in range(1, len(mean)):
        if counts[b] == 0 or counts[b - 1] == 0:
            continue
        if mean[b] <= level:
            r0 = (b - 0.5) * dr
            be = r0 + (mean[b - 1] - level) / (mean[b - 1] - mean[b]) * dr
            break
    if math.isnan(be):
        return um, nan, ti, nan, nan
    xs, ys = [], []
    for b in range(len(mean)):
        r = (b + 0.5) * dr
        if counts[b] > 0 and mean[b] >= 0.05 * um and r <= 2.0 * be:
            xs.append((r / be) ** 2)
            ys.append(math.log(mean[b] / um))
    n = len(xs)
    if n < 2:
        return um, be, ti, nan, nan
    sx, sy = sum(xs), sum(ys)
    sxx = sum(x * x for x in xs)
    sxy = sum(x * y for x, y in zip(xs, ys))
    den = n * sxx - sx * sx
    if den == 0:
        return um, be, ti, nan, nan
    slope = (n * sxy - sx * sy) / den
    icpt = (sy - slope * sx) / n
    return um, be, ti, math.exp(icpt), -slope

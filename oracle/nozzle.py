"""Solid bodies with interpolated no-slip walls: the nozzle cylinder of
Section 3.2 (a cylinder along the jet axis whose downstream end emits the
jet; its surface is a second-order interpolated no-slip wall after Bouzidi,
Firdaouss and Lallemand, cited there).

Test infrastructure: the plain, slow FP64 statement of the method that the
CUDA path is checked against.

Reading (the paper names the method, not its form): linear interpolation of
Bouzidi et al. for a link from a fluid cell x_f towards a solid cell
x_b = x_f + e_i that meets the wall at the fraction q of its length,
  q <  1/2:  f_ib(x_f, t+1) = 2q f~_i(x_f) + (1 - 2q) f~_i(x_f - e_i)
  q >= 1/2:  f_ib(x_f, t+1) = f~_i(x_f) / (2q) + (2q - 1) / (2q) f~_ib(x_f)
with ib the opposite of i and f~ the post-collision values at t.  Where
x_f - e_i is not a fluid cell the link falls back to half-way bounce-back,
f_ib(x_f, t+1) = f~_i(x_f).  The value is written into population ib of
the solid cell x_b before the pull streaming, so the pull of x_f takes it
unchanged.

The nozzle: solid cells are those whose centre lies in the closed cylinder
x0 <= x <= x1, (y - y0)^2 + (z - z0)^2 <= R^2 (coarse-cell units).  A link
whose segment (cell centre to cell centre) enters the cylinder first
through the downstream cap x = x1 is an inflow link: the solid cell then
acts as an inflow ghost, f_ib(x_b) = f_eq(rho(x_b + x^), u_bc(y_b, z_b)),
with the density of the fluid cell straight downstream and the inflow disc
velocity of the face inflow (the inflow moves from the face x = 0 onto the
cap; the face x = 0 holds u = 0).  Links entering through the side or the
upstream cap are no-slip links with the q of their entry point.

The body lies on one level l_n: the finest level whose blocks cover the
cylinder's bounding box grown by two cells of that level, each such block
and its 26 neighbours being non-refined blocks of level l_n (so links and
their second cells stay among active cells, and no interpolation stencil or
restriction of an interface reaches the body or a domain face).
"""
import math

import torch

from . import DTYPE

BLOCK = 8


class Cylinder:
    """The nozzle: closed cylinder along x (coarse-cell units); links that
    enter through the downstream cap x = x1 are inflow links."""

    def __init__(self, y0, z0, R, x0, x1):
        self.y0, self.z0, self.R, self.x0, self.x1 = (float(v) for v in (y0, z0, R, x0, x1))

    def inside(self, x, y, z):
        """Cell-centre test (tensors or floats, coarse units)."""
        dy, dz = y - self.y0, z - self.z0
        return (x >= self.x0) & (x <= self.x1) & (dy * dy + dz * dz <= self.R * self.R)

    def bbox(self, l):
        """Bounding box grown by two level-l cells, in level-l cell units."""
        s = float(2 ** l)
        return ((self.x0 * s - 2, self.x1 * s + 2), ((self.y0 - self.R) * s - 2, (self.y0 + self.R) * s + 2),
                ((self.z0 - self.R) * s - 2, (self.z0 + self.R) * s + 2))

    def entry(self, p, d):
        """Entry of the segment p + t d (t in [0, 1]; p outside, p + d
        inside): (t, inflow).  The cylinder is the intersection of the slab
        x0 <= x <= x1 and the infinite cylinder r <= R, so the segment enters
        it at the later of its entries into the two; an entry through the
        cap x = x1 is an inflow link."""
        px, py, pz = p[0], p[1] - self.y0, p[2] - self.z0
        dx, dy, dz = d
        if self.x0 <= px <= self.x1:
            ts, cap1 = 0.0, False
        elif px > self.x1:
            ts, cap1 = (self.x1 - px) / dx, True
        else:
            ts, cap1 = (self.x0 - px) / dx, False
        c = py * py + pz * pz - self.R * self.R
        if c <= 0:
            tc = 0.0
        else:
            a = dy * dy + dz * dz
            b = 2.0 * (py * dy + pz * dz)
            tc = (-b - math.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)
        if ts >= tc:
            return ts, cap1
        return tc, False


class Slab:
    """Solid layer a <= x <= b across the whole cross-section, both faces
    no-slip (plane walls at any position, for the pins)."""

    def __init__(self, a, b):
        self.a, self.b = float(a), float(b)

    def inside(self, x, y, z):
        return (x >= self.a) & (x <= self.b) & (y == y)

    def entry(self, p, d):
        t = (self.b - p[0]) / d[0] if p[0] > self.b else (self.a - p[0]) / d[0]
        return t, False


def nozzle_level(levels, geom):
    """The level holding the body (rule in the module docstring), or raise."""
    for l in range(len(levels) - 1, -1, -1):
        lv = levels[l]
        nbs = (lv.nbx, lv.nby, lv.nbz)
        box = geom.bbox(l)
        lo = [math.floor(a / BLOCK) for a, _ in box]
        hi = [math.floor(b / BLOCK) for _, b in box]
        if not all(lo[d] - 1 >= 0 and hi[d] + 1 <= nbs[d] - 1 for d in range(3)):
            continue
        reg, ref = lv.region_blocks, lv.refine_blocks
        ok = True
        for bz in range(lo[2], hi[2] + 1):
            for by in range(lo[1], hi[1] + 1):
                for bx in range(lo[0], hi[0] + 1):
                    nbh = (slice(bz - 1, bz + 2), slice(by - 1, by + 2), slice(bx - 1, bx + 2))
                    if not bool(reg[nbh].all()) or bool(ref[nbh].any()):
                        ok = False
        if ok:
            return l
    raise ValueError("the nozzle must lie inside non-refined blocks of one level, one block away "
                     "from its interfaces and the domain faces")


class Body:
    """Solid cells and links of a body on level l (padded level arrays)."""

    def __init__(self, geom, lv, l, e, periodic_x):
        self.geom, self.l = geom, l
        s = 1.0 / (2 ** l)
        NZ, NY, NXp = lv.region.shape
        xoff = lv.xoff
        zc = (torch.arange(NZ, dtype=DTYPE) + 0.5) * s
        yc = (torch.arange(NY, dtype=DTYPE) + 0.5) * s
        xc = (torch.arange(NXp, dtype=DTYPE) - xoff + 0.5) * s
        Z, Y, X = torch.meshgrid(zc, yc, xc, indexing="ij")
        self.solid = geom.inside(X, Y, Z)
        if not periodic_x:
            self.solid[:, :, 0] = False
            self.solid[:, :, -1] = False
        Q = e.shape[0]
        ev = [tuple(int(v) for v in e[i]) for i in range(Q)]
        opp = [ev.index((-a, -b, -c)) for (a, b, c) in ev]
        fl, bl, sl, pi, pib, q, inflow, has2 = [], [], [], [], [], [], [], []
        sol = self.solid
        for i in range(1, Q):
            ex, ey, ez = ev[i]
            # fluid cells whose neighbour x + e_i is solid
            nb = torch.roll(sol, shifts=(-ez, -ey, -ex), dims=(0, 1, 2))
            for z, y, x in torch.nonzero(nb & ~sol).tolist():
                p = (float(xc[x]), float(yc[y]), float(zc[z]))
                t, infl = geom.entry(p, (ex * s, ey * s, ez * s))
                z2, y2, x2 = (z - ez) % NZ, (y - ey) % NY, (x - ex) % NXp
                fl.append((z, y, x))
                bl.append(((z + ez) % NZ, (y + ey) % NY, (x + ex) % NXp))
                sl.append((z2, y2, x2))
                pi.append(i)
                pib.append(opp[i])
                q.append(t)
                inflow.append(infl)
                has2.append(not bool(sol[z2, y2, x2]))
        T = lambda v: torch.tensor(v, dtype=torch.long).reshape(-1, 3).t()
        self.f_idx = tuple(T(fl))
        self.b_idx = tuple(T(bl))
        self.s_idx = tuple(T(sl))
        self.i = torch.tensor(pi, dtype=torch.long)
        self.ib = torch.tensor(pib, dtype=torch.long)
        self.q = torch.tensor(q, dtype=DTYPE)
        self.inflow = torch.tensor(inflow, dtype=torch.bool)
        self.has2 = torch.tensor(has2, dtype=torch.bool)

    def wall_values(self, f):
        """Population ib at the solid cells of the links (Bouzidi linear
        interpolation; see the module docstring); inflow links are set
        apart by the caller."""
        a = f[self.i, self.f_idx[0], self.f_idx[1], self.f_idx[2]]
        b = f[self.i, self.s_idx[0], self.s_idx[1], self.s_idx[2]]
        c = f[self.ib, self.f_idx[0], self.f_idx[1], self.f_idx[2]]
        q = self.q
        lo = torch.where(self.has2, 2.0 * q * a + (1.0 - 2.0 * q) * b, a)
        hi = a / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * c
        return torch.where(q < 0.5, lo, hi)

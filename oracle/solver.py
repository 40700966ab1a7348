"""Time-nested stream-and-collide solver on the block grid (float64, CPU).

Stored state: the post-collision distributions f~(t) of every level, dense
over the level's whole domain, shape (Q, NZ, NY, NXp), [q][z][y][x].
One update of a level is pull streaming f(x, t+1) = f~(x - e_i, t) followed
by the collision of Section 2 (the left-hand sides of Eqs. lbgk / MRT are
the streaming; the collision is local, end of Section 2).

Time nesting (Sections 1 and 3.2, after Yu et al.): level l has grid spacing
and time step 2^-l of the coarse ones and takes 2 substeps per step of level
l-1, so nu_l = 2^l nu_0 in its own lattice units, i.e.
tau0_l - 1/2 = 2^l (tau0_0 - 1/2), with the same lattice velocity
(constant CFL, Section 3.2).  One step of level l (the reading of the cited
scheme used throughout this library):

  1. boundary ghosts of level l are filled from level-l values at time t;
  2. active and hidden-1 cells stream and collide -> f~_l(t+1);
  3. for fine substep s in (0, 1): the level-(l+1) ghost cells receive the
     coarse-to-fine transfer of F_s (F_0 = f~_l(t), F_1 = (f~_l(t)+f~_l(t+1))/2)
     and level l+1 takes its own step recursively;
  4. hidden cells of level l receive the fine-to-coarse transfer at t+1.

Coarse-to-fine: trilinear interpolation of all Q values from the 8 nearest
coarse cell centres (clamped at a non-periodic x face), then
f~_f = f_eq + r_cf (F^ - f_eq) about the equilibrium of the interpolated
moments, r_cf = (tau_f - 1) / (2 (tau_c - 1)).
Fine-to-coarse: per child f_eq + r_fc (f~ - f_eq), r_fc = 2 (tau_c - 1)/(tau_f - 1),
averaged over the 8 children.
With the Smagorinsky model the strain-rate norm |S| of each collision is
kept per cell and carried through the same interpolation; tau_c =
tau0_c + 3 Cs^2 |S|_c and tau_f = tau0_f + 3 Cs^2 |S|_c / 2 (|S| is halved in
fine lattice units).  Restriction takes tau_f from each child and
|S|_c = 2 |S|_child.

Boundaries (Section 3.2 names a constant inflow velocity; the rest is the
library's documented setup): x may be periodic; otherwise the ghost column
x = -1 holds f_eq(rho of the cell x = 0, u_bc) with the top-hat disc
velocity u_bc = u_in (1 + p xi_x, p xi_y, p xi_z) inside r < D/2 and 0
outside, and the ghost column x = NX holds a copy of cell x = NX - 1
(zero-gradient outflow).  y and z are periodic unless walls are requested.

Walls (Section 3.2 names no-slip walls for the tank and a free-slip top):
both faces of y and/or z may be walls of level 0 (refined blocks keep one
block away from them).  A population whose pull would cross a wall face is
reflected: at a no-slip face by half-way bounce-back, f_i(x, t+1) =
f~_opp(i)(x, t) (the wall lies half a cell outside the boundary cells); at a
free-slip face by specular reflection, the population with the wall-normal
velocity component flipped, pulled from the same layer, f_i(x, t+1) =
f~_m(i)(x - e_i + (e_i . n) n, t).  Where a link crosses two walls, a no-slip
crossing wins; two free-slip crossings reflect both components.  With x not
periodic, the face x = 0 (bit 4) and the face x = NX (bit 5) may be no-slip
walls too (the tank's upstream wall behind the nozzle; a closed box): they
replace the inflow or the outflow for the populations entering through them.

Pressure outlet (Section 3.2 replaces the tank's weir by a fixed pressure; the
scheme is not given): with outlet = 1 the ghost column x = NX of level 0
holds the equilibrium at the fixed density rho_out with the velocity of the
cell x = NX - 1, plus that cell's non-equilibrium part,
f_ghost = f_eq(rho_out, u_N) + (f_N - f_eq(rho_N, u_N)) (extrapolation of the
non-equilibrium part).  Its density is rho_out and its velocity u_N.  Refined
level-0 blocks keep one block away from the outlet face.
"""
import math

import numpy as np
import torch

from . import DTYPE
from .collision import Model
from .grid import build_levels
from .nozzle import Body, Cylinder, nozzle_level
from .rng import inflow_xi


class NestedSolver:
    def __init__(self, model, nb, periodic_x=True, refine=(), omega=1.0, cs=0.0, walls=0, slip=0,
                 outlet=0, nozzle=None, body=None):
        """walls: bit 0/1 the low/high y face, bit 2/3 the low/high z face are
        walls (both faces of an axis or neither), bit 4/5 the faces x = 0 and
        x = NX are no-slip walls (non-periodic x); slip: the y/z bits mark the
        free-slip walls among them (the others are no-slip).  outlet: 0
        zero-gradient outflow, 1 fixed-pressure outlet (non-periodic x).
        nozzle: (y0, z0, R, x0, x1) of the nozzle cylinder (oracle/nozzle.py),
        or None; body: another geometry of oracle/nozzle.py on a single-level
        grid (the pins' plane walls)."""
        self.m = Model(model)
        self.Q = self.m.Q
        if (walls & 3) not in (0, 3) or (walls & 12) not in (0, 12) or (walls & ~63) or (slip & ~(walls & 15)):
            raise ValueError("y/z walls come in pairs per axis; slip marks a subset of them")
        if (walls & 48) and periodic_x:
            raise ValueError("x walls need a non-periodic x axis")
        if (walls & 32) and outlet:
            raise ValueError("the face x = NX is either a wall or the pressure outlet")
        self.walls, self.slip = int(walls), int(slip)
        if outlet not in (0, 1) or (outlet and periodic_x):
            raise ValueError("outlet is 0 (zero-gradient) or 1 (fixed pressure, non-periodic x)")
        self.outlet = int(outlet)
        self.rho_out = 1.0
        refine = list(refine)
        if outlet and refine and bool(refine[0].bool()[:, :, -1].any()):
            raise ValueError("refined blocks must keep one block away from the pressure outlet")
        if walls and refine:
            r0 = refine[0].bool()
            near = torch.zeros_like(r0)
            if walls & 3:
                near[:, 0, :] = near[:, -1, :] = True
            if walls & 12:
                near[0] = near[-1] = True
            if walls & 16:
                near[:, :, 0] = True
            if walls & 32:
                near[:, :, -1] = True
            if bool((r0 & near).any()):
                raise ValueError("refined blocks must keep one block away from the walls")
        self.levels = build_levels(nb, periodic_x, refine)
        self.L = len(self.levels)
        self.body, self.nozzle = None, nozzle is not None
        if nozzle is not None or body is not None:
            if nozzle is not None:
                geom = Cylinder(*nozzle)
                ln = nozzle_level(self.levels, geom)
            else:
                if self.L != 1:
                    raise ValueError("a test body needs a single-level grid")
                geom, ln = body, 0
            self.body = Body(geom, self.levels[ln], ln, self.m.e, periodic_x)
            lv = self.levels[ln]
            for name in ("active", "update", "valid"):
                setattr(lv, name, getattr(lv, name) & ~self.body.solid)
        self.periodic_x = periodic_x
        self.omega0 = float(omega)
        self.cs = float(cs) if model == "d3q19" else 0.0
        tau00 = 1.0 / self.omega0
        self.tau0 = [0.5 + (2 ** l) * (tau00 - 0.5) for l in range(self.L)]
        self.f, self.S = [], []
        for lv in self.levels:
            shape = (lv.NZ, lv.NY, lv.NX + (0 if periodic_x else 2))
            f = torch.zeros((self.Q,) + shape, dtype=DTYPE)
            if self.m.name == "d3q27":
                f += self.m.w[:, None, None, None]
            self.f.append(f)
            self.S.append(torch.zeros(shape, dtype=DTYPE))
        self.force = None
        self.inflow = dict(y0=0.0, z0=0.0, D=0.0, u_in=0.0, perturb=0.0, seed=0)
        self.coarse_step = 0
        self._need_restrict = self.L > 1

    # ------------------------------------------------------------ set-up
    def real(self, l, a):
        """View of the real (non-ghost-column) x range of a level array."""
        o = self.levels[l].xoff
        return a[..., o:o + self.levels[l].NX]

    def set_inflow(self, y0, z0, D, u_in, perturb=0.01, seed=0):
        if self.periodic_x:
            raise ValueError("inflow needs a non-periodic x axis")
        self.inflow = dict(y0=float(y0), z0=float(z0), D=float(D), u_in=float(u_in),
                           perturb=float(perturb), seed=int(seed))

    def set_outlet(self, rho_out):
        """Density held at the pressure outlet (full density for both models)."""
        if not self.outlet:
            raise ValueError("the grid has no pressure outlet")
        self.rho_out = float(rho_out)

    def set_force(self, F):
        """Per-cell body force (3, NZ, NY, NX) on a single-level FCLB grid."""
        if self.L != 1 or self.m.name != "d3q27":
            raise ValueError("body force is defined for single-level D3Q27 grids")
        self.force = F.to(DTYPE).reshape(3, -1).clone()

    def init_equilibrium(self, l, rho=None, u=None):
        """f~ = f_eq(rho, u) on every real cell of level l (rest if None).

        rho is the full density for both models (D3Q19 stores rho - 1)."""
        lv = self.levels[l]
        n = lv.NX * lv.NY * lv.NZ
        r = torch.ones(n, dtype=DTYPE) if rho is None else rho.to(DTYPE).reshape(-1)
        v = torch.zeros(3, n, dtype=DTYPE) if u is None else u.to(DTYPE).reshape(3, -1)
        rl = r - 1.0 if self.m.name == "d3q19" else r
        feq = self.m.feq(rl, v).reshape(self.Q, lv.NZ, lv.NY, lv.NX)
        self.real(l, self.f[l])[...] = feq
        self.S[l].zero_()
        self._need_restrict = self.L > 1

    def set_state(self, l, f):
        self.real(l, self.f[l])[...] = f.to(DTYPE)
        self._need_restrict = False

    def state(self, l):
        return self.real(l, self.f[l]).clone()

    # ------------------------------------------------------------ pieces
    def _tau0(self, l):
        return self.tau0[l]

    def _apply_bc(self, l, sub):
        if self.periodic_x:
            return
        lv = self.levels[l]
        f = self.f[l]
        src_ok = lv.region | lv.ghost
        # inflow column x = -1 (padded index 0) from cell x = 0 (index 1)
        zz, yy = torch.nonzero(src_ok[:, :, 1], as_tuple=True)
        if len(zz):
            src = f[:, zz, yy, 1]
            rl = self.m.density_like(src)
            p = self.inflow
            sc = 1.0 / (2 ** l)
            yc = (yy.to(DTYPE) + 0.5) * sc
            zc = (zz.to(DTYPE) + 0.5) * sc
            inside = (yc - p["y0"]) ** 2 + (zc - p["z0"]) ** 2 < (0.5 * p["D"]) ** 2
            cell = (yy + lv.NY * zz).numpy()
            xi = [torch.from_numpy(inflow_xi(p["seed"], self.coarse_step, l, sub, cell, c))
                  for c in range(3)]
            u = torch.stack([p["u_in"] * (1.0 + p["perturb"] * xi[0]),
                             p["u_in"] * p["perturb"] * xi[1],
                             p["u_in"] * p["perturb"] * xi[2]])
            u = torch.where(inside[None], u, torch.zeros_like(u))
            if self.nozzle:                  # the inflow sits on the nozzle's cap
                u = torch.zeros_like(u)
            f[:, zz, yy, 0] = self.m.feq(rl, u)
        # outflow column x = NX (index NX+1) from cell x = NX-1 (index NX):
        # a copy (zero gradient), or at the pressure outlet the equilibrium at
        # rho_out with the cell's velocity plus the cell's non-equilibrium part
        zz, yy = torch.nonzero(src_ok[:, :, lv.NX], as_tuple=True)
        if len(zz):
            src = f[:, zz, yy, lv.NX]
            f[:, zz, yy, lv.NX + 1] = self._outlet_ghost(src) if self.outlet else src

    def _body_links(self, l, sub):
        """Populations of the solid cells that the body's links pull
        (oracle/nozzle.py): interpolated no-slip values, and on the nozzle's
        cap the inflow equilibrium from the fluid cell straight downstream."""
        b = self.body
        if b is None or l != b.l or len(b.i) == 0:
            return
        f = self.f[l]
        val = b.wall_values(f)
        if bool(b.inflow.any()):
            lv = self.levels[l]
            k = torch.nonzero(b.inflow, as_tuple=True)[0]
            bz, by, bx = (idx[k] for idx in b.b_idx)
            down = f[:, bz, by, bx + 1]
            rl = self.m.density_like(down)
            p = self.inflow
            sc = 1.0 / (2 ** l)
            yc = (by.to(DTYPE) + 0.5) * sc
            zc = (bz.to(DTYPE) + 0.5) * sc
            inside = (yc - p["y0"]) ** 2 + (zc - p["z0"]) ** 2 < (0.5 * p["D"]) ** 2
            cell = (by + lv.NY * bz).numpy()
            xi = [torch.from_numpy(inflow_xi(p["seed"], self.coarse_step, l, sub, cell, c)) for c in range(3)]
            u = torch.stack([p["u_in"] * (1.0 + p["perturb"] * xi[0]),
                             p["u_in"] * p["perturb"] * xi[1],
                             p["u_in"] * p["perturb"] * xi[2]])
            u = torch.where(inside[None], u, torch.zeros_like(u))
            feq = self.m.feq(rl, u)
            val[k] = feq[b.ib[k], torch.arange(len(k))]
        f[b.ib, b.b_idx[0], b.b_idx[1], b.b_idx[2]] = val

    def _outlet_ghost(self, src):
        """Pressure-outlet ghosts from the cells x = NX - 1 (Q, n): the
        equilibrium at rho_out with the cell's velocity plus the cell's
        non-equilibrium part."""
        u = self.m.velocity(src)
        rl_n = self.m.density_like(src)
        rl_out = torch.full_like(rl_n, self.rho_out - 1.0 if self.m.name == "d3q19" else self.rho_out)
        return self.m.feq(rl_out, u) + (src - self.m.feq(rl_n, u))

    def _vel_index(self, ex, ey, ez):
        for q in range(self.Q):
            if tuple(int(v) for v in self.m.e[q]) == (ex, ey, ez):
                return q
        raise KeyError((ex, ey, ez))

    def _wall_pulls(self, f, pre):
        """Replace the pulls that cross a wall face of level 0 (see the
        module docstring)."""
        NZ, NY, NXp = f.shape[1], f.shape[2], f.shape[3]
        zz = torch.arange(NZ).reshape(NZ, 1, 1)
        yy = torch.arange(NY).reshape(1, NY, 1)
        xx = torch.arange(NXp).reshape(1, 1, NXp)
        W, S = self.walls, self.slip
        x_lo, x_hi = 1, NXp - 2                       # padded indices of x = 0 and x = NX - 1
        for q in range(self.Q):
            ex, ey, ez = (int(v) for v in self.m.e[q])
            cy = torch.zeros((1, NY, 1), dtype=torch.bool)
            cz = torch.zeros((NZ, 1, 1), dtype=torch.bool)
            slip_y = slip_z = False
            if ey == 1 and W & 1:
                cy, slip_y = yy == 0, bool(S & 1)
            if ey == -1 and W & 2:
                cy, slip_y = yy == NY - 1, bool(S & 2)
            if ez == 1 and W & 4:
                cz, slip_z = zz == 0, bool(S & 4)
            if ez == -1 and W & 8:
                cz, slip_z = zz == NZ - 1, bool(S & 8)
            cx = torch.zeros((1, 1, NXp), dtype=torch.bool)
            if ex == 1 and W & 16:
                cx = xx == x_lo
            if ex == -1 and W & 32:
                cx = xx == x_hi
            cross = (cy | cz | cx).expand(pre[q].shape)
            if not bool(cross.any()):
                continue
            noslip = ((cy & (not slip_y)) | (cz & (not slip_z)) | cx).expand(pre[q].shape)
            both = (cy & cz).expand(pre[q].shape)
            only_y = (cy & ~cz).expand(pre[q].shape)
            bounce = f[self._vel_index(-ex, -ey, -ez)]
            mir_y = torch.roll(f[self._vel_index(ex, -ey, ez)], shifts=(ez, 0, ex), dims=(0, 1, 2))
            mir_z = torch.roll(f[self._vel_index(ex, ey, -ez)], shifts=(0, ey, ex), dims=(0, 1, 2))
            mir_yz = torch.roll(f[self._vel_index(ex, -ey, -ez)], shifts=(0, 0, ex), dims=(0, 1, 2))
            mirrored = torch.where(both, mir_yz, torch.where(only_y, mir_y, mir_z))
            pre[q] = torch.where(cross, torch.where(noslip, bounce, mirrored), pre[q])

    def _update(self, l, inplace=False):
        """Pull streaming and collision on the update mask of level l.

        The pulled value of population i at cell x is f_i(x - e_i) with the
        level array's periodic wrap (ghost columns included); with walls
        (level 0) the whole rolled array is formed and the wall pulls replace
        some of its entries, otherwise the same values are gathered at the
        updated cells alone.  inplace: write the result into the level's own
        arrays (the finest level, whose old state nothing reads)."""
        lv = self.levels[l]
        f = self.f[l]
        mask = lv.update
        if l == 0 and self.walls:
            pre = torch.empty_like(f)
            for q in range(self.Q):
                ex, ey, ez = (int(v) for v in self.m.e[q])
                pre[q] = torch.roll(f[q], shifts=(ez, ey, ex), dims=(0, 1, 2))
            self._wall_pulls(f, pre)
            fin = pre[:, mask]
        else:
            if getattr(lv, "update_cells", None) is None:
                lv.update_cells = torch.nonzero(mask, as_tuple=True)   # row-major, as mask indexing
            zz, yy, xx = lv.update_cells
            NZ, NY, NX = mask.shape
            fin = torch.empty((self.Q, len(zz)), dtype=DTYPE)
            for q in range(self.Q):
                ex, ey, ez = (int(v) for v in self.m.e[q])
                fin[q] = f[q, (zz - ez) % NZ, (yy - ey) % NY, (xx - ex) % NX]
        force = None
        if self.force is not None:
            force = self.force[:, self.real(l, mask).reshape(-1)]
        fout, sout = self.m.collide(fin, 1.0 / self._tau0(l), self.cs, force)
        if inplace:
            f[:, mask] = fout
            self.S[l][mask] = sout
            return f, self.S[l]
        new = f.clone()
        new[:, mask] = fout
        newS = self.S[l].clone()
        newS[mask] = sout
        return new, newS

    def _axis_stencil(self, X, n, periodic):
        """Coarse indices (i0, i1) and weights (w0, w1) for fine indices X."""
        i0 = torch.div(X - 1, 2, rounding_mode="floor")
        t = torch.where(X % 2 == 0, 0.75, 0.25).to(DTYPE)
        i1 = i0 + 1
        if periodic:
            i0, i1 = i0 % n, i1 % n
        else:
            i0, i1 = i0.clamp(0, n - 1), i1.clamp(0, n - 1)
        return (i0, i1), (1.0 - t, t)

    def _taus_cf(self, l, S_c):
        """(tau_c, tau_f) at an interface point from the coarse |S|."""
        tc = self.tau0[l] + 3.0 * self.cs ** 2 * S_c
        tf = self.tau0[l + 1] + 3.0 * self.cs ** 2 * S_c / 2.0
        return tc, tf

    def _c2f(self, l, s, old, new, oldS, newS):
        lc, lf = self.levels[l], self.levels[l + 1]
        F = old if s == 0 else 0.5 * (old + new)
        SS = oldS if s == 0 else 0.5 * (oldS + newS)
        zz, yy, xx = torch.nonzero(lf.ghost, as_tuple=True)
        X = xx - lf.xoff
        (x0, x1), (wx0, wx1) = self._axis_stencil(X, lc.NX, self.periodic_x)
        (y0, y1), (wy0, wy1) = self._axis_stencil(yy, lc.NY, True)
        (z0, z1), (wz0, wz1) = self._axis_stencil(zz, lc.NZ, True)
        Fh = torch.zeros(self.Q, len(zz), dtype=DTYPE)
        Sh = torch.zeros(len(zz), dtype=DTYPE)
        for zc, wz in ((z0, wz0), (z1, wz1)):
            for yc, wy in ((y0, wy0), (y1, wy1)):
                for xc, wx in ((x0, wx0), (x1, wx1)):
                    W = wz * wy * wx
                    assert bool(lc.update[zc, yc, xc + lc.xoff].all()), \
                        "interpolation stencil left the updated coarse cells"
                    Fh += W * F[:, zc, yc, xc + lc.xoff]
                    Sh += W * SS[zc, yc, xc + lc.xoff]
        rl = self.m.density_like(Fh)
        feq = self.m.feq(rl, self.m.velocity(Fh))
        tc, tf = self._taus_cf(l, Sh)
        r = (tf - 1.0) / (2.0 * (tc - 1.0))
        self.f[l + 1][:, zz, yy, xx] = feq + r * (Fh - feq)
        self.S[l + 1][zz, yy, xx] = Sh / 2.0

    def _f2c(self, l, new, newS):
        lc, lf = self.levels[l], self.levels[l + 1]
        hz, hy, hx = torch.nonzero(lc.hidden1 | lc.hidden2, as_tuple=True)
        X = hx - lc.xoff
        acc = torch.zeros(self.Q, len(hz), dtype=DTYPE)
        accS = torch.zeros(len(hz), dtype=DTYPE)
        ff, Sf = self.f[l + 1], self.S[l + 1]
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    cz, cy, cx = 2 * hz + dz, 2 * hy + dy, 2 * X + dx + lf.xoff
                    assert bool(lf.active[cz, cy, cx].all())
                    fc = ff[:, cz, cy, cx]
                    Sc = Sf[cz, cy, cx]
                    feq = self.m.feq(self.m.density_like(fc), self.m.velocity(fc))
                    tf = self.tau0[l + 1] + 3.0 * self.cs ** 2 * Sc
                    tc = self.tau0[l] + 3.0 * self.cs ** 2 * 2.0 * Sc
                    r = 2.0 * (tc - 1.0) / (tf - 1.0)
                    acc += feq + r * (fc - feq)
                    accS += 2.0 * Sc
        new[:, hz, hy, hx] = acc / 8.0
        newS[hz, hy, hx] = accS / 8.0

    def _restrict_all(self):
        for l in range(self.L - 2, -1, -1):
            self._f2c(l, self.f[l], self.S[l])
        self._need_restrict = False

    def _advance(self, l, sub):
        self._apply_bc(l, sub)
        self._body_links(l, sub)
        if l + 1 == self.L:
            self._update(l, inplace=True)
            return
        old, oldS = self.f[l].clone(), self.S[l].clone()
        new, newS = self._update(l)
        for s in (0, 1):
            self._c2f(l, s, old, new, oldS, newS)
            self._advance(l + 1, 2 * sub + s)
        self._f2c(l, new, newS)
        self.f[l], self.S[l] = new, newS

    # ------------------------------------------------------------ API
    def step(self, n=1):
        for _ in range(n):
            if self._need_restrict:
                self._restrict_all()
            self._advance(0, 0)
            self.coarse_step += 1

    def macroscopic(self, l):
        """(rho, u) on every real cell of level l; NaN where the level holds no
        valid value (outside its blocks, or deep inside refined blocks)."""
        lv = self.levels[l]
        f = self.real(l, self.f[l]).reshape(self.Q, -1)
        force = self.force if l == 0 else None
        rl = self.m.density_like(f)
        u = self.m.velocity(f, force) if self.m.name == "d3q27" else self.m.velocity(f)
        rho = rl + 1.0 if self.m.name == "d3q19" else rl
        valid = self.real(l, lv.valid).reshape(-1)
        rho = torch.where(valid, rho, torch.full_like(rho, float("nan")))
        u = torch.where(valid[None], u, torch.full_like(u, float("nan")))
        return rho.reshape(lv.NZ, lv.NY, lv.NX), u.reshape(3, lv.NZ, lv.NY, lv.NX)

    def mass_momentum(self):
        """Sum over active cells of all levels of (rho - 1, j) times the cell
        volume 8^-l (coarse units), j = sum f e."""
        out = torch.zeros(4, dtype=DTYPE)
        e = self.m.e.to(DTYPE)
        for l, lv in enumerate(self.levels):
            f = self.f[l][:, lv.active]
            d = f.sum(0) - (0.0 if self.m.name == "d3q19" else 1.0)
            j = e.t() @ f
            vol = 8.0 ** (-l)
            out[0] += vol * d.sum()
            out[1:] += vol * j.sum(1)
        return out

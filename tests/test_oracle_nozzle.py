"""Pins of the oracle's nozzle body (Section 3.2: a cylinder with
second-order interpolated no-slip walls after Bouzidi et al.; its
downstream end emits the jet)."""
import math

import numpy as np
import pytest
import torch

from oracle import DTYPE
from oracle.nozzle import Cylinder, Slab
from oracle.solver import NestedSolver
from tests.helpers import random_state

MODELS = ["d3q19", "d3q27"]
NOZ = (20.0, 20.0, 4.3, 10.25, 24.0)      # y0, z0, R, x0, x1 (cap on a cell face)


def bisect_entry(g, p, d, n=200):
    """Entry parameter of p + t d into the body by bisection on the
    cell-centre test (an independent route to the closed forms)."""
    lo, hi = 0.0, 1.0
    for _ in range(n):
        mid = 0.5 * (lo + hi)
        x, y, z = (p[k] + mid * d[k] for k in range(3))
        if bool(g.inside(x, y, z)):
            hi = mid
        else:
            lo = mid
    return hi


def test_link_fractions_match_bisection_and_axis_distances():
    """Every link's q equals the bisected entry of its segment; the links
    that enter through the downstream cap are exactly those whose entry
    point lies on the plane x = x1; and axis-parallel links in the plane
    through the axis have q = distance of the centre to the surface."""
    s = NestedSolver("d3q27", (5, 5, 5), periodic_x=False, nozzle=NOZ)
    b = s.body
    g = Cylinder(*NOZ)
    e = s.m.e
    assert len(b.q) > 1000
    for k in range(len(b.q)):
        z, y, x = (int(t[k]) for t in b.f_idx)
        p = (x - 1 + 0.5, y + 0.5, z + 0.5)              # padded x index -> x
        d = tuple(float(v) for v in e[int(b.i[k])])
        t = bisect_entry(g, p, d)
        assert abs(float(b.q[k]) - t) <= 1e-12, (k, float(b.q[k]), t)
        xe = p[0] + t * d[0]
        on_cap = abs(xe - NOZ[4]) <= 1e-9 and d[0] < 0
        assert bool(b.inflow[k]) == on_cap
    # links along -z through the side: the surface above a cell centre at
    # lateral offset dy lies at z0 + sqrt(R^2 - dy^2)
    n = 0
    for k in range(len(b.q)):
        z, y, x = (int(t[k]) for t in b.f_idx)
        if tuple(int(v) for v in e[int(b.i[k])]) == (0, 0, -1) and NOZ[3] < x - 0.5 < NOZ[4]:
            dy = y + 0.5 - NOZ[0]
            assert abs(float(b.q[k]) - ((z + 0.5) - NOZ[1] - math.sqrt(NOZ[2] ** 2 - dy ** 2))) <= 1e-12
            n += 1
    assert n > 50


@pytest.mark.parametrize("model", MODELS)
def test_rest_state_is_kept_with_a_nozzle(model):
    """Interpolations of equal values and the rest equilibrium on the cap
    keep a fluid at rest exactly at rest."""
    s = NestedSolver(model, (5, 5, 5), periodic_x=False, omega=1.3, cs=0.1 if model == "d3q19" else 0.0,
                     nozzle=NOZ)
    s.init_equilibrium(0)
    f0 = s.state(0)
    s.step(3)
    assert (s.state(0) - f0).abs().max().item() <= 1e-15


def plane_channel(slab, steps, omega=1.0 / 0.8):
    """Body-force-driven flow along y between the two faces of a solid slab in
    an x-periodic 16-cell box (D3Q27 FCLB), started from the exact profile.
    Returns (simulated u_y(x), exact u_y(x), u_max) on the fluid cells."""
    nb = (2, 1, 1)
    s = NestedSolver("d3q27", nb, periodic_x=True, omega=omega, body=slab)
    lv = s.levels[0]
    NX = lv.NX
    tau = 1.0 / omega
    nu = (tau - 0.5) / 3.0
    a, b = slab.a, slab.b
    H = NX + a - b
    umax = 0.01
    F = 8.0 * nu * umax / H ** 2
    xc = torch.arange(NX, dtype=DTYPE) + 0.5
    xu = torch.where(xc < a, xc + NX, xc)               # unwrap the channel
    fluid = (xc > b) | (xc < a)
    exact = torch.where(fluid, F / (2 * nu) * (xu - b) * (b + H - xu), torch.zeros_like(xc))
    u = torch.zeros(3, lv.NZ, lv.NY, NX, dtype=DTYPE)
    u[1] = exact[None, None, :]
    s.init_equilibrium(0, None, u)
    Fv = torch.zeros(3, lv.NZ, lv.NY, NX, dtype=DTYPE)
    Fv[1] = F
    s.set_force(Fv)
    s.step(steps)
    _, uu = s.macroscopic(0)
    return uu[1, 0, 0][fluid], exact[fluid], umax


@pytest.mark.parametrize("a,b", [(2.3, 5.2), (1.6, 4.45)])
def test_plane_walls_at_any_position_hold_poiseuille(a, b):
    """Plane no-slip walls cut at q = 0.3 / 0.8 and q = 0.05 / 0.1 of the
    links: the parabola between the true wall positions is held within
    2.5 % of its maximum over 300 steps.  The linear interpolation has a
    slip error of its own that grows with tau (1.2 % and 1.8 % here at
    tau = 0.8, 0.6 % for half-way bounce-back on walls at half cells);
    half-way bounce-back at the nearest half cell misses these profiles by
    8 % and 14 %."""
    sim, exact, umax = plane_channel(Slab(a, b), 300)
    assert (sim - exact).abs().max().item() <= 0.025 * umax, (sim - exact).abs().max().item() / umax


@pytest.mark.parametrize("model", MODELS)
def test_cap_inflow_equals_face_inflow(model):
    """The cap of the nozzle is the face inflow moved into the domain: with
    the same state downstream of the cap as behind the face x = 0, one step
    gives the same values on the first layers near the axis."""
    cs = 0.18 if model == "d3q19" else 0.0
    inflow = (20.0, 20.0, 6.0, 0.05, 0.02, 77)
    A = NestedSolver(model, (2, 5, 5), periodic_x=False, omega=1.7, cs=cs)
    B = NestedSolver(model, (5, 5, 5), periodic_x=False, omega=1.7, cs=cs, nozzle=NOZ)
    fa = torch.from_numpy(random_state(model, (16, 40, 40), 3, 0.1))
    fb = torch.from_numpy(random_state(model, (40, 40, 40), 4, 0.1))
    k = int(NOZ[4])
    fb[..., k:k + 16] = fa
    A.set_state(0, fa)
    B.set_state(0, fb)
    A.set_inflow(*inflow)
    B.set_inflow(*inflow)
    A.step(1)
    B.step(1)
    yy, zz = np.meshgrid(np.arange(40) + 0.5, np.arange(40) + 0.5, indexing="xy")
    near = torch.from_numpy((yy - 20.0) ** 2 + (zz - 20.0) ** 2 < (NOZ[2] - 1.5) ** 2)
    for j in range(3):
        da = A.state(0)[:, :, :, j][:, near]
        db = B.state(0)[:, :, :, k + j][:, near]
        assert (da - db).abs().max().item() <= 1e-14


def test_nozzle_placement_rules():
    r = torch.zeros(5, 5, 5, dtype=torch.bool)
    r[1:4, 1:4, 1:4] = True
    # inside level 1 with a block of margin: on level 1 (fine cells)
    s = NestedSolver("d3q27", (5, 5, 5), periodic_x=False, refine=[r], nozzle=(20.0, 20.0, 1.3, 18.25, 21.5))
    assert s.body.l == 1
    # too close to the level-1 interface: on level 0 it is refined -> rejected
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (5, 5, 5), periodic_x=False, refine=[r], nozzle=(20.0, 20.0, 4.3, 10.25, 24.0))
    with pytest.raises(ValueError):           # touches the domain's blocks next to the face
        NestedSolver("d3q27", (5, 5, 5), periodic_x=False, nozzle=(20.0, 20.0, 4.3, 2.25, 24.0))


def test_nozzle_next_to_refined_blocks_is_rejected():
    """A level-0 nozzle whose blocks touch a refined block would put solid
    cells into the coarse-to-fine stencils: rejected on both sides."""
    r = torch.zeros(5, 5, 5, dtype=torch.bool)
    r[2, 2, 4] = True                       # refined block next to the nozzle's blocks (x block 3)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (5, 5, 5), periodic_x=False, refine=[r], nozzle=NOZ)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("a,b", [(2.3, 5.2), (1.6, 4.45)])
def test_shear_wave_between_interpolated_walls_decays_at_the_true_width(model, a, b):
    """The lowest shear mode u_y = A sin(pi (x - b) / H) between plane
    no-slip walls at x = b and x = a + NX (cut at q = 0.3/0.8 and 0.05/0.1
    of the links) decays at nu (pi / H)^2 with H the true distance of the
    walls, within 0.5 % (walls at the nearest half cells would give 1.5 %
    and 12 % off), for both collision models."""
    tau = 0.8
    s = NestedSolver(model, (2, 1, 1), periodic_x=True, omega=1 / tau, cs=0.0, body=Slab(a, b))
    lv = s.levels[0]
    NX = lv.NX
    H = NX + a - b
    xc = torch.arange(NX, dtype=DTYPE) + 0.5
    xu = torch.where(xc < a, xc + NX, xc)
    fluid = (xc > b) | (xc < a)
    mode = torch.where(fluid, torch.sin(math.pi * (xu - b) / H), torch.zeros_like(xc))
    u = torch.zeros(3, lv.NZ, lv.NY, NX, dtype=DTYPE)
    u[1] = 1e-3 * mode[None, None, :]
    s.init_equilibrium(0, None, u)

    def amplitude():
        _, uu = s.macroscopic(0)
        v = torch.nan_to_num(uu[1, 0, 0])
        return float((v * mode).sum() / (mode * mode).sum())
    s.step(20)
    a0 = amplitude()
    s.step(200)
    rate = -math.log(amplitude() / a0) / 200
    expect = (tau - 0.5) / 3 * (math.pi / H) ** 2
    assert abs(rate / expect - 1) <= 0.005, rate / expect - 1

"""Pins of the oracle's block grid, time nesting, interface transfer and
boundary ghosts (Sections 1 and 3.2; the interface scheme is the reading
documented in oracle/solver.py)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle.grid import build_levels
from oracle.rng import inflow_xi, splitmix64
from oracle.solver import NestedSolver

D = torch.float64


def slab_refine(nb, axis, lo, hi):
    nbx, nby, nbz = nb
    r = torch.zeros(nbz, nby, nbx, dtype=torch.bool)
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(lo, hi)
    r[tuple(sl)] = True
    return r


def three_level_refine():
    """Smallest 3-level grid: 3x2x2 coarse blocks, two refined (full y-z
    cross-section, periodic), and two level-1 blocks refined again with a full
    ring of level-1 neighbours."""
    nb = (3, 2, 2)
    r0 = torch.zeros(2, 2, 3, dtype=torch.bool)
    r0[:, :, 0:2] = True
    r1 = torch.zeros(4, 4, 6, dtype=torch.bool)
    r1[1:3, 1:3, 1:3] = True
    return nb, [r0, r1]


def test_splitmix64_published_vector():
    """SplitMix64 from seed 1234567: the first outputs of the published
    reference generator (state advanced by the golden gamma before mixing)."""
    G = np.uint64(0x9E3779B97F4A7C15)
    s = np.uint64(1234567)
    out = []
    with np.errstate(over="ignore"):
        for _ in range(5):
            out.append(int(splitmix64(s)))
            s = s + G
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]
    xi = inflow_xi(5, 3, 1, 0, np.arange(10000), 2)
    assert xi.min() >= -1.0 and xi.max() < 1.0 and abs(xi.mean()) < 0.03


def test_slab_masks_counts():
    nb = (4, 2, 2)
    lv = build_levels(nb, True, [slab_refine(nb, 0, 1, 3)])
    c, f = lv
    assert int(c.refined.sum()) == 2 * 4 * 512
    assert int(c.hidden1.sum()) == 2 * 16 * 16
    assert int(c.hidden2.sum()) == 2 * 16 * 16
    assert int(c.active.sum()) == 8 * 512
    assert int(f.region.sum()) == 2 * 4 * 8 * 512
    assert int(f.ghost.sum()) == 2 * 32 * 32
    assert int(f.active.sum()) == int(f.region.sum())


def test_nesting_rule_rejects_touching_blocks():
    nb = (6, 4, 4)
    r0 = torch.zeros(4, 4, 6, dtype=torch.bool)
    r0[1:3, 1:3, 1:5] = True
    r1 = torch.zeros(8, 8, 12, dtype=torch.bool)
    r1[2:4, 3:5, 3:9] = True          # touches the level-1 boundary at z = 2
    with pytest.raises(ValueError):
        build_levels(nb, True, [r0, r1])
    r0b = r0.clone()
    r0b[0, 0, 0] = True
    r1b = torch.zeros(8, 8, 12, dtype=torch.bool)
    r1b[0, 0, 0] = True               # outside level 1? no: inside, but on its boundary
    with pytest.raises(ValueError):
        build_levels(nb, True, [r0b, r1b])


def test_jet_grid_sizes():
    """The 2-level jet grid: 27 648 coarse blocks, 32 refined block columns of
    48 blocks = 1 536, hence 12 288 fine blocks (6.29 M fine cells) and
    13.37 M active coarse cells, 25.95 M cell updates per coarse step."""
    flags, centre = synth.jet_two_level()
    r0 = torch.from_numpy(flags[0])
    assert r0.shape == (24, 24, 48) and centre == (96.0, 96.0)
    n_ref = int(r0.sum())
    assert n_ref == 1536
    coarse_active = (27648 - n_ref) * 512
    fine = 8 * n_ref * 512
    assert coarse_active == 13_369_344 and fine == 6_291_456
    assert coarse_active + 2 * fine == 25_952_256


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
@pytest.mark.parametrize("levels", [2, 3])
def test_uniform_flow_passes_refinement_unchanged(model, levels):
    if levels == 2:
        nb = (4, 2, 2)
        refine = [slab_refine(nb, 0, 1, 3)]
    else:
        nb, refine = three_level_refine()
    s = NestedSolver(model, nb, periodic_x=True, refine=refine, omega=1.6, cs=0.18)
    u0 = torch.tensor([0.05, 0.02, -0.01], dtype=D)
    for l, lv in enumerate(s.levels):
        s.init_equilibrium(l, None, u0[:, None, None, None].expand(3, lv.NZ, lv.NY, lv.NX))
    s.step(2)
    for l in range(len(s.levels)):
        rho, u = s.macroscopic(l)
        ok = ~torch.isnan(rho)
        assert (rho[ok] - 1).abs().max() < 1e-14
        assert (u[:, ok] - u0[:, None]).abs().max() < 1e-14


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_rest_state_with_zero_inflow_stays_at_rest(model):
    nb = (4, 2, 2)
    s = NestedSolver(model, nb, periodic_x=False, refine=[slab_refine(nb, 0, 0, 2)],
                     omega=1.7, cs=0.18)
    s.set_inflow(8.0, 8.0, 8.0, 0.0, 0.01, seed=3)
    for l in range(2):
        s.init_equilibrium(l)
    f0 = [s.state(l) for l in range(2)]
    s.step(2)
    for l in range(2):
        lv = s.levels[l]
        m = s.real(l, lv.valid)
        tol = 0.0 if model == "d3q19" else 1e-15    # FCLB f_eq is a linear solve
        assert (s.state(l)[:, m] - f0[l][:, m]).abs().max() <= tol


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_inflow_ghosts_carry_disc_velocity(model):
    """Inflow ghost column holds f_eq(rho of x = 0, u_bc): its velocity moment
    is u_in (1 + p xi) inside the disc and 0 outside (single level)."""
    s = NestedSolver(model, (2, 2, 2), periodic_x=False, omega=1.5)
    s.set_inflow(8.0, 7.0, 6.0, 0.05, 0.01, seed=11)
    s.init_equilibrium(0)
    s.step(1)
    lv = s.levels[0]
    s._apply_bc(0, 0)        # ghosts for coarse step 1, substep 0
    g = s.f[0][:, :, :, 0].reshape(s.Q, -1)
    u = s.m.velocity(g)
    zz, yy = torch.meshgrid(torch.arange(16), torch.arange(16), indexing="ij")
    inside = ((yy + 0.5 - 8.0) ** 2 + (zz + 0.5 - 7.0) ** 2 < 9.0).reshape(-1)
    cell = (yy + 16 * zz).reshape(-1).numpy()
    xi = torch.from_numpy(inflow_xi(11, 1, 0, 0, cell, 0))
    want = torch.where(inside, 0.05 * (1 + 0.01 * xi), torch.zeros_like(xi))
    assert inside.sum() > 20
    assert (u[0] - want).abs().max() < 1e-15


def composite_profile(s, NY0):
    """u_x(y) on coarse rows: coarse value where active, mean of fine children
    where the coarse cell is refined (2-level grids refined along y)."""
    rho0, u0 = s.macroscopic(0)
    c = s.levels[0]
    act = c.active[:, :, c.xoff:c.xoff + c.NX]
    prof = torch.zeros(NY0, dtype=D)
    _, u1 = s.macroscopic(1)
    for y in range(NY0):
        if bool(act[:, y, :].all()):
            prof[y] = u0[0][:, y, :].mean()
        else:
            prof[y] = u1[0][:, 2 * y:2 * y + 2, :].mean()
    return prof


def slab_decay_ratio(model, NY, omega=1.5, phase=0.0, drift=0.0):
    """Decay rate of a shear wave u_x = A sin(2 pi y/NY + phase) (with a uniform
    drift u_y) across a refined band y in [NY/4, 3NY/4), divided by the
    uniform-grid rate (window 10..40 coarse steps, scaled by (NY/32)^2).
    phase 0 puts the interfaces at velocity maxima (zero shear stress),
    phase pi/2 at velocity zeros (maximum shear stress)."""
    nb = (1, NY // 8, 1)
    k = 2 * math.pi / NY
    y = torch.arange(NY, dtype=D) + 0.5
    sc = (NY / 32) ** 2
    ts = (int(10 * sc), int(40 * sc))

    def run(refined):
        ref = [slab_refine(nb, 1, NY // 32, 3 * NY // 32)] if refined else []
        s = NestedSolver(model, nb, periodic_x=True, refine=ref, omega=omega)
        for l, lv in enumerate(s.levels):
            x, yy, z = synth.grid_coords(lv.NX, lv.NY, lv.NZ)
            u = np.zeros((3, lv.NZ, lv.NY, lv.NX))
            u[0] = 1e-3 * np.sin(2 * math.pi * yy / lv.NY + phase) * np.ones_like(x) * np.ones_like(z)
            u[1] = drift
            s.init_equilibrium(l, None, torch.from_numpy(u))
        amps = []
        for t in ts:
            s.step(t - s.coarse_step)
            prof = composite_profile(s, NY) if refined else s.macroscopic(0)[1][0].mean((0, 2))
            amps.append(abs(complex((prof * torch.cos(k * y)).sum(), (prof * torch.sin(k * y)).sum())))
        return -math.log(amps[1] / amps[0]) / (ts[1] - ts[0])

    return run(True) / run(False)


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_shear_wave_stress_crosses_interfaces(model):
    """Interfaces at the shear-stress maxima of the wave: the non-equilibrium
    rescaling must carry the viscous stress across both interfaces, so the
    decay rate equals the uniform-grid rate (measured within 0.1 %; without
    the rescaling it is 1.5 % slower)."""
    r = slab_decay_ratio(model, 32, phase=math.pi / 2)
    assert abs(r - 1.0) < 0.003, r


def drifting_wave_phase_advance(model, U, NY=32):
    """Phase advance of the shear wave u_x = A sin(k (y - U t) + phi0),
    carried through a refined band y in [NY/4, 3NY/4) by a uniform drift
    u_y = U, over coarse steps 10..40 (composite profile), divided by the
    closed-form advance k U (40 - 10).  phi0 puts a zero of u_x on the lower
    interface at the middle of the window (t = 25), where the profile is
    straight (no spatial interpolation error) and changes fastest in time,
    so the ghost values' temporal interpolation decides the phase."""
    nb = (1, NY // 8, 1)
    k = 2 * math.pi / NY
    y = torch.arange(NY, dtype=D) + 0.5
    ts = (10, 40)
    phi0 = math.pi / 2 + k * U * 25
    s = NestedSolver(model, nb, periodic_x=True, refine=[slab_refine(nb, 1, NY // 32, 3 * NY // 32)],
                     omega=1.5)
    for l, lv in enumerate(s.levels):
        x, yy, z = synth.grid_coords(lv.NX, lv.NY, lv.NZ)
        u = np.zeros((3, lv.NZ, lv.NY, lv.NX))
        u[0] = 1e-3 * np.sin(2 * math.pi * yy / lv.NY + phi0) * np.ones_like(x) * np.ones_like(z)
        u[1] = U
        s.init_equilibrium(l, None, torch.from_numpy(u))
    c = []
    for t in ts:
        s.step(t - s.coarse_step)
        prof = composite_profile(s, NY)
        c.append(complex((prof * torch.cos(k * y)).sum(), (prof * torch.sin(k * y)).sum()))
    ratio = c[1] / c[0]
    return abs(math.atan2(ratio.imag, ratio.real)) / (k * U * (ts[1] - ts[0]))


@pytest.mark.parametrize("U", [0.05, 0.1])
def test_drifting_wave_crosses_interfaces_at_the_exact_phase_speed(U):
    """Temporal interpolation of the coarse-to-fine ghosts (F_1 = the mean of
    the coarse post-collision fields at t and t+1).  A shear wave advected
    by a uniform drift travels at exactly the drift speed (Galilean
    invariance; the FCLB model keeps it on a uniform grid, measured 1e-6).
    Through a refined band, with a velocity zero on an interface, the ghost
    values lag or lead the coarse field by (w - 1/2) of a coarse step for a
    weight w on the new field, and the wave's phase advance changes by about
    1 % times (w - 1/2); with w = 1/2 the lag is second order.  Gate: within
    3e-4 of the closed form k U (t1 - t0) (measured 4e-5 at U = 0.05)."""
    r = drifting_wave_phase_advance("d3q27", U)
    assert abs(r - 1.0) < 3e-4, r


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_shear_wave_across_refined_slab(model):
    """Regression record, not a pin: interfaces at the velocity maxima of a
    wave drifting through them (u_y = 0.05) give a decay rate 3.65 % above
    the uniform rate (the linear ghost interpolation of the curved profile,
    first order: 1.8 % at NY = 64).  The window was drawn around the
    oracle's own value; the temporal interpolation is pinned by the phase
    speed above, the rescaling by the stress-crossing test."""
    r = slab_decay_ratio(model, 32, drift=0.05)
    assert 1.030 < r < 1.045, r


def test_shear_wave_across_refined_slab_converges():
    """The interface error of the decay rate halves when the resolution doubles
    (first order in the grid spacing): +3.7% at NY = 32, +1.8% at NY = 64."""
    e32 = slab_decay_ratio("d3q19", 32) - 1.0
    e64 = slab_decay_ratio("d3q19", 64) - 1.0
    assert 0 < e64 < 0.6 * e32


def test_nested_mass_drift_is_small():
    """The interface transfer is not exactly conservative (a documented
    property of the reading); the drift of a smooth flow stays small."""
    nb = (4, 2, 2)
    s = NestedSolver("d3q19", nb, periodic_x=True, refine=[slab_refine(nb, 0, 1, 3)],
                     omega=1.5, cs=0.1)
    for l, lv in enumerate(s.levels):
        rho, u = synth.taylor_green_3d(lv.NY, 0.03, shape=(lv.NX, lv.NY, lv.NZ))
        s.init_equilibrium(l, torch.from_numpy(rho), torch.from_numpy(u))
    s.step(1)
    m0 = s.mass_momentum()
    s.step(4)
    m1 = s.mass_momentum()
    vol = 32 * 16 * 16
    assert abs(float(m1[0] - m0[0])) / vol < 1e-5

"""Pins of the oracle's wall reflections (no-slip half-way bounce-back and
free-slip specular reflection on the y / z faces; Section 3.2 names no-slip
tank walls and a free-slip top)."""
import math

import numpy as np
import pytest
import torch

from oracle import DTYPE
from oracle.solver import NestedSolver
from tests.helpers import random_state

MODELS = ["d3q19", "d3q27"]


def solver(model, nb, walls, slip, omega=1.6, **kw):
    return NestedSolver(model, nb, periodic_x=True, omega=omega, cs=0.1 if model == "d3q19" else 0.0,
                        walls=walls, slip=slip, **kw)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", [(3, 0), (15, 12), (15, 2), (12, 12)])
def test_walls_conserve_mass(model, walls, slip):
    """Reflections only move populations: the total mass of a far-from-
    equilibrium state is conserved to round-off (the D3Q19 model stores
    the fluctuation, so its sum is the mass deviation)."""
    s = solver(model, (1, 2, 2), walls, slip)
    lv = s.levels[0]
    f = torch.from_numpy(random_state(model, (lv.NX, lv.NY, lv.NZ), 7, 0.2))
    s.set_state(0, f)
    m0 = s.state(0).sum().item()
    s.step(5)
    assert abs(s.state(0).sum().item() - m0) <= 1e-12 * f.numel()


@pytest.mark.parametrize("model", MODELS)
def test_free_slip_keeps_tangential_uniform_flow(model):
    """A uniform flow tangential to free-slip walls (both y and z faces) is an
    exact steady state: the mirrored equilibrium population is the same
    equilibrium value."""
    s = solver(model, (1, 1, 2), 15, 15)
    lv = s.levels[0]
    u = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    u[0] = 0.05
    s.init_equilibrium(0, None, u)
    f0 = s.state(0)
    s.step(5)
    assert (s.state(0) - f0).abs().max().item() <= 1e-14


def test_no_slip_poiseuille_profile():
    """Body-force-driven channel between no-slip y walls (half-way
    bounce-back puts them half a cell outside the boundary cells): the
    parabola u_x(y) = F / (2 nu) (y + 1/2) (H - 1/2 - y) is kept within 1 % of
    its maximum over 200 steps (D3Q27 FCLB, tau = 0.8)."""
    NY, tau, umax = 16, 0.8, 0.01
    nu = (tau - 0.5) / 3
    F = 8 * nu * umax / NY ** 2
    s = solver("d3q27", (1, 2, 1), 3, 0, omega=1 / tau)
    lv = s.levels[0]
    y = torch.arange(NY, dtype=DTYPE)
    ux = F / (2 * nu) * (y + 0.5) * (NY - 0.5 - y)
    u = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    u[0] = ux[None, :, None]
    s.init_equilibrium(0, None, u)
    Fv = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    Fv[0] = F
    s.set_force(Fv)
    s.step(200)
    _, uu = s.macroscopic(0)
    assert (uu[0] - ux[None, :, None]).abs().max().item() <= 0.01 * umax
    assert uu[1].abs().max().item() <= 1e-6 * umax


def test_walls_reject_refinement_next_to_them():
    r = torch.zeros(2, 2, 2, dtype=torch.bool)
    r[0, 0, 0] = True
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (2, 2, 2), refine=[r], walls=3)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (2, 2, 2), walls=1)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("slip", [0, 12, 3])
def test_closed_box_conserves_mass(model, slip):
    """All six faces walls (x faces no-slip, y/z mixed): the mass of a
    far-from-equilibrium state is conserved to round-off."""
    s = NestedSolver(model, (2, 1, 2), periodic_x=False, omega=1.6, cs=0.1 if model == "d3q19" else 0.0,
                     walls=63, slip=slip)
    lv = s.levels[0]
    f = torch.from_numpy(random_state(model, (lv.NX, lv.NY, lv.NZ), 17, 0.2))
    s.set_state(0, f)
    m0 = s.state(0).sum().item()
    s.step(5)
    assert abs(s.state(0).sum().item() - m0) <= 1e-12 * f.numel()


def test_x_walls_hold_poiseuille_profile():
    """Body-force-driven flow along y between no-slip walls at x = 0 and
    x = NX (half a cell outside the boundary cells): the parabola
    u_y(x) = F / (2 nu) (x + 1/2) (NX - 1/2 - x) is kept within 1 % of its
    maximum over 200 steps."""
    NX, tau, umax = 16, 0.8, 0.01
    nu = (tau - 0.5) / 3
    F = 8 * nu * umax / NX ** 2
    s = NestedSolver("d3q27", (2, 1, 1), periodic_x=False, omega=1 / tau, walls=48)
    lv = s.levels[0]
    x = torch.arange(NX, dtype=DTYPE)
    uy = F / (2 * nu) * (x + 0.5) * (NX - 0.5 - x)
    u = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    u[1] = uy[None, None, :]
    s.init_equilibrium(0, None, u)
    Fv = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    Fv[1] = F
    s.set_force(Fv)
    s.step(200)
    _, uu = s.macroscopic(0)
    assert (uu[1] - uy[None, None, :]).abs().max().item() <= 0.01 * umax
    assert uu[0].abs().max().item() <= 1e-6 * umax


def test_x_wall_rules():
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (2, 1, 1), periodic_x=True, walls=16)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (2, 1, 1), periodic_x=False, walls=32, outlet=1)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (2, 1, 1), periodic_x=False, walls=16, slip=16)
    r = torch.zeros(2, 2, 3, dtype=torch.bool)
    r[:, :, 0] = True
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (3, 2, 2), periodic_x=False, refine=[r], walls=16)
    NestedSolver("d3q27", (3, 2, 2), periodic_x=False, refine=[r], walls=32)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", [(3, 0), (15, 12)])
def test_shear_mode_between_no_slip_walls_decays_at_the_channel_rate(model, walls, slip):
    """u_x = A sin(pi (y + 1/2) / NY) between no-slip y walls (half a cell
    outside the boundary cells; free-slip z walls in the second case, which
    leave the mode alone) decays at nu (pi / NY)^2 within 0.5 %."""
    tau = 0.8
    s = NestedSolver(model, (1, 2, 1), periodic_x=True, omega=1 / tau, cs=0.0, walls=walls, slip=slip)
    lv = s.levels[0]
    y = torch.arange(lv.NY, dtype=DTYPE) + 0.5
    mode = torch.sin(math.pi * y / lv.NY)
    u = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    u[0] = 1e-3 * mode[None, :, None]
    s.init_equilibrium(0, None, u)

    def amplitude():
        _, uu = s.macroscopic(0)
        return float((uu[0, 0, :, 0] * mode).sum() / (mode * mode).sum())
    s.step(20)
    a0 = amplitude()
    s.step(200)
    rate = -math.log(amplitude() / a0) / 200
    expect = (tau - 0.5) / 3 * (math.pi / lv.NY) ** 2
    assert abs(rate / expect - 1) <= 0.005, rate / expect - 1

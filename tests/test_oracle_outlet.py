"""Pins of the oracle's fixed-pressure outlet (Section 3.2 replaces the tank's
weir by a fixed pressure; the scheme is read as the extrapolation of the
non-equilibrium part: f_ghost = f_eq(rho_out, u_N) + f_N - f_eq(rho_N, u_N))."""
import numpy as np
import pytest
import torch

from oracle import DTYPE
from oracle.solver import NestedSolver
from tests.helpers import random_state

MODELS = ["d3q19", "d3q27"]


def outlet_solver(model, nb, omega=1.2, **kw):
    return NestedSolver(model, nb, periodic_x=False, omega=omega, cs=0.1 if model == "d3q19" else 0.0,
                        outlet=1, **kw)


@pytest.mark.parametrize("model", MODELS)
def test_outlet_ghost_has_outlet_density_and_cell_velocity(model):
    """The ghost column carries rho_out and the velocity of the cell next to
    it, and the same non-equilibrium part (its second moment deviation from
    equilibrium equals the cell's)."""
    s = outlet_solver(model, (1, 1, 1))
    s.set_outlet(1.013)
    lv = s.levels[0]
    f = torch.from_numpy(random_state(model, (lv.NX, lv.NY, lv.NZ), 4, 0.05))
    s.set_state(0, f)
    s._apply_bc(0, 0)
    g = s.f[0][:, :, :, lv.NX + 1].reshape(s.Q, -1)
    n = s.f[0][:, :, :, lv.NX].reshape(s.Q, -1)
    rho_g = s.m.density_like(g) + (1.0 if model == "d3q19" else 0.0)
    assert (rho_g - 1.013).abs().max().item() <= 1e-13
    assert (s.m.velocity(g) - s.m.velocity(n)).abs().max().item() <= 1e-13
    e = s.m.e.to(DTYPE)

    def pi_neq(x):
        u = s.m.velocity(x)
        feq = s.m.feq(s.m.density_like(x), u)
        return torch.einsum("qa,qb,qn->abn", e, e, x - feq)
    assert (pi_neq(g) - pi_neq(n)).abs().max().item() <= 1e-13


@pytest.mark.parametrize("model", MODELS)
def test_outlet_keeps_uniform_flow_at_outlet_density(model):
    """A uniform equilibrium flow at rho_out, fed by an inflow disc covering
    the whole face, is an exact steady state."""
    s = outlet_solver(model, (2, 1, 1))
    lv = s.levels[0]
    u = torch.zeros(3, lv.NZ, lv.NY, lv.NX, dtype=DTYPE)
    u[0] = 0.04
    s.init_equilibrium(0, None, u)
    s.set_inflow(4.0, 4.0, 100.0, 0.04, 0.0, 1)
    f0 = s.state(0)
    s.step(5)
    assert (s.state(0) - f0).abs().max().item() <= 1e-14


@pytest.mark.parametrize("model", MODELS)
def test_outlet_drains_overpressure_to_rho_out(model):
    """Fluid at rest at rho = 1.02 behind a closed inflow (zero velocity,
    zero-gradient density): the outlet at rho_out = 1 lets the excess leave.
    The closed end and the open end make a weakly damped quarter-wave
    resonator, so the mean density oscillates about 1: its average over
    steps 200..400 is within a tenth of the initial excess of 1 (the
    zero-gradient outflow keeps the rest state at 1.02 for ever)."""
    s = outlet_solver(model, (2, 1, 1), omega=1.0)
    lv = s.levels[0]
    s.init_equilibrium(0, torch.full((lv.NZ, lv.NY, lv.NX), 1.02, dtype=DTYPE), None)
    s.set_inflow(4.0, 4.0, 0.0, 0.0, 0.0, 1)
    s.step(200)
    mean = []
    for _ in range(200):
        s.step(1)
        mean.append(s.macroscopic(0)[0].mean().item())
    assert abs(np.mean(mean) - 1.0) <= 0.1 * 0.02, np.mean(mean)
    z = NestedSolver(model, (2, 1, 1), periodic_x=False, omega=1.0, cs=s.cs)
    z.init_equilibrium(0, torch.full((lv.NZ, lv.NY, lv.NX), 1.02, dtype=DTYPE), None)
    z.set_inflow(4.0, 4.0, 0.0, 0.0, 0.0, 1)
    z.step(50)
    assert abs(z.macroscopic(0)[0].mean().item() - 1.02) <= 1e-12


@pytest.mark.parametrize("model", MODELS)
def test_outlet_cell_of_x_invariant_state_evolves_as_periodic(model):
    """For an x-invariant state at rho_out in every cell (random
    non-equilibrium parts, velocity varying in y and z), the extrapolated
    ghost equals the cell's own populations, so one step of the cells next to
    the outlet matches the x-periodic evolution of the same state."""
    nb = (1, 1, 1)
    s = outlet_solver(model, nb, omega=1.6)
    p = NestedSolver(model, nb, periodic_x=True, omega=1.6, cs=s.cs)
    lv = s.levels[0]
    f = torch.from_numpy(random_state(model, (1, lv.NY, lv.NZ), 9, 0.05)).expand(-1, -1, -1, lv.NX)
    f = f.clone()
    # shift the rest population so every cell has exactly rho_out = 1
    rl = f.sum(0)
    f[0] -= rl - (0.0 if model == "d3q19" else 1.0)
    s.set_state(0, f)
    p.set_state(0, f)
    s.step(1)
    p.step(1)
    a, b = s.state(0)[:, :, :, -1], p.state(0)[:, :, :, -1]
    assert (a - b).abs().max().item() <= 1e-14


def test_outlet_rejects_refinement_at_the_outlet_and_periodic_x():
    r = torch.zeros(2, 2, 3, dtype=torch.bool)
    r[:, :, 2] = True
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (3, 2, 2), periodic_x=False, refine=[r], outlet=1)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (3, 2, 2), periodic_x=True, outlet=1)

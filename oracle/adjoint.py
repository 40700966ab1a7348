"""Reference gradient of a loss of the final state w.r.t. a constant body
force, for the forced D3Q27 FCLB update on one periodic level (float64).

This is the plain definition: reverse-mode automatic differentiation
(torch.autograd) through the oracle's own forward steps (oracle/solver.py,
oracle/collision.py: central moments by definition, per-cell linear solves).
The paper has no adjoint; the forced update is this library's reading (the
force enters as u = (sum f e + F/2)/rho and a post-collision first central
moment F/(2 rho)).
"""
import torch

from . import DTYPE
from .solver import NestedSolver


def forward_final_state(f0, F, nb, omega, T):
    """f_T (27, NZ, NY, NX) after T forced steps from f0 (differentiable in F)."""
    s = NestedSolver("d3q27", nb, periodic_x=True, omega=omega)
    s.set_force(F)
    s.set_state(0, f0)
    s.step(T)
    return s.state(0)


def kinetic_energy_loss(fT, F, region):
    """L = 1/2 sum_region rho |u|^2, u = (sum f e + F/2)/rho (half-step velocity)."""
    from .lattice import velocities
    e = velocities(27).to(DTYPE)
    z0, z1, y0, y1, x0, x1 = region
    f = fT[:, z0:z1, y0:y1, x0:x1]
    Fr = F[:, z0:z1, y0:y1, x0:x1]
    rho = f.sum(0)
    j = torch.einsum("qzyx,qa->azyx", f, e) + 0.5 * Fr
    return 0.5 * ((j * j).sum(0) / rho).sum()


def reference_gradient(f0, F, nb, omega, T, region):
    """(L, dL/dF) by autograd through T oracle steps."""
    Fv = F.detach().clone().to(DTYPE).requires_grad_(True)
    fT = forward_final_state(f0.to(DTYPE), Fv, nb, omega, T)
    L = kinetic_energy_loss(fT, Fv, region)
    (g,) = torch.autograd.grad(L, Fv)
    return float(L.detach()), g

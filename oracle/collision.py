"""Collision operators of Section 2, written from their definitions in float64.

Arrays are (Q, N): population index first, N cells along the last axis.

Readings of the paper used here (each is a documented reading, not a guess):
* The collision term relaxes toward equilibrium, f* = f - M^-1 S (M f - m_eq);
  the printed '+' sign of Eqs. lbgk and MRT is read as this relaxation.
* The c_s factors printed in the incompressible equilibrium and in
  Eq. relaxationTau are read as the standard lattice form with c = 1:
  f_eq = w (drho + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2) and tau = 3 nu + 1/2.
* Pi^neq_ab = sum_i e_ia e_ib (f_i - f_eq_i); Q = sqrt(2 Pi:Pi) (Eq. EqnQ);
  tau_total from Eq. eqTauTotFinal with tau_0 = 1/omega.
* MRT basis = the raw moments of Table 1 plus density and momentum, with the
  misprints of Table 1 read as mu_113 +- mu_223 for the third s3/s4 entry.
* FCLB: central moments normalised by rho; the second-order deviatoric part
  is relaxed with omega (= Delta t / tau, the s1 group), the trace and every
  higher moment with rate 1, so they take their Table 2 equilibria built from
  the post-collision second-order moments.
"""
import itertools

import torch

from . import DTYPE
from .lattice import velocities, weights


# ---------------------------------------------------------------- D3Q19 MRT-LES

def moments_incompressible(f):
    """delta rho = sum f_i and u = sum f_i e_i / rho_0, rho_0 = 1 (Section 2)."""
    e = velocities(f.shape[0]).to(DTYPE)
    return f.sum(0), e.t() @ f


def feq_incompressible(drho, u, Q=19):
    """He-Luo incompressible equilibrium of Section 2 (c = 1 reading)."""
    e = velocities(Q).to(DTYPE)
    w = weights(Q)
    eu = e @ u                                   # (Q, N)
    uu = (u * u).sum(0)                          # (N,)
    return w[:, None] * (drho[None] + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu[None])


def mrt_matrix():
    """19 x 19 raw-moment matrix: density, momentum and the Table 1 groups.

    Row order: rho, j_x, j_y, j_z | s1: mu12, mu13, mu23, mu11-mu22, mu11-mu33 |
    s2: mu11+mu22+mu33 | s3: mu122+mu133, mu112+mu233, mu113+mu223 |
    s4: mu122-mu133, mu112-mu233, mu113-mu223 |
    s7: mu1122-2mu1133+mu2233, mu1122+mu1133-2mu2233, mu1122+mu1133+mu2233.
    mu_{1..2..3..} is sum_i f_i e_x^a e_y^b e_z^c (Section 2 index notation).
    """
    e = velocities(19).to(DTYPE)
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    rows = [
        torch.ones(19, dtype=DTYPE), x, y, z,
        x * y, x * z, y * z, x * x - y * y, x * x - z * z,
        x * x + y * y + z * z,
        x * y * y + x * z * z, x * x * y + y * z * z, x * x * z + y * y * z,
        x * y * y - x * z * z, x * x * y - y * z * z, x * x * z - y * y * z,
        x * x * y * y - 2 * x * x * z * z + y * y * z * z,
        x * x * y * y + x * x * z * z - 2 * y * y * z * z,
        x * x * y * y + x * x * z * z + y * y * z * z,
    ]
    return torch.stack(rows)


SHEAR_ROWS = slice(4, 9)


def tau_total(tau0, cs, Qn):
    """Eq. eqTauTotFinal in lattice units: tau0 + (sqrt(tau0^2 + 18 Cs^2 Q) - tau0)/2."""
    return tau0 + (torch.sqrt(tau0 * tau0 + 18.0 * cs * cs * Qn) - tau0) / 2.0


def strain_norm_q(fneq, Q=19):
    """Q = sqrt(2 sum_ab Pi_ab^2), Pi_ab = sum_i e_ia e_ib f^neq_i (Eq. EqnQ)."""
    e = velocities(Q).to(DTYPE)
    Pi = torch.einsum("qn,qa,qb->abn", fneq, e, e)
    return torch.sqrt(2.0 * (Pi * Pi).sum((0, 1)))


def mrt_les_collide(f, omega, cs, rates=None):
    """D3Q19 MRT with Smagorinsky eddy viscosity (Eqs. MRT, eqSmago..EqnQ).

    rates: optional (s2, s3, s4, s7); the paper's choice is all 1 (Section 2).
    Returns (f*, |S|) with |S| = 3 Q / (2 tau_total) the strain-rate norm of
    Eq. eqStrainRate (lattice units, sign dropped since it is a norm).
    """
    s2, s3, s4, s7 = (1.0, 1.0, 1.0, 1.0) if rates is None else rates
    drho, u = moments_incompressible(f)
    feq = feq_incompressible(drho, u)
    Qn = strain_norm_q(f - feq)
    tau0 = 1.0 / omega
    tau = tau_total(tau0, cs, Qn)
    s1 = 1.0 / tau                                          # (N,)
    n = f.shape[1]
    S = torch.empty(19, n, dtype=DTYPE)
    S[0:4] = 0.0
    S[4:9] = s1[None]
    S[9] = s2
    S[10:13] = s3
    S[13:16] = s4
    S[16:19] = s7
    M = mrt_matrix()
    Minv = torch.linalg.inv(M)          # Gaussian elimination with pivoting
    fstar = f - Minv @ (S * (M @ f - M @ feq))
    return fstar, 1.5 * Qn / tau


# ---------------------------------------------------------------- D3Q27 FCLB

# central moment index (a, b, c) = powers of (e_x - u_x, e_y - u_y, e_z - u_z)
ORDERS = [(a, b, c) for c in range(3) for b in range(3) for a in range(3)]
IDX = {abc: k for k, abc in enumerate(ORDERS)}


def central_moment_matrix(u):
    """K(u)[n, k, i] = prod_alpha (e_i,alpha - u_alpha,n)^{p_alpha(k)} (Section 2)."""
    e = velocities(27).to(DTYPE)                              # (27, 3)
    d = e[None, :, :] - u.t()[:, None, :]                     # (N, 27, 3)
    one = torch.ones_like(d[:, :, 0])
    pw = [[one, d[:, :, k], d[:, :, k] * d[:, :, k]] for k in range(3)]
    rows = [pw[0][a] * pw[1][b] * pw[2][c] for (a, b, c) in ORDERS]
    return torch.stack(rows, 1)                               # (N, 27k, 27i)


def moments_compressible(f, force=None):
    """rho = sum f_i, rho u = sum f_i e_i (Eqs. momZero..momOne).

    With a body force F the velocity is taken half a step forward,
    u = (sum f e + F/2)/rho (reading for the forced runs; the paper has no force).
    """
    e = velocities(27).to(DTYPE)
    rho = f.sum(0)
    j = e.t() @ f
    if force is not None:
        j = j + 0.5 * force
    return rho, j / rho


def fclb_relax(kappa, omega, rho, force=None):
    """Post-collision normalised central moments kappa' (Table 2 equilibria).

    kappa: (N, 27) normalised central moments.  Second order: deviatoric part
    relaxed by (1 - omega), trace set to 1; third and fifth order 0; fourth and
    sixth order the products of the post-collision second-order moments.
    """
    k = kappa
    out = torch.zeros_like(k)
    g = lambda abc: k[:, IDX[abc]]
    out[:, IDX[(0, 0, 0)]] = 1.0
    if force is not None:
        out[:, IDX[(1, 0, 0)]] = 0.5 * force[0] / rho
        out[:, IDX[(0, 1, 0)]] = 0.5 * force[1] / rho
        out[:, IDX[(0, 0, 1)]] = 0.5 * force[2] / rho
    mean = (g((2, 0, 0)) + g((0, 2, 0)) + g((0, 0, 2))) / 3.0
    xx = 1.0 / 3.0 + (1.0 - omega) * (g((2, 0, 0)) - mean)
    yy = 1.0 / 3.0 + (1.0 - omega) * (g((0, 2, 0)) - mean)
    zz = 1.0 / 3.0 + (1.0 - omega) * (g((0, 0, 2)) - mean)
    xy = (1.0 - omega) * g((1, 1, 0))
    xz = (1.0 - omega) * g((1, 0, 1))
    yz = (1.0 - omega) * g((0, 1, 1))
    out[:, IDX[(2, 0, 0)]] = xx
    out[:, IDX[(0, 2, 0)]] = yy
    out[:, IDX[(0, 0, 2)]] = zz
    out[:, IDX[(1, 1, 0)]] = xy
    out[:, IDX[(1, 0, 1)]] = xz
    out[:, IDX[(0, 1, 1)]] = yz
    # fourth order (s7, s8 groups): M11M22, M11M33, M22M33, M33M12, M22M13, M11M23
    out[:, IDX[(2, 2, 0)]] = xx * yy
    out[:, IDX[(2, 0, 2)]] = xx * zz
    out[:, IDX[(0, 2, 2)]] = yy * zz
    out[:, IDX[(1, 1, 2)]] = zz * xy
    out[:, IDX[(1, 2, 1)]] = yy * xz
    out[:, IDX[(2, 1, 1)]] = xx * yz
    # sixth order (s10): M11M22M33
    out[:, IDX[(2, 2, 2)]] = xx * yy * zz
    return out


def fclb_collide(f, omega, force=None):
    """D3Q27 factorized cascaded collision, recomputing whole moments (Section 2).

    f: (27, N) full distributions (not shifted).  Returns f*.
    The forward transform is the central-moment definition; the backward
    transform solves K(u) g = kappa' per cell (Gaussian elimination).
    """
    rho, u = moments_compressible(f, force)
    K = central_moment_matrix(u)                                  # (N,27,27)
    kappa = torch.einsum("nki,in->nk", K, f) / rho[:, None]
    kp = fclb_relax(kappa, omega, rho, force)
    g = torch.linalg.solve(K, kp)                                  # (N, 27)
    return (rho[:, None] * g).t().contiguous()


REST_CENTRAL = {0: 1.0, 1: 0.0, 2: 1.0 / 3.0}


def feq_fclb(rho, u):
    """Equilibrium of the FCLB model: the distribution whose normalised central
    moments are the Table 2 equilibria at rest shape (second order 1/3, fourth
    1/9, sixth 1/27, all others 0), solved from the definition."""
    K = central_moment_matrix(u)
    kap = torch.tensor([REST_CENTRAL[a] * REST_CENTRAL[b] * REST_CENTRAL[c]
                        for (a, b, c) in ORDERS], dtype=DTYPE)
    g = torch.linalg.solve(K, kap.expand(K.shape[0], 27))
    return (rho[:, None] * g).t().contiguous()


# ---------------------------------------------------------------- model wrapper

class Model:
    """Uniform view of the two collision models used by the solver."""

    def __init__(self, name):
        if name not in ("d3q19", "d3q27"):
            raise ValueError(name)
        self.name = name
        self.Q = 19 if name == "d3q19" else 27
        self.e = velocities(self.Q)
        self.w = weights(self.Q)

    def density_like(self, f):
        """delta rho for the incompressible D3Q19 model, rho for D3Q27."""
        return f.sum(0)

    def velocity(self, f, force=None):
        if self.name == "d3q19":
            return moments_incompressible(f)[1]
        return moments_compressible(f, force)[1]

    def feq(self, rho_like, u):
        if self.name == "d3q19":
            return feq_incompressible(rho_like, u)
        return feq_fclb(rho_like, u)

    def collide(self, f, omega, cs, force=None):
        """Returns (f*, |S|); |S| is zero for FCLB (no eddy viscosity)."""
        if self.name == "d3q19":
            return mrt_les_collide(f, omega, cs)
        return fclb_collide(f, omega, force), torch.zeros(f.shape[1], dtype=DTYPE)

    def rest_density_like(self):
        """Density-like value of the fluid at rest: delta rho = 0 or rho = 1."""
        return 0.0 if self.name == "d3q19" else 1.0

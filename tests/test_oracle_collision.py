"""Pins of the oracle's collision operators (Section 2) against properties the
paper and the mathematics fix: conservation, equilibrium fixed points, the
BGK special case, a closed form of the MRT projection, the Smagorinsky
closed form and the Table 2 polynomials."""
import os
import re

import numpy as np
import pytest
import torch

import synth
from oracle.collision import (IDX, ORDERS, central_moment_matrix, fclb_collide, feq_fclb,
                              feq_incompressible, moments_compressible,
                              moments_incompressible, mrt_les_collide, mrt_matrix,
                              strain_norm_q, tau_total)
from oracle.lattice import velocities, weights

D = torch.float64
HERE = os.path.dirname(os.path.abspath(__file__))


def near_eq19(n, seed, amp=1e-3):
    g = torch.Generator().manual_seed(seed)
    drho = 0.01 * torch.randn(n, generator=g, dtype=D)
    u = 0.05 * torch.randn(3, n, generator=g, dtype=D)
    return feq_incompressible(drho, u) + amp * torch.randn(19, n, generator=g, dtype=D) / 19


def near_eq27(n, seed, amp=1e-3):
    g = torch.Generator().manual_seed(seed)
    rho = 1.0 + 0.01 * torch.randn(n, generator=g, dtype=D)
    u = 0.05 * torch.randn(3, n, generator=g, dtype=D)
    return feq_fclb(rho, u) + amp * torch.randn(27, n, generator=g, dtype=D) / 27


# ---------------------------------------------------------------- D3Q19 MRT-LES

def test_mrt_matrix_rank_and_conditioning():
    M = mrt_matrix()
    assert torch.linalg.matrix_rank(M) == 19
    assert torch.linalg.cond(M) < 20.0


@pytest.mark.parametrize("cs", [0.0, 0.1, 0.18])
def test_mrt_conserves_density_and_momentum(cs):
    f = near_eq19(500, 1, amp=1e-2)
    fs, _ = mrt_les_collide(f, 1.7, cs)
    r0, j0 = moments_incompressible(f)
    r1, j1 = moments_incompressible(fs)
    assert torch.allclose(r0, r1, atol=1e-15, rtol=0)
    assert torch.allclose(j0, j1, atol=1e-15, rtol=0)


@pytest.mark.parametrize("cs", [0.0, 0.18])
def test_mrt_equilibrium_is_fixed_point(cs):
    g = torch.Generator().manual_seed(3)
    drho = 0.01 * torch.randn(200, generator=g, dtype=D)
    u = 0.08 * torch.randn(3, 200, generator=g, dtype=D)
    feq = feq_incompressible(drho, u)
    fs, S = mrt_les_collide(feq, 1.3, cs)
    assert (fs - feq).abs().max() < 1e-16
    assert S.abs().max() < 1e-13


def test_mrt_with_all_rates_omega_is_bgk():
    """All s_i = omega reduces Eq. MRT to the single-relaxation Eq. lbgk."""
    f = near_eq19(300, 5, amp=3e-2)
    om = 1.37
    fs, _ = mrt_les_collide(f, om, 0.0, rates=(om, om, om, om))
    drho, u = moments_incompressible(f)
    bgk = f - om * (f - feq_incompressible(drho, u))
    assert (fs - bgk).abs().max() < 1e-15


def test_mrt_omega_one_gives_equilibrium():
    f = near_eq19(300, 7, amp=3e-2)
    fs, _ = mrt_les_collide(f, 1.0, 0.0)
    drho, u = moments_incompressible(f)
    assert (fs - feq_incompressible(drho, u)).abs().max() < 1e-16


def test_mrt_shear_projection_closed_form():
    """With every non-shear rate 1 the raw-moment MRT equals
    f_eq + (1 - s1) P(f - f_eq), where P puts 1/2 (Pi_aa - tr/3) on the axis
    links and 1/4 e_a e_b Pi_ab on the diagonal links (derived by hand from
    the shear columns of M^-1: each column is the unique distribution whose
    only non-zero Table 1 moment is that shear moment)."""
    f = near_eq19(400, 9, amp=5e-2)
    om = 1.61
    fs, _ = mrt_les_collide(f, om, 0.0)
    drho, u = moments_incompressible(f)
    feq = feq_incompressible(drho, u)
    n = f - feq
    e = velocities(19).to(D)
    Pi = torch.einsum("qn,qa,qb->abn", n, e, e)
    tr = Pi[0, 0] + Pi[1, 1] + Pi[2, 2]
    P = torch.zeros_like(n)
    for i, v in enumerate(e.tolist()):
        nz = [a for a in range(3) if v[a] != 0]
        if len(nz) == 1:
            a = nz[0]
            P[i] = 0.5 * (Pi[a, a] - tr / 3.0)
        elif len(nz) == 2:
            a, b = nz
            P[i] = 0.25 * v[a] * v[b] * Pi[a, b]
    assert (fs - (feq + (1.0 - om) * P)).abs().max() < 1e-16


def test_smagorinsky_tau_solves_quadratic():
    """tau_total = tau0 + 3 nu_T with nu_T = Cs^2 |S|, |S| = 3Q/(2 tau_total)."""
    Qn = torch.logspace(-8, 0, 50, dtype=D)
    for tau0 in (0.5003, 0.515, 0.8, 1.4):
        for cs in (0.0, 0.1, 0.18):
            t = tau_total(tau0, cs, Qn)
            resid = t - (tau0 + 3.0 * cs * cs * 1.5 * Qn / t)
            assert resid.abs().max() < 1e-15 * (1 + t.max())


def test_smagorinsky_cs_zero_is_plain_mrt_and_small_q_scaling():
    f = near_eq19(300, 11, amp=2e-2)
    a, Sa = mrt_les_collide(f, 1.5, 0.0)
    drho, u = moments_incompressible(f)
    Qn = strain_norm_q(f - feq_incompressible(drho, u))
    # Cs = 0: s1 = omega everywhere; reproduce via rates of the plain model
    b, _ = mrt_les_collide(f, 1.5, 0.0, rates=(1.0, 1.0, 1.0, 1.0))
    assert torch.equal(a, b)
    # nu_T = (tau_total - tau0)/3 ~ Cs^2 * 3Q/(2 tau0) for small Q
    tau0 = 1.0 / 1.5
    for cs in (0.05, 0.1):
        nuT = (tau_total(tau0, cs, Qn) - tau0) / 3.0
        approx = cs * cs * 1.5 * Qn / tau0
        assert torch.allclose(nuT, approx, rtol=1e-2)


def test_strain_rate_from_nonequilibrium_matches_velocity_gradient():
    """Eq. eqStrainRate: |S| from Pi^neq equals sqrt(2 S:S) of a linear shear
    flow u_x = G y measured after one collision-free streaming of its
    equilibrium (Chapman-Enskog: Pi^neq = -2 rho c_s^2 tau S to first order)."""
    G = 1e-4
    N = 16
    y = torch.arange(N, dtype=D) + 0.5
    u = torch.zeros(3, N, dtype=D)
    u[0] = G * (y - N / 2)
    om = 1.0 / 0.8
    feq = feq_incompressible(torch.zeros(N, dtype=D), u)
    # relax to steady state in a 1-D channel periodic along the shear is not
    # possible, so check the first-order Chapman-Enskog relation instead:
    # streaming feq by e_y gives f - feq = -e_y d_y feq, whose Pi^neq_xy = -G/3
    e = velocities(19).to(D)
    dfeq = torch.stack([(feq[:, (i + 1) % N] - feq[:, (i - 1) % N]) / 2 for i in range(N)], 1)
    fneq = -(e[:, 1:2] * dfeq) * 0.8
    Qn = strain_norm_q(fneq[:, 4:12])
    S_exact = G  # sqrt(2 S:S) with S_xy = S_yx = G/2
    assert torch.allclose(1.5 * Qn / 0.8, torch.full_like(Qn, S_exact), rtol=1e-10)


# ---------------------------------------------------------------- D3Q27 FCLB

def test_central_moments_match_table2_polynomials():
    """The oracle's central moments (definition, Section 2) agree with every
    Table 2 row that is consistent; the three fourth-order diagonal rows and
    M123 disagree as printed and agree in their corrected reading."""
    f = near_eq27(64, 13, amp=5e-2)
    rho, u = moments_compressible(f)
    K = central_moment_matrix(u)
    kappa = torch.einsum("nki,in->nk", K, f) / rho[:, None]
    e = velocities(27).to(D)
    mu = {}
    for a in range(5):
        for b in range(5):
            for c in range(5):
                if a + b + c == 0 or a > 2 or b > 2 or c > 2:
                    continue
                name = "mu_" + "1" * a + "2" * b + "3" * c
                mu[name] = (f * (e[:, 0:1] ** a) * (e[:, 1:2] ** b) * (e[:, 2:3] ** c)).sum(0) / rho
    rows = []
    with open(os.path.join(HERE, "golden", "table2_central_moments.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, status, expr = (s.strip() for s in line.split("|"))
            rows.append((name, status, expr))
    assert len(rows) == 27  # 23 printed rows + 4 corrected readings
    for name, status, expr in rows:
        idx = name[1:]
        abc = (idx.count("1"), idx.count("2"), idx.count("3"))
        val = eval(expr, {}, dict(mu))
        err = (val - kappa[:, IDX[abc]]).abs().max().item()
        if status == "misprint":
            assert err > 1e-3, name
        else:
            assert err < 1e-14, (name, err)


def test_fclb_equilibrium_is_product_of_d1q3():
    """f_eq = rho prod_a phi(e_a, u_a), phi(0,u) = 2/3 - u^2,
    phi(+-1,u) = (1/3 + u^2 +- u)/2; at u = 0 this is rho w_i (D3Q27)."""
    g = torch.Generator().manual_seed(17)
    n = 100
    rho = 1.0 + 0.02 * torch.randn(n, generator=g, dtype=D)
    u = 0.1 * torch.randn(3, n, generator=g, dtype=D)
    fe = feq_fclb(rho, u)
    e = velocities(27)
    phi = lambda c, v: (2.0 / 3.0 - v * v) if c == 0 else 0.5 * (1.0 / 3.0 + v * v + c * v)
    ref = torch.stack([rho * phi(int(v[0]), u[0]) * phi(int(v[1]), u[1]) * phi(int(v[2]), u[2])
                       for v in e])
    assert (fe - ref).abs().max() < 2e-15
    fe0 = feq_fclb(torch.ones(1, dtype=D), torch.zeros(3, 1, dtype=D))[:, 0]
    assert (fe0 - weights(27)).abs().max() < 1e-15


def test_fclb_conserves_and_fixed_point():
    f = near_eq27(300, 19, amp=3e-2)
    fs = fclb_collide(f, 1.8)
    r0, u0 = moments_compressible(f)
    r1, u1 = moments_compressible(fs)
    assert (r0 - r1).abs().max() < 2e-15
    assert ((r0 * u0) - (r1 * u1)).abs().max() < 2e-15
    g = torch.Generator().manual_seed(23)
    rho = 1.0 + 0.02 * torch.randn(50, generator=g, dtype=D)
    u = 0.08 * torch.randn(3, 50, generator=g, dtype=D)
    fe = feq_fclb(rho, u)
    assert (fclb_collide(fe, 1.3) - fe).abs().max() < 2e-15


def test_fclb_omega_one_gives_product_equilibrium():
    f = near_eq27(200, 29, amp=5e-2)
    rho, u = moments_compressible(f)
    assert (fclb_collide(f, 1.0) - feq_fclb(rho, u)).abs().max() < 2e-15


def test_fclb_rest_central_moments():
    """kappa_200 = 1/3, kappa_220 = 1/9, kappa_222 = 1/27 for the equilibrium."""
    u = torch.tensor([[0.03], [-0.02], [0.05]], dtype=D)
    fe = feq_fclb(torch.tensor([1.1], dtype=D), u)
    K = central_moment_matrix(u)
    k = (K[0] @ fe[:, 0]) / 1.1
    assert abs(k[IDX[(2, 0, 0)]] - 1 / 3) < 1e-15
    assert abs(k[IDX[(2, 2, 0)]] - 1 / 9) < 1e-15
    assert abs(k[IDX[(2, 2, 2)]] - 1 / 27) < 1e-15
    assert abs(k[IDX[(1, 1, 0)]]) < 1e-15 and abs(k[IDX[(2, 1, 0)]]) < 1e-15


def test_fclb_second_order_relaxation():
    """Deviatoric second-order central moments relax by (1 - omega); trace -> 1."""
    f = near_eq27(100, 31, amp=5e-2)
    om = 1.45
    fs = fclb_collide(f, om)
    rho, u = moments_compressible(f)
    K = central_moment_matrix(u)
    k0 = torch.einsum("nki,in->nk", K, f) / rho[:, None]
    k1 = torch.einsum("nki,in->nk", K, fs) / rho[:, None]
    for a in ((1, 1, 0), (1, 0, 1), (0, 1, 1)):
        assert (k1[:, IDX[a]] - (1 - om) * k0[:, IDX[a]]).abs().max() < 1e-15
    tr1 = k1[:, IDX[(2, 0, 0)]] + k1[:, IDX[(0, 2, 0)]] + k1[:, IDX[(0, 0, 2)]]
    assert (tr1 - 1.0).abs().max() < 1e-15
    d0 = k0[:, IDX[(2, 0, 0)]] - k0[:, IDX[(0, 2, 0)]]
    d1 = k1[:, IDX[(2, 0, 0)]] - k1[:, IDX[(0, 2, 0)]]
    assert (d1 - (1 - om) * d0).abs().max() < 1e-15
    for a in ((2, 1, 0), (1, 1, 1), (2, 2, 1)):
        assert k1[:, IDX[a]].abs().max() < 1e-15


def test_fclb_force_adds_momentum():
    f = near_eq27(50, 37, amp=2e-2)
    g = torch.Generator().manual_seed(41)
    F = 1e-4 * torch.randn(3, 50, generator=g, dtype=D)
    fs = fclb_collide(f, 1.6, force=F)
    e = velocities(27).to(D)
    assert ((e.t() @ fs) - (e.t() @ f) - F).abs().max() < 2e-15
    assert (fs.sum(0) - f.sum(0)).abs().max() < 1e-15

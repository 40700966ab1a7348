"""Physics pins of the oracle solver: the viscosity of Eq. relaxationTau
recovered from closed-form decays, on one level and across a refined slab."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle.solver import NestedSolver

D = torch.float64


def amplitude(u_x, y_centres, ly):
    """Projection of u_x(y) on sin(2 pi y/ly) (average over x and z)."""
    prof = u_x.mean(dim=(0, 2))
    s = torch.sin(2 * math.pi * y_centres / ly)
    return float((prof * s).sum() / (s * s).sum())


def shear_decay_rate(model, omega, drift=0.0, NY=32, t1=20, t2=120, cs=0.0):
    s = NestedSolver(model, (1, NY // 8, 1), periodic_x=True, omega=omega, cs=cs)
    rho, u = synth.shear_wave(8, NY, 8, 1e-3, drift_y=drift)
    s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
    y = torch.arange(NY, dtype=D) + 0.5
    k = 2 * math.pi / NY
    def amp_complex():
        _, uu = s.macroscopic(0)
        prof = uu[0].mean(dim=(0, 2))
        return complex((prof * torch.cos(k * y)).sum(), (prof * torch.sin(k * y)).sum())
    s.step(t1)
    a1 = abs(amp_complex())
    s.step(t2 - t1)
    a2 = abs(amp_complex())
    return -math.log(a2 / a1) / (k * k * (t2 - t1))


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
@pytest.mark.parametrize("omega", [1.2, 1.8])
def test_shear_wave_viscosity(model, omega):
    """u_x = A sin(k y) decays as exp(-nu k^2 t), nu = (1/omega - 1/2)/3."""
    nu = (1.0 / omega - 0.5) / 3.0
    nu_fit = shear_decay_rate(model, omega)
    assert abs(nu_fit / nu - 1.0) < 0.01


def test_shear_wave_viscosity_converges():
    """The discrete decay rate converges to nu as the wave is resolved better."""
    omega = 1.5
    nu = (1.0 / omega - 0.5) / 3.0
    e16 = abs(shear_decay_rate("d3q19", omega, NY=16, t1=5, t2=35) / nu - 1)
    e32 = abs(shear_decay_rate("d3q19", omega, NY=32, t1=20, t2=140) / nu - 1)
    assert e32 < e16 or e32 < 1e-4


def test_fclb_galilean_shear_wave():
    """The FCLB decay rate is unchanged (1%) by a uniform drift U = 0.05 along k."""
    r0 = shear_decay_rate("d3q27", 1.4)
    r1 = shear_decay_rate("d3q27", 1.4, drift=0.05)
    assert abs(r1 / r0 - 1.0) < 0.01


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_taylor_green_2d_decay(model):
    """2-D Taylor-Green vortex (exact NS solution): KE ~ exp(-4 nu k^2 t)."""
    N, omega = 32, 1.4
    nu = (1.0 / omega - 0.5) / 3.0
    s = NestedSolver(model, (N // 8, N // 8, 1), periodic_x=True, omega=omega)
    rho, u = synth.taylor_green_2d(N, 0.01, NZ=8)
    s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
    k = 2 * math.pi / N
    s.step(10)
    ke1 = float((s.macroscopic(0)[1] ** 2).sum())
    s.step(60)
    ke2 = float((s.macroscopic(0)[1] ** 2).sum())
    nu_fit = -math.log(ke2 / ke1) / (4 * k * k * 60)
    assert abs(nu_fit / nu - 1.0) < 0.01


def tgv3d_rate(N, omega, u0, cs=0.0, T=60):
    """Least-squares slope of ln KE over t in [T/3, T], divided by 2 nu |k|^2."""
    nu = (1.0 / omega - 0.5) / 3.0
    k = 2 * math.pi / N
    s = NestedSolver("d3q19", (N // 8, N // 8, N // 8), periodic_x=True, omega=omega, cs=cs)
    rho, u = synth.taylor_green_3d(N, u0)
    s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
    ke = []
    for _ in range(T + 1):
        ke.append(float((s.macroscopic(0)[1] ** 2).sum()))
        s.step(1)
    t = np.arange(T // 3, T + 1)
    slope = np.polyfit(t, np.log(np.array(ke[T // 3:])), 1)[0]
    return -slope / (2 * nu * 3 * k * k)


def test_taylor_green_3d_early_decay():
    """3-D Taylor-Green vortex: at early times d ln KE/dt = -2 nu |k|^2,
    |k|^2 = 3 k^2 (every Fourier mode of the field has that wavenumber)."""
    assert abs(tgv3d_rate(32, 1.4, 0.05) - 1.0) < 0.01


def test_taylor_green_3d_low_viscosity_converges():
    """At the 32^3 test-case viscosity nu = 0.005 (tau = 0.515) the paper's rate
    choice (every non-shear rate 1) adds an O(k^2) error to the decay rate of
    this 3-D mode; it shrinks with resolution (measured: 23% at N = 16, 11% at
    N = 32, 2.6% at N = 64), and the Smagorinsky run (Cs = 0.1) decays faster."""
    omega = 1.0 / 0.515
    e16 = tgv3d_rate(16, omega, 0.002, T=30) - 1.0
    e32 = tgv3d_rate(32, omega, 0.002, T=60) - 1.0
    assert 0 < e32 < 0.6 * e16 and e32 < 0.15
    les = tgv3d_rate(32, omega, 0.05, cs=0.1, T=60)
    dns = tgv3d_rate(32, omega, 0.05, cs=0.0, T=60)
    assert dns < les < 1.05 * dns


def test_single_level_conserves_mass_and_momentum():
    for model in ("d3q19", "d3q27"):
        s = NestedSolver(model, (2, 1, 1), periodic_x=True, omega=1.3, cs=0.18)
        rho, u = synth.taylor_green_3d(16, 0.05, shape=(16, 8, 8))
        s.init_equilibrium(0, torch.from_numpy(rho), torch.from_numpy(u))
        m0 = s.mass_momentum()
        s.step(5)
        m1 = s.mass_momentum()
        assert (m1 - m0).abs().max() < 1e-12

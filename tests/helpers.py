"""Shared helpers of the GPU parity tests: run the CUDA library and the oracle
on the same seeded input and compare.  The oracle is only ever fed inputs
(from synth or from states read back after upload); expected values never
come from the CUDA path."""
import numpy as np
import torch

import synth
from oracle.solver import NestedSolver


def gpu():
    from paper_1206_0389_gb300 import lbm
    return lbm


def make_pair(model, storage, nb, periodic_x=True, refine=(), omega=1.6, cs=0.0, walls=0, slip=0,
              outlet=0, nozzle=None):
    lbm = gpu()
    ctx = lbm.lbm_create(model, storage, nb, periodic_x, [np.asarray(r) for r in refine], omega, cs,
                         walls=walls, slip=slip, outlet=outlet, nozzle=nozzle)
    orc = NestedSolver(model, nb, periodic_x=periodic_x,
                       refine=[torch.as_tensor(np.asarray(r)).bool() for r in refine],
                       omega=omega, cs=cs, walls=walls, slip=slip, outlet=outlet, nozzle=nozzle)
    return ctx, orc


def upload_same_state(ctx, orc, states):
    """Upload per-level dense states to the GPU, read back the rounded values
    and give exactly those to the oracle."""
    lbm = gpu()
    got = []
    for l, f in enumerate(states):
        lbm.lbm_set_state(ctx, l, f)
        back = lbm.lbm_get_state(ctx, l)
        orc.set_state(l, torch.from_numpy(back))
        got.append(back)
    return got


def init_both(ctx, orc, fields):
    """init_equilibrium on both sides from per-level (rho, u) fields."""
    lbm = gpu()
    for l, (rho, u) in enumerate(fields):
        lbm.lbm_init_equilibrium(ctx, l, rho, u)
        orc.init_equilibrium(l, torch.from_numpy(rho), torch.from_numpy(u))


def valid_mask(orc, l):
    lv = orc.levels[l]
    return orc.real(l, lv.valid).numpy()


def compare_levels(ctx, orc, rel=None, abs_=None, levels=None):
    """Max |f_gpu - f_oracle| over cells holding a value of each level.
    Returns (max abs diff, max |f_oracle|) over all compared levels."""
    lbm = gpu()
    worst, scale = 0.0, 0.0
    for l in (range(len(orc.levels)) if levels is None else levels):
        fg = lbm.lbm_get_state(ctx, l)
        fo = orc.state(l).numpy()
        m = valid_mask(orc, l)
        d = np.abs(fg[:, m] - fo[:, m])
        assert np.isfinite(fg[:, m]).all()
        worst = max(worst, float(d.max()))
        scale = max(scale, float(np.abs(fo[:, m]).max()))
    return worst, scale


def shear_base(model):
    Q = 19 if model == "d3q19" else 27
    if model == "d3q19":
        return None, Q
    from oracle.lattice import weights
    return weights(27).numpy(), Q


def random_state(model, shape, seed, amp):
    """Random far-from-equilibrium distributions for a level of the given
    (NX, NY, NZ); D3Q19 gets a fluctuation state, D3Q27 a full state."""
    NX, NY, NZ = shape
    if model == "d3q19":
        return synth.random_fluctuations(19, (NZ, NY, NX), seed, amp=amp)
    return synth.random_distributions(27, (NZ, NY, NX), seed, amp=amp)

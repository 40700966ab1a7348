"""Long-horizon parity on nested grids: 1000 coarse steps of a shear wave
carried by a uniform drift through the refined bands of 2- and 3-level
grids (both collision models, time nesting with 2:1 refinement, Sections 1
and 3.2), every level's velocity field on the GPU against the float64
oracle's.  The oracle's result is stored in tests/golden/nested_long_*.txt,
written by tests/golden/make_nested_long.py from the oracle alone (the
oracle takes minutes to half an hour per case on the host).

Gates: velocity relative L2 after 1000 coarse steps <= 1e-4 for FP32
storage and <= 1e-9 for FP64, the L2 taken over every cell holding a value
of a level, weighted by the cell volume 8^-l, relative to the wave (the
velocity minus the uniform drift)."""
import importlib.util
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_spec = importlib.util.spec_from_file_location(
    "make_nested_long", os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_nested_long.py"))
M = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(M)


def run_gpu(case, storage):
    from paper_1206_0389_gb300 import lbm
    c = M.CASES[case]
    nb, ref = M.grid(c["levels"])
    ctx = lbm.lbm_create(c["model"], storage, nb, True, ref, M.OMEGA, M.cs_of(c["model"]))
    for l, (rho, u) in enumerate(M.initial_fields(nb, c["levels"])):
        lbm.lbm_init_equilibrium(ctx, l, rho, u)
    lbm.lbm_step(ctx, M.STEPS)
    out = [lbm.lbm_macroscopic(ctx, l) for l in range(c["levels"])]
    lbm.lbm_destroy(ctx)
    return out


def compare(case, fields):
    gold = M.read(case)
    num = den = 0.0
    for l, (rho_g, u_g) in enumerate(fields):
        rows, vals = gold[l]
        held = np.where(~np.isnan(rho_g).all(axis=(0, 2)))[0]
        assert np.array_equal(held, rows), (l, held, rows)   # same cells hold values
        ug = u_g[:, :, rows, :]
        assert np.isfinite(ug).all()
        uo = vals[:, 1:4].T[:, None, :, None]                 # [3][1][rows][1], invariant in x, z
        w = 8.0 ** -l
        num += w * float(((ug - uo) ** 2).sum())
        wave = np.broadcast_to(uo - np.array([0.0, M.DRIFT, 0.0])[:, None, None, None], ug.shape)
        den += w * float((wave ** 2).sum())
    return np.sqrt(num / den)


@pytest.mark.parametrize("case", sorted(M.CASES))
@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_long_horizon_nested_parity(case, storage, tol):
    err = compare(case, run_gpu(case, storage))
    print(case, storage, "velocity relative L2 after %d coarse steps: %.3e" % (M.STEPS, err))
    assert err <= tol, err

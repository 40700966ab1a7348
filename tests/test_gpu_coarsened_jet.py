"""The paper-scale 3-level jet's layout on a 4x-coarsened domain (coarse
128 x 64 x 64, nozzle D = 8, D3Q27 FCLB, inflow with a seeded 1 %
perturbation, zero-gradient outflow; Section 3.2's round jet on a
time-nested grid) run from rest on the GPU against the float64 oracle's run
stored in tests/golden/coarsened_jet.txt (written by
tests/golden/make_coarsened_jet.py from the oracle alone; about two minutes
of host time per coarse step).  Compared: per level, the time mean of u_x
over the second half of the run on the cells around the jet axis (the
paper's centreline quantity, Section 3.3), u_x there after the last step,
and rho and u of sampled cells of every level after the last step.

Gates (relative to the largest |u| of the compared values over all levels,
about u_in): FP64 storage 1e-9; FP32 storage 1e-4 (the velocity tolerance of
the long-run tests)."""
import importlib.util
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_spec = importlib.util.spec_from_file_location(
    "make_coarsened_jet", os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_coarsened_jet.py"))
C = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(C)


def run_gpu(storage, steps):
    from paper_1206_0389_gb300 import lbm
    flags, (y0, z0) = C.grid()
    ctx = lbm.lbm_create("d3q27", storage, C.NB, False, flags, C.OMEGA, 0.0)
    lbm.lbm_set_inflow(ctx, y0, z0, C.D, C.U_IN, C.PERTURB, C.SEED)
    L = len(flags) + 1
    lbm.lbm_step(ctx, steps // 2)
    lbm.lbm_stats_reset(ctx)
    for _ in range(steps - steps // 2):
        lbm.lbm_step(ctx, 1)
        lbm.lbm_stats_accumulate(ctx)
    out = {"mean": {}, "final": {}, "cells": {}}
    for l in range(L):
        jy, jz = C.axis_rows(l, y0, z0)
        mean, _, n = lbm.lbm_stats_get(ctx, l)
        assert n == steps - steps // 2
        out["mean"][l] = mean[1, jz:jz + 2, jy:jy + 2, :].mean(axis=(0, 1))
        rho, u = lbm.lbm_macroscopic(ctx, l)
        out["final"][l] = u[0, jz:jz + 2, jy:jy + 2, :].mean(axis=(0, 1))
        out["cells"][l] = (rho.reshape(-1), u.reshape(3, -1))
    lbm.lbm_destroy(ctx)
    return out


@pytest.mark.parametrize("storage,tol", [("f64", 1e-9), ("f32", 1e-4)])
def test_coarsened_paper_jet_against_stored_oracle_run(storage, tol):
    gold = C.read()
    got = run_gpu(storage, gold["steps"])
    # one scale for every level: after the stored run the jet has not reached
    # level 0's part of the axis, whose values there are round-off (~1e-15)
    scale = max([np.abs(uo).max() for kind in ("mean", "final") for _, uo in gold[kind].values()] +
                [np.abs(vals[:, 1:]).max() for _, vals in gold["cells"].values()])
    assert scale > 0.01, scale
    worst = {}
    for kind in ("mean", "final"):
        for l, (xs, uo) in gold[kind].items():
            ug = got[kind][l][xs]
            assert np.isfinite(ug).all()
            worst["%s_%d" % (kind, l)] = float(np.abs(ug - uo).max() / scale)
    for l, (idx, vals) in gold["cells"].items():
        rho, u = got["cells"][l]
        gu = np.stack([rho[idx], u[0][idx], u[1][idx], u[2][idx]], axis=1)
        worst["cells_u_%d" % l] = float(np.abs(gu[:, 1:] - vals[:, 1:]).max() / scale)
        worst["cells_rho_%d" % l] = float(np.abs(gu[:, 0] - vals[:, 0]).max())
    print(storage, "after %d coarse steps:" % gold["steps"], {k: "%.2e" % v for k, v in worst.items()})
    assert max(worst.values()) <= tol, worst

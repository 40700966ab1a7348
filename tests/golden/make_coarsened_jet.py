"""Writes the expected values of the coarsened paper-jet parity test
(tests/test_gpu_coarsened_jet.py) with the float64 oracle only.

The 3-level round jet of the paper's scale (Section 3.2: a nozzle jet at
Re 10^4 on a time-nested grid, D3Q27 FCLB) on a 4x-coarsened domain: coarse
128 x 64 x 64 cells in 8^3 blocks, nozzle D = 8 on the axis at x = 0, top-hat
inflow u = 0.05 with a 1 % seeded perturbation, zero-gradient outflow,
nu_c = u D / Re; level 1 the disc r < 12 coarse cells over x < 48, level 2
the disc r < 8 over x < 24 (a literal 4x coarsening of the paper-scale rings
is thinner than one block).  The oracle runs STEPS coarse steps from rest;
the file holds, per level, the time mean of u_x over the second half of the
run on the cells nearest the jet axis (the mean of the 2 x 2 cells around it,
per x layer that holds a value of the level), u_x there after the last step,
and rho and u of SAMPLES cells per level drawn with a fixed seed among the
cells holding a value of the level, after the last step.

Usage: python tests/golden/make_coarsened_jet.py [steps]   (default STEPS)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
PATH = os.path.join(HERE, "coarsened_jet.txt")

NB = (16, 8, 8)
D, U_IN, PERTURB, SEED, RE = 8.0, 0.05, 0.01, 5120, 1e4
STEPS, SAMPLES = 500, 400
NU_C = U_IN * D / RE
OMEGA = 1.0 / (3 * NU_C + 0.5)


def grid():
    """(refine flags per level, axis (y0, z0) in coarse cells)."""
    sys.path.insert(0, ROOT)
    import synth
    return synth.jet_three_level(*NB, r1=(0.0, 12.0), r2=(0.0, 8.0), x1=(0, 48), x2=(0, 24))


def axis_rows(level, y0, z0):
    """Level-local (y, z) indices of the 2 x 2 cells around the axis."""
    s = 1 << level
    jy, jz = int(round(y0 * s)) - 1, int(round(z0 * s)) - 1
    return jy, jz


def sample_cells(valid, rng):
    """SAMPLES flat indices (z, y, x order) of cells holding a value."""
    idx = np.flatnonzero(valid.ravel())
    return np.sort(rng.choice(idx, size=min(SAMPLES, idx.size), replace=False))


def read():
    """{"mean": {l: (xs, u)}, "final": {l: (xs, u)}, "cells": {l: (idx, [n][4])}, "steps": n}."""
    out = {"mean": {}, "final": {}, "cells": {}}
    for line in open(PATH):
        if line.startswith("# steps"):
            out["steps"] = int(line.split()[2])
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        kind, l = v[0], int(v[1])
        if kind in ("mean", "final"):
            xs, us = out[kind].setdefault(l, ([], []))
            xs.append(int(v[2]))
            us.append(float(v[3]))
        else:
            idx, vals = out["cells"].setdefault(l, ([], []))
            idx.append(int(v[2]))
            vals.append([float(t) for t in v[3:7]])
    for k in ("mean", "final", "cells"):
        out[k] = {l: (np.array(a), np.array(b)) for l, (a, b) in out[k].items()}
    return out


def run(steps):
    sys.path.insert(0, ROOT)
    import torch
    from oracle.solver import NestedSolver
    flags, (y0, z0) = grid()
    s = NestedSolver("d3q27", NB, periodic_x=False, refine=[torch.from_numpy(f) for f in flags],
                     omega=OMEGA, cs=0.0)
    s.set_inflow(y0, z0, D, U_IN, PERTURB, SEED)
    L = len(s.levels)
    sums = [None] * L
    n = 0
    for t in range(1, steps + 1):
        s.step(1)
        if t > steps // 2:
            n += 1
            for l in range(L):
                _, u = s.macroscopic(l)
                jy, jz = axis_rows(l, y0, z0)
                ax = u[0, jz:jz + 2, jy:jy + 2, :].mean(dim=(0, 1)).numpy()
                sums[l] = ax if sums[l] is None else sums[l] + ax
        if t % 10 == 0:
            print("step", t, flush=True)
    rng = np.random.default_rng(SEED)
    with open(PATH, "w") as fh:
        fh.write("# coarsened paper jet: oracle (float64), D3Q27 FCLB, coarse blocks %s, 3 levels, D = %g, "
                 "u_in = %g, perturbation %g (seed %d), nu_c = %g (omega_0 = %.17g)\n"
                 % (NB, D, U_IN, PERTURB, SEED, NU_C, OMEGA))
        fh.write("# steps %d\n" % steps)
        fh.write("# written by tests/golden/make_coarsened_jet.py; rows: 'mean' level x <u_x> on the axis "
                 "(steps %d..%d), 'final' level x u_x on the axis, 'cell' level index rho u_x u_y u_z\n"
                 % (steps // 2 + 1, steps))
        for l in range(L):
            rho, u = s.macroscopic(l)
            jy, jz = axis_rows(l, y0, z0)
            fin = u[0, jz:jz + 2, jy:jy + 2, :].mean(dim=(0, 1)).numpy()
            mean = sums[l] / n
            for x in range(fin.size):
                if np.isfinite(fin[x]):
                    fh.write("mean %d %d %.17g\n" % (l, x, mean[x]))
                    fh.write("final %d %d %.17g\n" % (l, x, fin[x]))
            rho, u = rho.numpy(), u.numpy()
            for i in sample_cells(~np.isnan(rho), rng):
                z, rem = divmod(int(i), rho.shape[1] * rho.shape[2])
                y, x = divmod(rem, rho.shape[2])
                fh.write("cell %d %d %s\n" % (l, i, " ".join("%.17g" % v for v in
                                                            (rho[z, y, x], u[0, z, y, x], u[1, z, y, x],
                                                             u[2, z, y, x]))))


if __name__ == "__main__":
    run(int(sys.argv[1]) if len(sys.argv) > 1 else STEPS)
    print("wrote", PATH)

"""Writes the expected values of the long-horizon nested-grid parity tests
(tests/test_gpu_long_nested.py) with the float64 oracle only.

Each case is a shear wave u_x = A sin(2 pi y / NY + phi0) carried by a
uniform drift u_y = U through refined bands of a grid that is one coarse
block wide in x and z (periodic in every direction): time nesting with 2:1
refinement after Yu et al. (Sections 1 and 3.2), the drift taking the wave
through every interface several times over the run.  The flow is invariant
along x and z, so a level's state is fixed by its profile over y: the file
holds, at two times, for every level and every row y of cells that hold a
value of the level, rho and u (the oracle's macroscopic fields; the cells of
a row agree to round-off, and the row mean is kept).  The two times are
1000 steps of the finest level (1000 / 2^(L-1) coarse steps) and 1000
coarse steps.

Usage: python tests/golden/make_nested_long.py [case ...]   (default: all)
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

# coarse steps, wave amplitude, drift, level-0 omega, Smagorinsky constant
STEPS, AMP, DRIFT, OMEGA = 1000, 0.02, 0.05, 1.8


def checkpoints(levels):
    """Coarse steps at which the state is recorded: 1000 steps of the finest
    level, and STEPS coarse steps."""
    return (STEPS >> (levels - 1), STEPS)


def grid(levels):
    """(nb, refine flags per level [z][y][x]) of the banded grids: 2 levels
    on 1 x 4 x 1 coarse blocks (level 1 = coarse block rows 1..2), 3 levels
    on 1 x 6 x 1 (level 1 = rows 2..3, level 2 = level-1 rows 5..6; every
    block touching a refined level-1 block is a level-1 block)."""
    if levels == 2:
        nb = (1, 4, 1)
        r0 = np.zeros((1, 4, 1), dtype=bool)
        r0[:, 1:3, :] = True
        return nb, [r0]
    nb = (1, 6, 1)
    r0 = np.zeros((1, 6, 1), dtype=bool)
    r0[:, 2:4, :] = True
    r1 = np.zeros((2, 12, 2), dtype=bool)
    r1[:, 5:7, :] = True
    return nb, [r0, r1]


CASES = {"slab2_%s" % m: dict(model=m, levels=2) for m in ("d3q19", "d3q27")}
CASES.update({"slab3_%s" % m: dict(model=m, levels=3) for m in ("d3q19", "d3q27")})


def cs_of(model):
    return 0.1 if model == "d3q19" else 0.0


def initial_fields(nb, levels):
    """Per level (rho, u) of the drifting wave, the zero of u_x on the lower
    level-0/1 interface at t = 0."""
    NY0 = 8 * nb[1]
    out = []
    for l in range(levels):
        s = 1 << l
        NX, NY, NZ = 8 * nb[0] * s, 8 * nb[1] * s, 8 * nb[2] * s
        y = (np.arange(NY) + 0.5) / s                     # coarse units
        y_if = 8.0 * (1 if levels == 2 else 2)            # lower level-0/1 interface
        prof = AMP * np.sin(2 * math.pi * (y - y_if) / NY0)
        u = np.zeros((3, NZ, NY, NX))
        u[0] = prof[None, :, None]
        u[1] = DRIFT
        out.append((np.ones((NZ, NY, NX)), u))
    return out


def path(case):
    return os.path.join(HERE, "nested_long_%s.txt" % case)


def read(case):
    """{coarse step: {level: (rows, [n][4] of rho, u_x, u_y, u_z)}} from a
    case's file."""
    data = {}
    for line in open(path(case)):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        t, l, y = int(v[0]), int(v[1]), int(v[2])
        rows, vals = data.setdefault(t, {}).setdefault(l, ([], []))
        rows.append(y)
        vals.append([float(x) for x in v[3:7]])
    return {t: {l: (np.array(r), np.array(a)) for l, (r, a) in d.items()} for t, d in data.items()}


def run(case):
    sys.path.insert(0, ROOT)
    import torch
    from oracle.solver import NestedSolver
    c = CASES[case]
    nb, ref = grid(c["levels"])
    s = NestedSolver(c["model"], nb, periodic_x=True, refine=[torch.from_numpy(r) for r in ref],
                     omega=OMEGA, cs=cs_of(c["model"]))
    for l, (rho, u) in enumerate(initial_fields(nb, c["levels"])):
        s.init_equilibrium(l, torch.from_numpy(rho), torch.from_numpy(u))
    with open(path(case), "w") as fh:
        fh.write("# %s: oracle (float64), %s, %d levels, coarse blocks %s, refine rows as in grid(), "
                 "omega_0 = %g, Cs = %g\n" % (case, c["model"], c["levels"], nb, OMEGA, cs_of(c["model"])))
        fh.write("# u_x = %g sin(2 pi (y - y_if) / NY0), drift u_y = %g, after %s coarse steps\n"
                 % (AMP, DRIFT, " and ".join(str(t) for t in checkpoints(c["levels"]))))
        fh.write("# written by tests/golden/make_nested_long.py; columns: coarse step, level, row y, rho, u_x, "
                 "u_y, u_z\n")
        for t in checkpoints(c["levels"]):
            s.step(t - s.coarse_step)
            write_state(fh, s, c["levels"], t)


def write_state(fh, s, levels, t):
    """Rows of every level after coarse step t."""
    for l in range(levels):
        rho, u = s.macroscopic(l)
        rho, u = rho.numpy(), u.numpy()
        for y in range(rho.shape[1]):
            row = rho[:, y, :]
            if np.isnan(row).all():
                continue
            assert not np.isnan(row).any()
            # the flow is invariant along x and z (to round-off: the oracle's
            # batched operations may round cells of a row apart in the last
            # bit): one value per row, the row mean
            vals = [row.mean()] + [u[a, :, y, :].mean() for a in range(3)]
            assert np.abs(row - vals[0]).max() <= 1e-13
            assert all(np.abs(u[a, :, y, :] - vals[1 + a]).max() <= 1e-13 for a in range(3))
            fh.write("%d %d %d %s\n" % (t, l, y, " ".join("%.17g" % v for v in vals)))


if __name__ == "__main__":
    for case in (sys.argv[1:] or sorted(CASES)):
        run(case)
        print("wrote", path(case))

"""CPU tests of the C ABI: the library loads, exports every symbol declared in
include/lbm.h, plans grids on the host exactly like the oracle's masks, and
reports errors without touching a GPU."""
import os
import re

import numpy as np
import pytest
import torch

import synth
from oracle.grid import build_levels
from oracle.solver import NestedSolver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
lbm = pytest.importorskip("paper_1206_0389_gb300.lbm")


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm.EXPORTED)


def slab_refine(nb, lo, hi):
    r = np.zeros((nb[2], nb[1], nb[0]), dtype=bool)
    r[:, :, lo:hi] = True
    return r


GRIDS = {
    "slab2": ((4, 2, 2), True, [slab_refine((4, 2, 2), 1, 3)]),
    "slab2_open": ((4, 2, 2), False, [slab_refine((4, 2, 2), 0, 2)]),
    "three": ((3, 2, 2), True, None),
    "jet_small": ((6, 4, 4), False, None),
}


def grid(name):
    nb, px, ref = GRIDS[name]
    if name == "three":
        r0 = np.zeros((2, 2, 3), dtype=bool)
        r0[:, :, 0:2] = True
        r1 = np.zeros((4, 4, 6), dtype=bool)
        r1[1:3, 1:3, 1:3] = True
        ref = [r0, r1]
    if name == "jet_small":
        flags, _ = synth.jet_two_level(6, 4, 4, radius=12.0)
        ref = flags
    return nb, px, ref


@pytest.mark.parametrize("name", list(GRIDS))
def test_plan_counts_match_oracle_masks(name):
    nb, px, ref = grid(name)
    info = lbm.lbm_plan(nb, px, ref, "d3q27", "f32")
    lv = build_levels(nb, px, [torch.from_numpy(r) for r in ref])
    assert info.levels == len(lv)
    upd = 0
    for l, L in enumerate(lv):
        assert info.active_cells[l] == int(L.active.sum())
        assert info.updated_cells[l] == int(L.update.sum())
        assert info.hidden_cells[l] == int((L.hidden1 | L.hidden2).sum())
        assert info.ghost_cells[l] == int(L.ghost.sum())
        assert info.level_blocks[l] == int(L.region_blocks.sum())
        upd += int(L.update.sum()) << l
    assert info.updates_per_coarse_step == upd


def test_jet_plan_sizes():
    flags, _ = synth.jet_two_level()
    info = lbm.lbm_plan((48, 24, 24), False, flags, "d3q27", "f32")
    assert info.active_cells[0] == 13_369_344 and info.active_cells[1] == 6_291_456
    assert info.active_updates_per_coarse_step == 25_952_256


@pytest.mark.parametrize("model,Q", [("d3q27", 27), ("d3q19", 19)])
def test_plan_rejects_a_cross_section_just_past_the_32_bit_offset_limit(model, Q):
    """The stream-collide kernels form x / y neighbour offsets in 32 bits
    (one z layer of blocks below 2^31 stored values; z neighbours use 64-bit
    bases): the planner accepts the largest such layer and refuses the next."""
    from paper_1206_0389_gb300 import lbm
    limit = (1 << 31) // (512 * Q)          # blocks per z layer that still fit
    nbx = 512
    ok_y, bad_y = limit // nbx, limit // nbx + 1
    assert nbx * ok_y * 512 * Q < 1 << 31 <= nbx * bad_y * 512 * Q
    info = lbm.lbm_plan((nbx, ok_y, 1), True, [], model, "f16")
    assert info.blocks[0] == nbx * ok_y
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_plan((nbx, bad_y, 1), True, [], model, "f16")
    assert e.value.status == lbm.LBM_ERR_ARG


def test_plan_rejects_bad_grids():
    r0 = np.zeros((2, 2, 3), dtype=bool)
    r0[:, :, 0:2] = True
    r1 = np.zeros((4, 4, 6), dtype=bool)
    r1[1:3, 1:3, 2:4] = True   # x block 3 touches the level-1 boundary at x = 4
    with pytest.raises(ValueError):
        build_levels((3, 2, 2), True, [torch.from_numpy(r0), torch.from_numpy(r1)])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plan((3, 2, 2), True, [r0, r1])
    bad = np.zeros((2, 2, 3), dtype=bool)
    with pytest.raises(lbm.LbmError):           # a level that refines nothing
        lbm.lbm_plan((3, 2, 2), True, [bad, np.zeros((4, 4, 6), dtype=bool)])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plan((0, 2, 2), True, [])


@pytest.mark.parametrize("walls,slip,px,ok", [(0, 0, True, True), (3, 0, True, True), (12, 12, True, True),
                                               (15, 9, True, True), (1, 0, True, False), (6, 0, True, False),
                                               (3, 4, True, False), (16, 0, True, False), (16, 0, False, True),
                                               (63, 12, False, True), (48, 16, False, False), (64, 0, False, False)])
def test_plan_wall_rules_match_oracle(walls, slip, px, ok):
    """y/z walls come in pairs per axis, slip is a subset of them, x walls
    need a non-periodic x: the planner and the oracle accept and reject the
    same settings."""
    try:
        NestedSolver("d3q27", (2, 2, 2), periodic_x=px, walls=walls, slip=slip)
        oracle_ok = True
    except ValueError:
        oracle_ok = False
    assert oracle_ok == ok
    if ok:
        lbm.lbm_plan((2, 2, 2), px, [], walls=walls, slip=slip)
    else:
        with pytest.raises(lbm.LbmError):
            lbm.lbm_plan((2, 2, 2), px, [], walls=walls, slip=slip)


def test_plan_rejects_refinement_next_to_walls():
    r = np.zeros((3, 3, 4), dtype=bool)
    r[1, 1, 0:2] = True                      # one block away from every y/z face
    lbm.lbm_plan((4, 3, 3), False, [r], walls=15, slip=8)
    NestedSolver("d3q27", (4, 3, 3), periodic_x=False, refine=[torch.from_numpy(r)], walls=15)
    for bad_wall in (3, 12):
        r2 = r.copy()
        if bad_wall == 3:
            r2[1, 0, 0] = True                   # touches the low y face
        else:
            r2[2, 1, 0] = True                   # touches the high z face
        with pytest.raises(lbm.LbmError):
            lbm.lbm_plan((4, 3, 3), False, [r2], walls=bad_wall)
        with pytest.raises(ValueError):
            NestedSolver("d3q27", (4, 3, 3), periodic_x=False, refine=[torch.from_numpy(r2)],
                         walls=bad_wall)
        # the same refinement is fine while that axis stays periodic
        lbm.lbm_plan((4, 3, 3), False, [r2], walls=15 - bad_wall)


def test_plan_outlet_rules_match_oracle():
    """The pressure outlet needs a non-periodic x axis and keeps refined blocks
    one block away from its face; its ghost column doubles the level-0
    boundary cells."""
    r = np.zeros((2, 2, 3), dtype=bool)
    r[:, :, 0] = True
    info = lbm.lbm_plan((3, 2, 2), False, [r], outlet=1)
    plain = lbm.lbm_plan((3, 2, 2), False, [r])
    assert info.bc_cells[0] == plain.bc_cells[0] + 16 * 16
    NestedSolver("d3q27", (3, 2, 2), periodic_x=False, refine=[torch.from_numpy(r)], outlet=1)
    bad = np.zeros((2, 2, 3), dtype=bool)
    bad[:, :, 2] = True
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plan((3, 2, 2), False, [bad], outlet=1)
    with pytest.raises(ValueError):
        NestedSolver("d3q27", (3, 2, 2), periodic_x=False, refine=[torch.from_numpy(bad)], outlet=1)
    lbm.lbm_plan((3, 2, 2), False, [bad])            # fine with the zero-gradient outflow
    for bad_args in (dict(periodic_x=True, outlet=1), dict(periodic_x=False, outlet=2)):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_plan((3, 2, 2), bad_args["periodic_x"], [], outlet=bad_args["outlet"])
        with pytest.raises(ValueError):
            NestedSolver("d3q27", (3, 2, 2), **bad_args)


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_plan_nozzle_matches_oracle(model):
    """The planner and the oracle pick the same level for the nozzle and agree
    on its solid cells, its links and the remaining active cells."""
    cases = [((5, 5, 5), [], (20.0, 20.0, 4.3, 10.25, 24.0), 0)]
    r = np.zeros((5, 5, 5), dtype=bool)
    r[1:4, 1:4, 1:4] = True
    cases.append(((5, 5, 5), [r], (20.0, 20.0, 1.3, 18.25, 21.5), 1))
    for nb, ref, noz, level in cases:
        info = lbm.lbm_plan(nb, False, ref, model, "f32", nozzle=noz)
        s = NestedSolver(model, nb, periodic_x=False, refine=[torch.from_numpy(x) for x in ref], nozzle=noz)
        assert info.nozzle_level == s.body.l == level
        assert info.solid_cells == int(s.body.solid.sum())
        assert info.nozzle_links == len(s.body.q)
        for l, lv in enumerate(s.levels):
            assert info.active_cells[l] == int(lv.active.sum())
            assert info.updated_cells[l] == int(lv.update.sum())
    with pytest.raises(lbm.LbmError):                 # next to the level-1 interface
        lbm.lbm_plan((5, 5, 5), False, [r], model, "f32", nozzle=(20.0, 20.0, 4.3, 10.25, 24.0))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plan((5, 5, 5), False, [], model, "f32", nozzle=(20.0, 20.0, 4.3, 24.0, 10.0))
    for bad in ((20.0, 20.0, 4.3, 10.0, 1e300), (float("nan"), 20.0, 4.3, 10.0, 20.0), (20.0, 20.0, 1e7, 10.0, 20.0)):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_plan((5, 5, 5), False, [], model, "f32", nozzle=bad)
    assert lbm.lbm_plan((5, 5, 5), False, [], model, "f32").nozzle_level == -1
    r2 = np.zeros((5, 5, 5), dtype=bool)
    r2[2, 2, 4] = True                      # refined block next to the level-0 nozzle's blocks
    with pytest.raises(lbm.LbmError):
        lbm.lbm_plan((5, 5, 5), False, [r2], model, "f32", nozzle=(20.0, 20.0, 4.3, 10.25, 24.0))


def test_create_without_gpu_reports_cuda_error():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create("d3q19", "f32", (2, 2, 2))
    assert e.value.status == lbm.LBM_ERR_CUDA
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create("d3q19", "f32", (2, 2, 2), omega=2.5)
    assert e.value.status == lbm.LBM_ERR_ARG


def test_jet_fit_matches_oracle_on_the_host():
    """lbm_jet_fit (host arithmetic in the library) against the oracle's
    statement on noisy Gaussian, parabolic, uniform and empty profiles."""
    import math
    from oracle.jetstats import jet_fit, radial_profile
    N, Y0 = 96, 48.3
    y = np.arange(N) + 0.5
    r = np.sqrt((y[None, :] - Y0) ** 2 + (y[:, None] - Y0) ** 2)
    rng = np.random.default_rng(5)
    fields = [0.05 * np.exp(-(r / 9.0) ** 2) * (1 + 0.01 * rng.standard_normal(r.shape)),
              np.where(r < 30, 0.04 * (1 - (r / 30) ** 2), 0.0),
              np.full_like(r, 0.03)]
    for fm in fields:
        mean = np.repeat(fm[:, :, None], 2, axis=2)
        var = np.repeat((1e-5 * np.abs(fm))[:, :, None], 2, axis=2)
        for dr in (1.0, 1.7):
            pm, pv, pc = radial_profile(mean, var, 0, Y0, Y0, dr, 40, [0.5])
            o = jet_fit(pm[0], pv[0], pc[0], dr)
            g = lbm.lbm_jet_fit(pm[0], pv[0], pc[0], dr)
            for a, b in zip(o, g):
                assert (math.isnan(a) and math.isnan(b)) or abs(a - b) <= 1e-12 * max(1.0, abs(a))
    empty = lbm.lbm_jet_fit(np.full(5, np.nan), np.full(5, np.nan), np.zeros(5, dtype=np.int64), 1.0)
    assert all(math.isnan(v) for v in empty)


def test_plan_nozzle_random_placements_match_oracle():
    """Random nozzle placements (radius, ends and axis off the cell lattice):
    the planner and the oracle agree on the level, the solid cells and the
    number of links, or both reject the placement."""
    rng = np.random.default_rng(20)
    agree = 0
    for _ in range(12):
        R = float(rng.uniform(1.2, 6.0))
        y0, z0 = (float(v) for v in rng.uniform(17.0, 23.0, size=2))
        x0 = float(rng.uniform(9.0, 14.0))
        x1 = float(rng.uniform(x0 + 2.0, 30.0))
        noz = (y0, z0, R, x0, x1)
        try:
            s = NestedSolver("d3q19", (5, 5, 5), periodic_x=False, nozzle=noz)
        except ValueError:
            with pytest.raises(lbm.LbmError):
                lbm.lbm_plan((5, 5, 5), False, [], "d3q19", "f32", nozzle=noz)
            continue
        info = lbm.lbm_plan((5, 5, 5), False, [], "d3q19", "f32", nozzle=noz)
        assert info.nozzle_level == s.body.l
        assert info.solid_cells == int(s.body.solid.sum())
        assert info.nozzle_links == len(s.body.q)
        agree += 1
    assert agree >= 4

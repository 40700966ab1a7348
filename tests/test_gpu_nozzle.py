"""GPU parity of the nozzle (Section 3.2: a cylinder with Bouzidi
interpolated no-slip walls whose downstream cap emits the jet) against the
FP64 oracle, through the C ABI.

Tolerances as in the other parity tests: F64 storage <= 1e-12 absolute; F32
<= 1e-6 of max|f| per step; F16 four half-precision roundings of the largest
(f - w)/w per step."""
import numpy as np
import pytest
import torch

import synth
from tests.helpers import (compare_levels, gpu, init_both, make_pair, random_state,
                           upload_same_state, valid_mask)

pytestmark = pytest.mark.gpu

MODELS = ["d3q19", "d3q27"]
NOZ = (20.0, 20.0, 4.3, 10.25, 24.0)          # y0, z0, R, x0, x1 on level 0 of a 40^3 grid
NOZ1 = (20.0, 20.0, 1.3, 18.25, 21.5)         # on level 1 of the nested grid below
INFLOW = (20.0, 20.0, 7.0, 0.05, 0.02, 41)


def dims(nb, l=0):
    return tuple(8 * n << l for n in nb)


def nested_grid():
    r = np.zeros((5, 5, 5), dtype=bool)
    r[1:4, 1:4, 1:4] = True
    return (5, 5, 5), [r]


def pair(model, storage, nb, refine=(), nozzle=NOZ, omega=1.7, cs=0.18, **kw):
    ctx, orc = make_pair(model, storage, nb, False, refine, omega=omega, cs=cs, nozzle=nozzle, **kw)
    gpu().lbm_set_inflow(ctx, *INFLOW)
    orc.set_inflow(*INFLOW)
    return ctx, orc


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("variant", ["128,1,0", "256,4,1"])
def test_nozzle_single_level_f64(model, variant, monkeypatch):
    """Two steps from a random far-from-equilibrium state: Bouzidi links on
    the side and the upstream cap (both branches of q, and the half-way
    fallback), the inflow on the downstream cap, the closed face x = 0."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (5, 5, 5)
    ctx, orc = pair(model, "f64", nb)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 23, 0.2)])
    gpu().lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    rg, ug = gpu().lbm_macroscopic(ctx, 0)
    ro, uo = orc.macroscopic(0)
    assert np.array_equal(np.isnan(rg), np.isnan(ro.numpy()))       # solid cells hold no value
    ok = ~np.isnan(rg)
    assert np.abs(ug[:, ok] - uo.numpy()[:, ok]).max() < 1e-12
    gpu().lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_nozzle_on_the_fine_level_f64(model):
    """The nozzle on level 1 of a nested grid (two fine substeps per coarse
    step), with the FP64 audit."""
    lbm = gpu()
    nb, ref = nested_grid()
    ctx, orc = pair(model, "f64", nb, ref, nozzle=NOZ1)
    fields = [synth.taylor_green_3d(lv.NY, 0.03, shape=(lv.NX, lv.NY, lv.NZ)) for lv in orc.levels]
    init_both(ctx, orc, fields)
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    mg = lbm.lbm_mass_momentum(ctx)
    mo = orc.mass_momentum().numpy()
    assert np.abs(mg - mo).max() <= 1e-10 * max(1.0, np.abs(mo).max())
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_nozzle_per_step_reduced_precision(model, storage):
    lbm = gpu()
    nb = (5, 5, 5)
    ctx, orc = pair(model, storage, nb, omega=1.9, cs=0.1)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 29, 0.2)])
    lbm.lbm_step(ctx, 1)
    orc.set_state(0, torch.from_numpy(lbm.lbm_get_state(ctx, 0)))
    orc.coarse_step = lbm.lbm_get_step(ctx)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    m = valid_mask(orc, 0)
    fg = lbm.lbm_get_state(ctx, 0)[:, m]
    fo = orc.state(0).numpy()[:, m]
    if storage == "f32":
        assert np.abs(fg - fo).max() / np.abs(fo).max() <= 1e-6
    else:
        from oracle.lattice import weights
        Q = 19 if model == "d3q19" else 27
        w = weights(Q).numpy()
        shift = w if model == "d3q27" else np.zeros_like(w)
        err = np.abs(fg - fo) / w[:, None]
        bound = 4 * 2.0 ** -11 * (np.abs(fo - shift[:, None]) / w[:, None]).max() + 1e-6
        assert err.max() <= bound, (err.max(), bound)
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_nozzle_graph_and_direct_launches_agree(model, storage, monkeypatch):
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,1,0")
    lbm = gpu()
    nb, ref = nested_grid()
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, storage, nb, False, ref, 1.7, 0.18, nozzle=NOZ1)
        lbm.lbm_set_inflow(ctx, *INFLOW)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 3)
        lbm.lbm_sync(ctx)
        out.append([lbm.lbm_get_raw_state(ctx, l) for l in range(2)])
        lbm.lbm_destroy(ctx)
    for l in range(2):
        assert np.array_equal(out[0][l], out[1][l])


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_level0_nozzle_graph_and_direct_launches_agree(model, storage, monkeypatch):
    """The nozzle on level 0 of a nested grid (a refined patch downstream):
    for FP16 storage the coarse-step graph starts the level-0 update after
    the level-0 inflow and the nozzle links, on a branch beside the fine
    level; the same bits as the sequential launches (one launch shape)."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,1,0")
    lbm = gpu()
    nb = (7, 5, 5)
    r = np.zeros((5, 5, 7), dtype=bool)
    r[1:4, 1:4, 5] = True
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, storage, nb, False, [r], 1.7, 0.18, nozzle=NOZ)
        lbm.lbm_set_inflow(ctx, *INFLOW)
        for l in range(2):
            NX, NY, NZ = ctx.dims(l)
            rho, u = synth.taylor_green_3d(NY, 0.02, shape=(NX, NY, NZ))
            lbm.lbm_init_equilibrium(ctx, l, rho, u)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 3)
        lbm.lbm_sync(ctx)
        out.append([lbm.lbm_get_raw_state(ctx, l) for l in range(2)])
        lbm.lbm_destroy(ctx)
    for l in range(2):
        assert np.array_equal(out[0][l], out[1][l])


def test_nozzle_keeps_rest_and_rejects_bad_placement():
    lbm = gpu()
    ctx = lbm.lbm_create("d3q27", "f32", (5, 5, 5), False, [], 1.3, 0.0, nozzle=NOZ)
    r0, u0 = lbm.lbm_macroscopic(ctx, 0)
    lbm.lbm_step(ctx, 20)
    r1, u1 = lbm.lbm_macroscopic(ctx, 0)
    ok = ~np.isnan(r0)
    assert np.abs(r1[ok] - 1.0).max() <= 1e-6 and np.abs(u1[:, ok]).max() <= 1e-6
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_forward(ctx, 4, 2)
    lbm.lbm_destroy(ctx)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create("d3q27", "f32", (5, 5, 5), False, [], 1.3, 0.0, nozzle=(20.0, 20.0, 4.3, 2.25, 24.0))


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls", [15, 31])
def test_paper_tank_all_boundaries_f64(model, walls):
    """The paper's tank on a small nested grid: no-slip side walls and
    bottom, free-slip top, pressure outlet, the nozzle on the fine level with
    the inflow on its cap, with or without the upstream wall at x = 0; two
    coarse steps against the oracle."""
    lbm = gpu()
    nb, ref = nested_grid()
    ctx, orc = pair(model, "f64", nb, ref, nozzle=NOZ1, walls=walls, slip=8, outlet=1)
    lbm.lbm_set_outlet(ctx, 0.998)
    orc.set_outlet(0.998)
    fields = [synth.taylor_green_3d(lv.NY, 0.02, shape=(lv.NX, lv.NY, lv.NZ)) for lv in orc.levels]
    init_both(ctx, orc, fields)
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    lbm.lbm_destroy(ctx)


def test_full_size_paper_tank_keeps_rest():
    """The bench's paper-tank grid at full size (coarse 384x192x192, walls,
    free-slip top, pressure outlet at rho_out = 1, the nozzle on the fine
    level) with zero inflow: every boundary maps the rest state to itself, so
    three coarse steps leave it at rest to FP32 round-off."""
    lbm = gpu()
    flags, centre = synth.jet_two_level()
    flags = [flags[0].copy()]
    flags[0][:, :, -1] = False
    ctx = lbm.lbm_create("d3q27", "f32", (48, 24, 24), False, flags, 1.0 / (3 * 8e-5 + 0.5), 0.0,
                         walls=15, slip=8, outlet=1, nozzle=(centre[0], centre[1], 8.0, 8.0, 48.0))
    lbm.lbm_set_outlet(ctx, 1.0)
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 16.0, 0.0, 0.01, 3)
    for l in range(2):
        lbm.lbm_init_equilibrium(ctx, l)
    lbm.lbm_step(ctx, 3)
    for l in range(2):
        rho, u = lbm.lbm_macroscopic(ctx, l)
        ok = ~np.isnan(rho)
        assert ok.sum() > 0
        assert np.abs(rho[ok] - 1).max() <= 1e-6
        assert np.abs(u[:, ok]).max() <= 1e-7
    lbm.lbm_destroy(ctx)

"""GPU parity of the fixed-pressure outlet (Section 3.2 holds the tank's
outflow at a fixed pressure; read as the extrapolation of the
non-equilibrium part) against the FP64 oracle, through the C ABI.

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


def dims(nb, l=0):
    return tuple(8 * n << l for n in nb)


def pair(model, storage, nb, refine=(), omega=1.7, cs=0.18, walls=0, slip=0, rho_out=1.01):
    ctx, orc = make_pair(model, storage, nb, False, refine, omega=omega, cs=cs, walls=walls, slip=slip,
                         outlet=1)
    gpu().lbm_set_outlet(ctx, rho_out)
    orc.set_outlet(rho_out)
    return ctx, orc


def inflow(ctx, orc, *args):
    gpu().lbm_set_inflow(ctx, *args)
    orc.set_inflow(*args)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", [(0, 0), (15, 8)])
@pytest.mark.parametrize("variant", ["128,1,0", "256,4,1"])
def test_outlet_single_level_f64(model, walls, slip, variant, monkeypatch):
    """Two steps from a random far-from-equilibrium state with the inflow disc
    on x = 0 and the pressure outlet on x = NX, with and without tank walls."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (3, 2, 2)
    ctx, orc = pair(model, "f64", nb, walls=walls, slip=slip)
    inflow(ctx, orc, 8.0, 8.0, 10.0, 0.05, 0.01, 11)
    st = random_state(model, dims(nb), 31, 0.2)
    upload_same_state(ctx, orc, [st])
    gpu().lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    gpu().lbm_destroy(ctx)


def tank_jet():
    nb = (4, 3, 3)
    r = np.zeros((3, 3, 4), dtype=bool)
    r[1, 1, 0:2] = True
    return nb, [r]


@pytest.mark.parametrize("model", MODELS)
def test_outlet_nested_tank_jet_f64(model):
    """The time-nested jet in a tank with the pressure outlet: every level,
    the FP64 audit and the macroscopic fields."""
    lbm = gpu()
    nb, ref = tank_jet()
    ctx, orc = pair(model, "f64", nb, ref, walls=15, slip=8, rho_out=0.995)
    fields = []
    for lv in orc.levels:
        fields.append(synth.taylor_green_3d(lv.NY, 0.03, shape=(lv.NX, lv.NY, lv.NZ)))
    init_both(ctx, orc, fields)
    inflow(ctx, orc, 12.0, 12.0, 8.0, 0.05, 0.01, 5)
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    mg = lbm.lbm_mass_momentum(ctx)
    mo = orc.mass_momentum().numpy()
    assert np.abs(mg - mo).max() <= 1e-10 * max(1.0, np.abs(mo).max())
    rg, ug = lbm.lbm_macroscopic(ctx, 0)
    ro, uo = orc.macroscopic(0)
    ok = ~np.isnan(rg)
    assert np.abs(rg[ok] - ro.numpy()[ok]).max() < 1e-12
    assert np.abs(ug[:, ok] - uo.numpy()[:, ok]).max() < 1e-12
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_outlet_per_step_reduced_precision(model, storage):
    """One step from the GPU's rounded state, F32 and F16 storage."""
    lbm = gpu()
    nb = (3, 2, 2)
    ctx, orc = pair(model, storage, nb, omega=1.9, cs=0.1, rho_out=1.02)
    inflow(ctx, orc, 8.0, 8.0, 10.0, 0.05, 0.01, 2)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 17, 0.2)])
    lbm.lbm_step(ctx, 1)
    orc.set_state(0, torch.from_numpy(lbm.lbm_get_state(ctx, 0)))
    orc.coarse_step = lbm.lbm_get_step(ctx)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    if storage == "f32":
        d, s = compare_levels(ctx, orc)
        assert d / s <= 1e-6, d / s
    else:
        from oracle.lattice import weights
        Q = 19 if model == "d3q19" else 27
        w = weights(Q).numpy()
        shift = w if model == "d3q27" else np.zeros_like(w)
        m = valid_mask(orc, 0)
        fg = lbm.lbm_get_state(ctx, 0)[:, m]
        fo = orc.state(0).numpy()[:, m]
        err = np.abs(fg - fo) / w[:, None]
        bound = 4 * 2.0 ** -11 * (np.abs(fo - shift[:, None]) / w[:, None]).max() + 1e-6
        assert err.max() <= bound, (err.max(), bound)
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_outlet_graph_and_direct_launches_agree(model, storage, monkeypatch):
    """The coarse-step graph (outlet and inflow launch beside the
    coarse-to-fine launch) and the sequential profiled launches give the same
    bits (one launch shape)."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,1,0")
    lbm = gpu()
    nb, ref = tank_jet()
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, storage, nb, False, ref, 1.7, 0.18, walls=15, slip=8, outlet=1)
        lbm.lbm_set_outlet(ctx, 0.99)
        lbm.lbm_set_inflow(ctx, 12.0, 12.0, 12.0, 0.05, 0.01, 77)
        for l in range(2):
            NX, NY, NZ = ctx.dims(l)
            rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
            lbm.lbm_init_equilibrium(ctx, l, rho, u)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 4)
        lbm.lbm_sync(ctx)
        out.append([lbm.lbm_get_raw_state(ctx, l) for l in range(2)])
        lbm.lbm_destroy(ctx)
    for l in range(2):
        assert np.array_equal(out[0][l], out[1][l])


def test_outlet_error_codes():
    lbm = gpu()
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), False, [], 1.5, 0.0)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_outlet(ctx, 1.0)
    assert e.value.status == lbm.LBM_ERR_STATE
    lbm.lbm_destroy(ctx)
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), False, [], 1.5, 0.0, outlet=1)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_outlet(ctx, 3.0)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_outlet(ctx, float("nan"))
    assert e.value.status == lbm.LBM_ERR_NONFINITE
    lbm.lbm_destroy(ctx)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.5, 0.0, outlet=1)

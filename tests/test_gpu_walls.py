"""GPU parity of the wall reflections on the y / z faces (Section 3.2 names
the tank's no-slip walls and a free-slip top) against the FP64 oracle, on the
same seeded inputs, through the C ABI.

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
VARIANTS = ["128,1,0", "128,8,0", "256,4,1", "128,7,0"]
# (walls, slip): no-slip y walls; free-slip z walls; a tank (no-slip sides,
# free-slip top z); free-slip y with no-slip z; four free-slip faces
WALLS = [(3, 0), (12, 12), (15, 8), (15, 3), (15, 15)]


def dims(nb, l=0):
    return tuple(8 * n << l for n in nb)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", WALLS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_walls_single_level_f64(model, walls, slip, variant, monkeypatch):
    """Two steps from a random far-from-equilibrium state on a ragged grid
    (several blocks per face, edge and corner cells where a link crosses
    two walls) in every compiled launch shape."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (2, 3, 2)
    ctx, orc = make_pair(model, "f64", nb, omega=1.7, cs=0.18, walls=walls, slip=slip)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 21, 0.3)])
    gpu().lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    gpu().lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", [(15, 8), (15, 5)])
def test_walls_single_block_f64(model, walls, slip):
    """One block: both faces of an axis are in the same block."""
    nb = (1, 1, 1)
    ctx, orc = make_pair(model, "f64", nb, omega=1.3, cs=0.1, walls=walls, slip=slip)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 5, 0.3)])
    gpu().lbm_step(ctx, 3)
    orc.step(3)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    gpu().lbm_destroy(ctx)


def tank_jet():
    """A two-level jet in a tank: inflow face x = 0, outflow x = NX, the
    refined patch one block away from the walls."""
    nb = (4, 3, 3)
    r = np.zeros((3, 3, 4), dtype=bool)
    r[1, 1, 0:2] = True
    return nb, [r]


def tank_fields(orc):
    out = []
    for lv in orc.levels:
        rho, u = synth.taylor_green_3d(lv.NY, 0.03, shape=(lv.NX, lv.NY, lv.NZ))
        out.append((rho, u))
    return out


@pytest.mark.parametrize("model", MODELS)
def test_walls_nested_jet_f64(model):
    """Time-nested jet with inflow disc, outflow and a tank of no-slip side
    walls and a free-slip top: every level, the FP64 mass/momentum audit and
    the macroscopic fields."""
    lbm = gpu()
    nb, ref = tank_jet()
    ctx, orc = make_pair(model, "f64", nb, False, ref, omega=1.7, cs=0.18, walls=15, slip=8)
    init_both(ctx, orc, tank_fields(orc))
    lbm.lbm_set_inflow(ctx, 12.0, 12.0, 8.0, 0.05, 0.01, 77)
    orc.set_inflow(12.0, 12.0, 8.0, 0.05, 0.01, 77)
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    mg = lbm.lbm_mass_momentum(ctx)
    mo = orc.mass_momentum().numpy()
    assert np.abs(mg - mo).max() <= 1e-10 * max(1.0, np.abs(mo).max())
    for l in range(2):
        rg, ug = lbm.lbm_macroscopic(ctx, l)
        ro, uo = orc.macroscopic(l)
        ok = ~np.isnan(rg)
        assert np.array_equal(~ok, np.isnan(ro.numpy()))
        assert np.abs(ug[:, ok] - uo.numpy()[:, ok]).max() < 1e-12
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_walls_nested_jet_f32_per_step(model):
    lbm = gpu()
    nb, ref = tank_jet()
    ctx, orc = make_pair(model, "f32", nb, False, ref, omega=1.9, cs=0.1, walls=15, slip=8)
    init_both(ctx, orc, tank_fields(orc))
    lbm.lbm_set_inflow(ctx, 12.0, 12.0, 8.0, 0.05, 0.01, 3)
    orc.set_inflow(12.0, 12.0, 8.0, 0.05, 0.01, 3)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    for l in range(2):
        orc.set_state(l, torch.from_numpy(lbm.lbm_get_state(ctx, l)))
    orc.coarse_step = lbm.lbm_get_step(ctx)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    d, s = compare_levels(ctx, orc)
    assert d / s <= 1e-6, d / s
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_walls_f16_per_step(model):
    """FP16 storage with walls on all four faces (mixed types): one step from
    the GPU's rounded state; the bound allows four roundings of the largest
    (f - w)/w."""
    lbm = gpu()
    nb = (2, 2, 2)
    ctx, orc = make_pair(model, "f16", nb, omega=1.6, cs=0.1, walls=15, slip=6)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 8, 0.2)])
    lbm.lbm_step(ctx, 1)
    orc.set_state(0, torch.from_numpy(lbm.lbm_get_state(ctx, 0)))
    lbm.lbm_step(ctx, 1)
    orc.step(1)
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


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_walls_conserve_mass_over_many_steps(storage):
    """Reflections only move populations: the FP64 mass audit of a random
    state stays constant over 100 steps between no-slip and free-slip walls
    (D3Q27 FCLB)."""
    lbm = gpu()
    nb = (2, 3, 2)
    ctx = lbm.lbm_create("d3q27", storage, nb, True, [], 1.5, 0.0, walls=15, slip=4)
    lbm.lbm_set_state(ctx, 0, random_state("d3q27", dims(nb), 13, 0.1))
    m0 = lbm.lbm_mass_momentum(ctx)[0]
    lbm.lbm_step(ctx, 100)
    m1 = lbm.lbm_mass_momentum(ctx)[0]
    tol = 1e-11 if storage == "f64" else 1e-4
    assert abs(m1 - m0) <= tol * abs(m0), (m0, m1)
    lbm.lbm_destroy(ctx)


def test_walls_poiseuille_f32():
    """Body-force-driven channel between no-slip y walls, 32 cells wide, in
    FP32 storage: the parabola u_x(y) = F / (2 nu) (y + 1/2) (H - 1/2 - y)
    of half-way bounce-back is kept within 1 % of its maximum over 500 steps
    and the other components stay at rest."""
    lbm = gpu()
    NY, tau, umax = 32, 0.8, 0.01
    nu = (tau - 0.5) / 3
    F = 8 * nu * umax / NY ** 2
    nb = (1, 4, 1)
    NX, _, NZ = dims(nb)
    ctx = lbm.lbm_create("d3q27", "f32", nb, True, [], 1 / tau, 0.0, walls=3, slip=0)
    y = np.arange(NY, dtype=np.float64)
    ux = F / (2 * nu) * (y + 0.5) * (NY - 0.5 - y)
    u = np.zeros((3, NZ, NY, NX))
    u[0] = ux[None, :, None]
    lbm.lbm_init_equilibrium(ctx, 0, np.ones((NZ, NY, NX)), u)
    Fv = np.zeros((3, NZ, NY, NX))
    Fv[0] = F
    lbm.lbm_set_force(ctx, Fv)
    lbm.lbm_step(ctx, 500)
    _, uu = lbm.lbm_macroscopic(ctx, 0)
    assert np.abs(uu[0] - ux[None, :, None]).max() <= 0.01 * umax
    assert np.abs(uu[1:]).max() <= 1e-4 * umax
    lbm.lbm_destroy(ctx)


def test_walls_reject_bad_settings_and_the_adjoint():
    lbm = gpu()
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.5, 0.0, walls=1)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.5, 0.0, walls=3, slip=4)
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.5, 0.0, walls=3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_forward(ctx, 4, 2)
    assert e.value.status == lbm.LBM_ERR_STATE
    lbm.lbm_destroy(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("walls,slip", [(63, 0), (63, 12), (48, 0), (31, 8)])
@pytest.mark.parametrize("variant", ["128,1,0", "128,7,0"])
def test_x_walls_f64(model, walls, slip, variant, monkeypatch):
    """No-slip walls on the x faces (a closed box with mixed y/z walls, a
    channel between x walls, the tank's upstream wall with an open outflow):
    two steps from a random state against the oracle."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (3, 2, 2)
    ctx, orc = make_pair(model, "f64", nb, False, omega=1.7, cs=0.18, walls=walls, slip=slip)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 37, 0.3)])
    gpu().lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    gpu().lbm_destroy(ctx)


def test_closed_box_conserves_mass_f64():
    lbm = gpu()
    nb = (2, 2, 2)
    ctx = lbm.lbm_create("d3q27", "f64", nb, False, [], 1.5, 0.0, walls=63, slip=8)
    lbm.lbm_set_state(ctx, 0, random_state("d3q27", dims(nb), 41, 0.1))
    m0 = lbm.lbm_mass_momentum(ctx)[0]
    lbm.lbm_step(ctx, 100)
    m1 = lbm.lbm_mass_momentum(ctx)[0]
    assert abs(m1 - m0) <= 1e-11 * abs(m0)
    lbm.lbm_destroy(ctx)

"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (stated per storage):
* F64 storage, float64 arithmetic: |f_gpu - f_oracle| <= 1e-12 (the two
  sides differ only in rounding order: closed forms vs. matrix solves).
* F32 storage: per-step post-collision relative error <= 1e-6 of max|f|;
  velocity relative L2 <= 1e-4 after 1000 steps (non-chaotic flows).
* F16 storage ((f - w)/w in half precision): per-step error <= 2^-10 of the
  largest |f - w| / w, times w_i, per population (the rounding of the store).
"""
import math

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


def close(ctx):
    gpu().lbm_destroy(ctx)


# ---------------------------------------------------------------- uniform grids

# every compiled stream-collide variant: no register cap, 64-register cap
# (one CTA per block and persistent)
VARIANTS = ["128,1,0", "128,8,0", "256,4,1", "128,7,0"]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("nb", [(3, 2, 1), (1, 1, 1), (2, 3, 5)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_single_step_f64(model, nb, variant, monkeypatch):
    """One stream-collide step from a random far-from-equilibrium state,
    ragged block counts (several CTAs and a partial last wave) and the
    single-block grid whose neighbours are all itself."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    ctx, orc = make_pair(model, "f64", nb, omega=1.7, cs=0.18)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 11, 0.3)])
    gpu().lbm_step(ctx, 1)
    orc.step(1)
    d, s = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_single_step_f32(model, variant, monkeypatch):
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (3, 2, 2)
    ctx, orc = make_pair(model, "f32", nb, omega=1.9, cs=0.1)
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 5, 0.3)])
    gpu().lbm_step(ctx, 1)
    orc.step(1)
    d, s = compare_levels(ctx, orc)
    assert d / s <= 1e-6, d / s
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_single_step_f16(model, variant, monkeypatch):
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", variant)
    nb = (2, 2, 2)
    lbm = gpu()
    ctx, orc = make_pair(model, "f16", nb, omega=1.5, cs=0.1)
    rho, u = synth.taylor_green_3d(16, 0.05)
    init_both(ctx, orc, [(rho, u)])
    # start both from the half-precision state the GPU holds
    orc.set_state(0, torch.from_numpy(lbm.lbm_get_state(ctx, 0)))
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    from oracle.lattice import weights
    w = weights(19 if model == "d3q19" else 27).numpy()
    fg = lbm.lbm_get_state(ctx, 0)
    fo = orc.state(0).numpy()
    shift = w if model == "d3q27" else np.zeros_like(w)
    scaled = np.abs(fo - shift[:, None, None, None]) / w[:, None, None, None]
    err = np.abs(fg - fo) / w[:, None, None, None]
    bound = 2.0 ** -10 * scaled.max() + 1e-6
    assert err.max() <= bound, (err.max(), bound)
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_graph_and_direct_launches_agree(model, monkeypatch):
    """The CUDA-graph path and the profiled direct-launch path are identical
    (for one launch shape: the autotuner of each context may pick another,
    and register-capped shapes may round differently)."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,1,0")
    lbm = gpu()
    nb = (2, 2, 2)
    st = random_state(model, dims(nb), 3, 0.2)
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, "f32", nb, True, [], 1.6, 0.1)
        lbm.lbm_set_state(ctx, 0, st)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 3)
        out.append(lbm.lbm_get_state(ctx, 0))
        if prof:
            ms, n = lbm.lbm_get_profile(ctx)
            assert n[0] == 3 and ms[0] > 0
        close(ctx)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("model", MODELS)
def test_nested_graph_and_direct_launches_agree(model, monkeypatch):
    """A nested grid with inflow whose refined patch meets the inflow face:
    the coarse-step graph (inflow launch beside the coarse-to-fine launch,
    inflow ghosts fed by ghost cells written by the latter) gives the same
    bits as the sequential launches of the profiled path (one launch shape)."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,1,0")
    lbm = gpu()
    nb = (4, 3, 3)
    r = np.zeros((3, 3, 4), dtype=bool)
    r[1, 1, 0:2] = True
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, "f32", nb, False, [r], 1.7, 0.18)
        lbm.lbm_set_inflow(ctx, 12.0, 12.0, 12.0, 0.05, 0.01, 77)
        for l in range(2):
            NX, NY, NZ = ctx.dims(l)
            rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
            lbm.lbm_init_equilibrium(ctx, l, rho, u)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 4)
        lbm.lbm_sync(ctx)
        out.append([lbm.lbm_get_raw_state(ctx, l) for l in range(2)])
        close(ctx)
    for l in range(2):
        assert np.array_equal(out[0][l], out[1][l])


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_three_level_graph_and_direct_launches_agree(model, storage, monkeypatch):
    """Three levels with inflow on a grid large enough to fill the GPU (coarse
    128 x 64 x 64): the coarse-step graph runs the first substep's level-0
    update and the restriction into level 0 on branches beside the fine
    levels' chain; it gives the same bits as the sequential launches of the
    profiled path (one launch shape)."""
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "128,8,0")
    lbm = gpu()
    nb = (16, 8, 8)
    flags, (y0, z0) = synth.jet_three_level(*nb, r1=(0.0, 12.0), r2=(0.0, 8.0), x1=(0, 48), x2=(0, 24))
    out = []
    for prof in (False, True):
        ctx = lbm.lbm_create(model, storage, nb, False, flags, 1.9, 0.18)
        lbm.lbm_set_inflow(ctx, y0, z0, 8.0, 0.05, 0.01, 91)
        for l in range(3):
            NX, NY, NZ = ctx.dims(l)
            rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
            lbm.lbm_init_equilibrium(ctx, l, rho, u)
        lbm.lbm_set_profiling(ctx, prof)
        lbm.lbm_step(ctx, 5)
        lbm.lbm_sync(ctx)
        out.append([lbm.lbm_get_raw_state(ctx, l) for l in range(3)])
        close(ctx)
    for l in range(3):
        assert np.array_equal(out[0][l], out[1][l]), l


def test_taylor_green_32_f64_200_steps():
    """32^3 Taylor-Green vortex, D3Q19 MRT + Smagorinsky (Cs = 0.1), FP64,
    u0 = 0.05, nu = 0.005, 200 steps: identical to the oracle to 1e-12, mass
    and momentum conserved to round-off."""
    lbm = gpu()
    nu = 0.005
    omega = 1.0 / (3 * nu + 0.5)
    ctx, orc = make_pair("d3q19", "f64", (4, 4, 4), omega=omega, cs=0.1)
    rho, u = synth.taylor_green_3d(32, 0.05)
    init_both(ctx, orc, [(rho, u)])
    m0 = lbm.lbm_mass_momentum(ctx)
    lbm.lbm_step(ctx, 200)
    orc.step(200)
    d, s = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    m1 = lbm.lbm_mass_momentum(ctx)
    assert np.abs(m1 - m0).max() < 1e-11
    mo = orc.mass_momentum().numpy()
    assert np.abs(m1 - mo).max() < 1e-11
    close(ctx)


@pytest.mark.parametrize("model,N", [("d3q19", 32), ("d3q27", 16)])
def test_velocity_l2_after_1000_steps_f32(model, N):
    """Non-chaotic Taylor-Green flow, FP32 storage vs the FP64 oracle:
    velocity relative L2 error <= 1e-4 after 1000 steps."""
    lbm = gpu()
    omega = 1.0 / (3 * 0.01 + 0.5)
    nb = (N // 8,) * 3
    ctx, orc = make_pair(model, "f32", nb, omega=omega, cs=0.0)
    rho, u = synth.taylor_green_3d(N, 0.03)
    init_both(ctx, orc, [(rho, u)])
    lbm.lbm_step(ctx, 1000)
    orc.step(1000)
    _, ug = lbm.lbm_macroscopic(ctx, 0)
    _, uo = orc.macroscopic(0)
    uo = uo.numpy()
    l2 = np.sqrt(((ug - uo) ** 2).sum() / (uo ** 2).sum())
    print("velocity relative L2 after 1000 steps:", l2)
    assert l2 <= 1e-4
    close(ctx)


def fp16_velocity_bound(f0, u_final, model, steps):
    """Stated bound on the velocity relative L2 error of FP16 storage after
    `steps` steps: B = sqrt(N) 2^-11 ||I||_2 / ||u_N||_2 with
        I = sqrt(sum_i |e_i|^2 g_i^2)   per cell, from the initial state,
    g_i the stored deviation (f_i - w_i for D3Q27, f_i for the incompressible
    D3Q19 distribution) and u_N the velocity field after the N steps.  One
    step stores every g_i with a relative rounding of at most 2^-11 (half
    precision of g_i / w_i), which moves a cell's momentum by at most
    sum_i |e_i| 2^-11 |g_i|; the roundings of different values and steps are
    independent and unbiased (round to nearest), and the stream-collide map
    does not amplify a perturbation of a stable non-chaotic flow, so the
    error variances add: the absolute L2 error after N steps is about
    sqrt(N) 2^-11 ||I|| / sqrt(3), and B allows sqrt(3) over it.  I is taken
    at t = 0, where the deviations of a decaying flow are largest."""
    from oracle.lattice import velocities, weights
    Q = f0.shape[0]
    e = velocities(Q).numpy().astype(np.float64).T        # [3][Q]
    w = weights(Q).numpy()
    f = f0.reshape(Q, -1)
    g = f - w[:, None] if model == "d3q27" else f
    inj = np.sqrt(((e ** 2).sum(0)[:, None] * g * g).sum(0))
    return math.sqrt(steps) * 2.0 ** -11 * np.sqrt((inj ** 2).sum()) / np.sqrt((u_final ** 2).sum())


@pytest.mark.parametrize("model,N", [("d3q19", 32), ("d3q27", 16)])
def test_fp16_velocity_l2_after_1000_steps_within_stated_bound(model, N):
    """Non-chaotic Taylor-Green flow (u0 = 0.03, nu = 0.002: the velocity
    keeps about 80 % (32^3) or 40 % (16^3) of its amplitude), FP16 storage vs
    the FP64 oracle after 1000 steps: the measured velocity relative L2 error
    stays below the stated bound sqrt(N) 2^-11 ||I|| / ||u_N|| (I from the
    initial state)."""
    lbm = gpu()
    omega = 1.0 / (3 * 0.002 + 0.5)
    nb = (N // 8,) * 3
    ctx, orc = make_pair(model, "f16", nb, omega=omega, cs=0.0)
    rho, u = synth.taylor_green_3d(N, 0.03)
    init_both(ctx, orc, [(rho, u)])
    f0 = orc.state(0).numpy()
    lbm.lbm_step(ctx, 1000)
    orc.step(1000)
    _, ug = lbm.lbm_macroscopic(ctx, 0)
    _, uo = orc.macroscopic(0)
    uo = uo.numpy()
    bound = fp16_velocity_bound(f0, uo, model, 1000)
    l2 = np.sqrt(((ug - uo) ** 2).sum() / (uo ** 2).sum())
    print("FP16 velocity relative L2 after 1000 steps: %.3e, stated bound %.3e" % (l2, bound))
    assert l2 <= bound
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_body_force_step_f64(model):
    if model == "d3q19":
        pytest.skip("body force is defined for the FCLB model")
    lbm = gpu()
    nb = (2, 2, 1)
    ctx, orc = make_pair(model, "f64", nb, omega=1.6)
    F = synth.random_force((8, 16, 16), 7, sigma=1e-4)
    lbm.lbm_set_force(ctx, F)
    orc.set_force(torch.from_numpy(F))
    upload_same_state(ctx, orc, [random_state(model, dims(nb), 9, 0.1)])
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, _ = compare_levels(ctx, orc)
    assert d <= 1e-12
    r1, u1 = lbm.lbm_macroscopic(ctx, 0)
    r2, u2 = orc.macroscopic(0)
    assert np.abs(u1 - u2.numpy()).max() < 1e-13
    close(ctx)


# ---------------------------------------------------------------- nested grids

def jet_grid(levels):
    if levels == 2:
        nb = (4, 2, 2)
        r = np.zeros((2, 2, 4), dtype=bool)
        r[:, :, 0:2] = True
        return nb, [r]
    nb = (3, 2, 2)
    r0 = np.zeros((2, 2, 3), dtype=bool)
    r0[:, :, 0:2] = True
    r1 = np.zeros((4, 4, 6), dtype=bool)
    r1[1:3, 1:3, 1:3] = True
    return nb, [r0, r1]


def nested_fields(orc):
    out = []
    for l, lv in enumerate(orc.levels):
        rho, u = synth.taylor_green_3d(lv.NY, 0.03, shape=(lv.NX, lv.NY, lv.NZ))
        out.append((rho, u))
    return out


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("levels", [2, 3])
@pytest.mark.parametrize("periodic_x", [True, False])
def test_nested_parity_f64(model, levels, periodic_x):
    """Time-nested grid with interface transfer, Smagorinsky |S| carried across
    levels, inflow disc with perturbation and zero-gradient outflow."""
    lbm = gpu()
    nb, ref = jet_grid(levels)
    ctx, orc = make_pair(model, "f64", nb, periodic_x, ref, omega=1.7, cs=0.18)
    init_both(ctx, orc, nested_fields(orc))
    if not periodic_x:
        lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 1234)
        orc.set_inflow(8.0, 8.0, 8.0, 0.05, 0.01, 1234)
    lbm.lbm_step(ctx, 2)
    orc.step(2)
    d, s = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    mg = lbm.lbm_mass_momentum(ctx)
    mo = orc.mass_momentum().numpy()
    assert np.abs(mg - mo).max() <= 1e-10 * max(1.0, np.abs(mo).max())
    for l in range(levels):
        rg, ug = lbm.lbm_macroscopic(ctx, l)
        ro, uo = orc.macroscopic(l)
        assert np.array_equal(np.isnan(rg), np.isnan(ro.numpy()))
        ok = ~np.isnan(rg)
        assert np.abs(rg[ok] - ro.numpy()[ok]).max() < 1e-12
        assert np.abs(ug[:, ok] - uo.numpy()[:, ok]).max() < 1e-12
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_nested_parity_refined_patch_on_inflow_face(model):
    """A refined patch that touches the inflow face only in part: fine ghost
    cells lie on x = 0, so fine inflow ghosts take their density from
    coarse-to-fine ghost cells, and the disc straddles the patch edge."""
    lbm = gpu()
    nb = (4, 3, 3)
    r = np.zeros((3, 3, 4), dtype=bool)
    r[1, 1, 0:2] = True
    ctx, orc = make_pair(model, "f64", nb, False, [r], omega=1.7, cs=0.18)
    init_both(ctx, orc, nested_fields(orc))
    lbm.lbm_set_inflow(ctx, 12.0, 12.0, 12.0, 0.05, 0.01, 77)
    orc.set_inflow(12.0, 12.0, 12.0, 0.05, 0.01, 77)
    lbm.lbm_step(ctx, 3)
    orc.step(3)
    d, s = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_time_statistics_match_oracle(model):
    """Time-averaged rho, u and the velocity variances over three coarse steps
    of a nested run with inflow, against the same averages of the oracle's
    macroscopic fields (float64)."""
    lbm = gpu()
    nb, ref = jet_grid(2)
    ctx, orc = make_pair(model, "f64", nb, False, ref, omega=1.7, cs=0.18)
    init_both(ctx, orc, nested_fields(orc))
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 4321)
    orc.set_inflow(8.0, 8.0, 8.0, 0.05, 0.01, 4321)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_stats_accumulate(ctx)
    lbm.lbm_stats_reset(ctx)
    acc = [None, None]
    for _ in range(3):
        lbm.lbm_step(ctx, 1)
        orc.step(1)
        lbm.lbm_stats_accumulate(ctx)
        for l in range(2):
            ro, uo = orc.macroscopic(l)
            ro, uo = ro.numpy(), uo.numpy()
            v = np.concatenate([ro[None], uo, uo * uo])
            acc[l] = v if acc[l] is None else acc[l] + v
    for l in range(2):
        mean, var, n = lbm.lbm_stats_get(ctx, l)
        assert n == 3
        mo = acc[l][:4] / 3
        vo = acc[l][4:] / 3 - mo[1:] ** 2
        assert np.array_equal(np.isnan(mean), np.isnan(mo))
        ok = ~np.isnan(mo[0])
        assert np.abs(mean[:, ok] - mo[:, ok]).max() <= 1e-12
        assert np.abs(var[:, ok] - vo[:, ok]).max() <= 1e-12
        assert var[:, ok].max() > 0
    close(ctx)


def test_coarsened_paper_jet_parity_f64():
    """The paper-scale 3-level jet's layout on a 4x-coarsened domain (coarse
    128 x 64 x 64, nozzle D = 8, level 1 within 12 coarse cells of the axis
    over x < 48, level 2 within 8 over x < 24), D3Q27 FCLB in float64 with
    inflow and outflow: one coarse step (every level's substeps, both
    interfaces of both level pairs) against the oracle."""
    lbm = gpu()
    nb = (16, 8, 8)
    flags, centre = synth.jet_three_level(*nb, r1=(0.0, 12.0), r2=(0.0, 8.0), x1=(0, 48), x2=(0, 24))
    nu_c = 0.05 * 8 / 1e4
    omega = 1.0 / (3 * nu_c + 0.5)
    ctx, orc = make_pair("d3q27", "f64", nb, False, flags, omega=omega, cs=0.0)
    assert len(orc.levels) == 3
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 8.0, 0.05, 0.01, 5120)
    orc.set_inflow(centre[0], centre[1], 8.0, 0.05, 0.01, 5120)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    d, s = compare_levels(ctx, orc)
    assert d <= 1e-12, d
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_nested_parity_f32_per_step(model):
    lbm = gpu()
    nb, ref = jet_grid(2)
    ctx, orc = make_pair(model, "f32", nb, False, ref, omega=1.9, cs=0.1)
    init_both(ctx, orc, nested_fields(orc))
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 99)
    orc.set_inflow(8.0, 8.0, 8.0, 0.05, 0.01, 99)
    lbm.lbm_step(ctx, 1)           # restriction + one step on both sides
    orc.step(1)
    for l in range(2):             # restart both from the GPU's rounded state
        orc.set_state(l, torch.from_numpy(lbm.lbm_get_state(ctx, l)))
    orc.coarse_step = lbm.lbm_get_step(ctx)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    d, s = compare_levels(ctx, orc)
    assert d / s <= 1e-6, d / s
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_nested_parity_f16_per_step(model):
    """FP16 storage on the nested jet with inflow: one coarse step (two fine
    substeps, both interface transfers, the inflow) from the GPU's rounded
    state, against the float64 oracle.  Each stored value carries the
    half-precision rounding of (f - w)/w (2^-11 relative) once per substep;
    the bound allows four roundings of the largest deviation."""
    lbm = gpu()
    nb, ref = jet_grid(2)
    ctx, orc = make_pair(model, "f16", nb, False, ref, omega=1.9, cs=0.1)
    init_both(ctx, orc, nested_fields(orc))
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 99)
    orc.set_inflow(8.0, 8.0, 8.0, 0.05, 0.01, 99)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    for l in range(2):
        orc.set_state(l, torch.from_numpy(lbm.lbm_get_state(ctx, l)))
    orc.coarse_step = lbm.lbm_get_step(ctx)
    lbm.lbm_step(ctx, 1)
    orc.step(1)
    from oracle.lattice import weights
    Q = 19 if model == "d3q19" else 27
    w = weights(Q).numpy()
    shift = w if model == "d3q27" else np.zeros_like(w)
    for l in range(2):
        m = valid_mask(orc, l)
        fg = lbm.lbm_get_state(ctx, l)[:, m]
        fo = orc.state(l).numpy()[:, m]
        scaled = np.abs(fo - shift[:, None]) / w[:, None]
        err = np.abs(fg - fo) / w[:, None]
        bound = 4 * 2.0 ** -11 * scaled.max() + 1e-6
        assert err.max() <= bound, (l, err.max(), bound)
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_rest_state_with_zero_inflow_stays_at_rest(model):
    lbm = gpu()
    nb, ref = jet_grid(2)
    ctx = lbm.lbm_create(model, "f32", nb, False, ref, 1.8, 0.18)
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.0, 0.01, 5)
    for l in range(2):
        lbm.lbm_init_equilibrium(ctx, l)
    f0 = [lbm.lbm_get_state(ctx, l) for l in range(2)]
    lbm.lbm_step(ctx, 3)
    for l in range(2):
        f1 = lbm.lbm_get_state(ctx, l)
        ok = ~np.isnan(f0[l])
        assert np.abs(f1[ok] - f0[l][ok]).max() == 0.0
    close(ctx)


# ---------------------------------------------------------------- full size

@pytest.mark.parametrize("model,storage", [("d3q27", "f32"), ("d3q19", "f32"), ("d3q27", "f16")])
def test_full_size_256_sampled_cells(model, storage):
    """256^3 decaying-turbulence workload (k^4 spectrum field, k0 = 4,
    u_rms = 0.04, nu = 1e-4) in the launch configuration the benchmark times:
    one step on the GPU, then 2048 sampled cells recomputed by the oracle from
    their 27 (19) upstream neighbours read before the step."""
    lbm = gpu()
    N = 256
    omega = 1.0 / (3e-4 + 0.5)
    Q = 19 if model == "d3q19" else 27
    ctx = lbm.lbm_create(model, storage, (32, 32, 32), True, [], omega, 0.1 if model == "d3q19" else 0.0)
    rho, u = synth.spectrum_field(N, seed=1206)
    lbm.lbm_init_equilibrium(ctx, 0, rho, u)
    rng = np.random.default_rng(77)
    xs = np.concatenate([rng.integers(0, N, (2000, 3)),
                         np.array([[0, 0, 0], [255, 255, 255], [7, 8, 15], [8, 7, 16]] * 12)])
    from oracle.collision import Model
    from oracle.lattice import velocities
    e = velocities(Q).numpy()
    src = []
    for i in range(Q):
        p = (xs - e[i][None, :]) % N
        src.append(p[:, 0] + N * (p[:, 1] + N * p[:, 2]))
    before = [lbm.lbm_get_cells(ctx, 0, s) for s in src]
    pre = np.stack([before[i][:, i] for i in range(Q)])
    lbm.lbm_step(ctx, 1)
    after = lbm.lbm_get_cells(ctx, 0, xs[:, 0] + N * (xs[:, 1] + N * xs[:, 2]))
    m = Model(model)
    fo, _ = m.collide(torch.from_numpy(pre), omega, 0.1 if model == "d3q19" else 0.0)
    fo = fo.numpy().T
    if storage == "f32":
        assert np.abs(after - fo).max() / np.abs(fo).max() <= 1e-6
    else:
        from oracle.lattice import weights
        w = weights(Q).numpy()
        err = np.abs(after - fo) / w[None, :]
        assert err.max() <= 2.0 ** -10 * (np.abs(fo - w[None, :]) / w[None, :]).max() + 1e-6
    close(ctx)


def test_full_size_conservation_f32():
    """Mass and momentum of the 256^3 FCLB run stay constant (float64 audit)."""
    lbm = gpu()
    ctx = lbm.lbm_create("d3q27", "f32", (32, 32, 32), True, [], 1.0 / (3e-4 + 0.5), 0.0)
    rho, u = synth.spectrum_field(256, seed=1206)
    lbm.lbm_init_equilibrium(ctx, 0, rho, u)
    m0 = lbm.lbm_mass_momentum(ctx)
    lbm.lbm_step(ctx, 20)
    m1 = lbm.lbm_mass_momentum(ctx)
    ncell = 256 ** 3
    assert abs(m1[0] - m0[0]) / ncell < 1e-8
    assert np.abs(m1[1:] - m0[1:]).max() / ncell < 1e-8
    close(ctx)


def test_jet_grid_two_levels_runs_and_matches_plan():
    """The 2-level jet grid (coarse 384x192x192, fine cylinder of radius 24
    coarse cells) builds, steps and stays finite; plan sizes as derived."""
    lbm = gpu()
    flags, centre = synth.jet_two_level()
    ctx = lbm.lbm_create("d3q27", "f32", (48, 24, 24), False, flags, 1.0 / (3 * 8e-5 + 0.5), 0.0)
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 16.0, 0.05, 0.01, 389)
    lbm.lbm_step(ctx, 4)
    m = lbm.lbm_mass_momentum(ctx)
    assert np.isfinite(m).all() and m[1] > 0
    close(ctx)


# ---------------------------------------------------------------- errors

def test_error_codes():
    lbm = gpu()
    ctx = lbm.lbm_create("d3q19", "f32", (1, 1, 1))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_inflow(ctx, 4, 4, 2, 0.05)
    assert e.value.status == lbm.LBM_ERR_STATE
    bad = np.ones((8, 8, 8))
    bad[1, 2, 3] = np.nan
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_init_equilibrium(ctx, 0, bad, None)
    assert e.value.status == lbm.LBM_ERR_NONFINITE
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_get_state(ctx, 1)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_force(ctx, np.zeros((3, 8, 8, 8)))
    assert e.value.status == lbm.LBM_ERR_STATE
    st = np.full((19, 8, 8, 8), np.inf)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_state(ctx, 0, st)
    assert e.value.status == lbm.LBM_ERR_NONFINITE
    # a NaN planted in the state (NaN entries are skipped by set_state, so
    # write it through a second context's state) is caught by the audit
    close(ctx)


# ---------------------------------------------------------------- checkpoint, audit, full-size nested

def valid_cells(lbm, ctx, l):
    rho, _ = lbm.lbm_macroscopic(ctx, l)
    return ~np.isnan(rho)


# launch shapes grouped by compiled kernel variant (threads per CTA and the
# register cap of min CTAs per SM): within a group only the thread count and
# the grid differ
SHAPE_GROUPS = [["128,1,0", "256,1,0", "128,1,1", "256,1,1"],
                ["128,8,0", "128,8,1"], ["256,4,0", "256,4,1"], ["128,7,0", "128,7,1"]]


def run_with_shape(lbm, monkeypatch, sh, model, storage, steps=4):
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", sh)
    nb, ref = jet_grid(2)
    ctx = lbm.lbm_create(model, storage, nb, False, ref, 1.8, 0.18)
    t, m, c = lbm.lbm_get_tuning(ctx)
    assert (t, m, c > 0) == tuple(int(v) for v in sh.split(",")[:2]) + (sh.endswith(",1"),)
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 21)
    for l in range(2):
        NX, NY, NZ = ctx.dims(l)
        rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
        lbm.lbm_init_equilibrium(ctx, l, rho, u)
    lbm.lbm_step(ctx, steps)
    out = [lbm.lbm_get_raw_state(ctx, l) for l in range(2)]
    close(ctx)
    return out


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_results_do_not_depend_on_threads_or_grid(model, storage, monkeypatch):
    """The thread count per CTA and the grid (one CTA per block or a
    persistent grid) do not change a single bit of a nested run with inflow.
    (Kernel variants compiled for another register cap may round a few
    operations differently: the compiler contracts multiply-adds per variant.)"""
    lbm = gpu()
    for group in SHAPE_GROUPS:
        out = [run_with_shape(lbm, monkeypatch, sh, model, storage) for sh in group]
        for sh, o in zip(group[1:], out[1:]):
            for l in range(2):
                assert np.array_equal(o[l], out[0][l]), (sh, l)


def test_launch_shape_override_rejects_unlisted_shapes(monkeypatch):
    lbm = gpu()
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", "96,1,0")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create("d3q27", "f32", (2, 1, 1), True, [], 1.5, 0.0)
    assert e.value.status == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("model", MODELS)
def test_checkpoint_resume_is_bitwise(model, monkeypatch):
    """The raw state of every level (distributions and, for nested D3Q19, the
    Smagorinsky strain carried across levels) plus the step counter resume a
    nested run with inflow bit for bit."""
    lbm = gpu()
    nb, ref = jet_grid(2)
    a = lbm.lbm_create(model, "f32", nb, False, ref, 1.8, 0.18)
    # the resumed context runs the same kernel variant as the saved one
    t, m, c = lbm.lbm_get_tuning(a)
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", f"{t},{m},{int(c > 0)}")
    lbm.lbm_set_inflow(a, 8.0, 8.0, 8.0, 0.05, 0.01, 21)
    lbm.lbm_step(a, 3)
    raw = [lbm.lbm_get_raw_state(a, l) for l in range(2)]
    step = lbm.lbm_get_step(a)
    lbm.lbm_step(a, 4)
    ref_state = [lbm.lbm_get_state(a, l) for l in range(2)]
    b = lbm.lbm_create(model, "f32", nb, False, ref, 1.8, 0.18)
    lbm.lbm_set_inflow(b, 8.0, 8.0, 8.0, 0.05, 0.01, 21)
    for l in range(2):
        lbm.lbm_set_raw_state(b, l, raw[l])
    lbm.lbm_set_step(b, step)
    lbm.lbm_step(b, 4)
    for l in range(2):
        m = valid_cells(lbm, a, l)
        got = lbm.lbm_get_state(b, l)
        assert np.array_equal(got[:, m], ref_state[l][:, m])
    close(a)
    close(b)


def test_dense_state_round_trip_and_strain():
    """The dense float64 state and the strain field read back what was set."""
    lbm = gpu()
    nb, ref = jet_grid(2)
    a = lbm.lbm_create("d3q19", "f64", nb, True, ref, 1.7, 0.18)
    for l in range(2):
        NX, NY, NZ = a.dims(l)
        rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
        lbm.lbm_init_equilibrium(a, l, rho, u)
    lbm.lbm_step(a, 2)
    for l in range(2):
        f = lbm.lbm_get_state(a, l)
        S = lbm.lbm_get_strain(a, l)
        assert np.nanmax(S) > 0
        lbm.lbm_set_state(a, l, f)
        lbm.lbm_set_strain(a, l, S)
        assert np.array_equal(np.isnan(f), np.isnan(lbm.lbm_get_state(a, l)))
        ok = ~np.isnan(f)
        assert np.array_equal(lbm.lbm_get_state(a, l)[ok], f[ok])
        ok = ~np.isnan(S)
        assert np.array_equal(lbm.lbm_get_strain(a, l)[ok], S[ok])
    close(a)


def test_audit_reports_nonfinite_state():
    """A value beyond the float32 range, planted on the host through the
    state (finite as float64, so it passes the input check), is stored as Inf;
    after two steps the float64 audit reports the non-finite state."""
    lbm = gpu()
    ctx = lbm.lbm_create("d3q27", "f32", (2, 1, 1), True, [], 1.5, 0.0)
    lbm.lbm_init_equilibrium(ctx, 0)
    f = lbm.lbm_get_state(ctx, 0)
    f[5, 3, 4, 5] = 1e39
    lbm.lbm_set_state(ctx, 0, f)
    lbm.lbm_step(ctx, 2)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_mass_momentum(ctx)
    assert e.value.status == lbm.LBM_ERR_NONFINITE
    close(ctx)


@pytest.mark.parametrize("model", MODELS)
def test_full_size_jet_grid_uniform_flow_invariance(model):
    """The 2-level jet grid at full size (coarse 384x192x192, 6.3 M fine
    cells) with x made periodic: a uniform flow passes the interfaces
    unchanged to FP32 round-off after 3 coarse steps."""
    lbm = gpu()
    flags, _ = synth.jet_two_level()
    ctx = lbm.lbm_create(model, "f32", (48, 24, 24), True, flags, 1.0 / 0.5003, 0.18)
    u0 = np.array([0.05, 0.02, -0.01])
    for l in range(2):
        NX, NY, NZ = ctx.dims(l)
        lbm.lbm_init_equilibrium(ctx, l, None, np.broadcast_to(u0[:, None, None, None], (3, NZ, NY, NX)).copy())
    lbm.lbm_step(ctx, 3)
    for l in range(2):
        rho, u = lbm.lbm_macroscopic(ctx, l)
        ok = ~np.isnan(rho)
        assert np.abs(rho[ok] - 1).max() < 2e-6
        assert np.abs(u[:, ok] - u0[:, None]).max() < 2e-6
    close(ctx)


def test_paper_scale_three_level_jet_runs():
    """The 3-level jet with 40.09 M active cells (1.08e9 D3Q27 values) builds,
    matches its plan and takes coarse steps with finite, sane audits."""
    lbm = gpu()
    flags, centre = synth.jet_paper_scale()
    info = lbm.lbm_plan((64, 32, 32), False, flags, "d3q27", "f32")
    assert sum(info.active_cells[l] for l in range(3)) == 40_091_648
    ctx = lbm.lbm_create("d3q27", "f32", (64, 32, 32), False, flags, 1.0 / (3 * 1.6e-4 + 0.5), 0.0)
    lbm.lbm_set_inflow(ctx, centre[0], centre[1], 32.0, 0.05, 0.01, 5120)
    lbm.lbm_step(ctx, 3)
    m = lbm.lbm_mass_momentum(ctx)
    assert np.isfinite(m).all() and m[1] > 0
    close(ctx)

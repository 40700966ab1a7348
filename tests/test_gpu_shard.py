"""Block sharding (the paper partitions its blocks over processes with a
halo exchange, Sections 1 and 3.2): a grid cut into 2 to 4 parts along x,
each part its own context with halo columns filled by the pack / copy /
unpack exchange before every coarse step, must reproduce the unsharded
context bit for bit on every level (same stream-collide variant for all
contexts).  Cases: uniform periodic (both models), an open channel with
inflow and outflow, 2- and 3-level grids with the refinement in the first
part (and a refined patch on the inflow face), the tank with walls, a
free-slip top and the pressure outlet, and the nozzle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SHAPE = "128,1,0"


def fields(nb, levels, seed):
    """Per-level (rho, u) of a Taylor-Green field plus a small seeded density
    ripple, so every population differs from cell to cell."""
    out = []
    rng = np.random.default_rng(seed)
    for l in range(levels):
        s = 8 << l
        NX, NY, NZ = nb[0] * s, nb[1] * s, nb[2] * s
        rho, u = synth.taylor_green_3d(NY, 0.03, shape=(NX, NY, NZ))
        rho = rho + 0.002 * rng.standard_normal(rho.shape)
        out.append((rho, u))
    return out


def run_both(monkeypatch, model, storage, nb, nparts, steps=6, periodic_x=True, refine=(), omega=1.7, cs=0.1,
             inflow=None, **kw):
    from paper_1206_0389_gb300 import lbm
    monkeypatch.setenv("LBM_LAUNCH_SHAPE", SHAPE)
    levels = len(refine) + 1
    fl = fields(nb, levels, 7)
    ctx = lbm.lbm_create(model, storage, nb, periodic_x, refine, omega, cs, **kw)
    sh = lbm.lbm_shard_create(model, storage, nb, periodic_x, refine, omega, cs, nparts, **kw)
    for l, (rho, u) in enumerate(fl):
        lbm.lbm_init_equilibrium(ctx, l, rho, u)
        lbm.lbm_shard_init_equilibrium(sh, l, rho, u)
    if inflow is not None:
        lbm.lbm_set_inflow(ctx, *inflow)
        lbm.lbm_shard_set_inflow(sh, *inflow)
    lbm.lbm_step(ctx, steps)
    lbm.lbm_shard_step(sh, steps)
    for l in range(levels):
        a, b = lbm.lbm_get_state(ctx, l), lbm.lbm_shard_get_state(sh, l)
        same = np.isnan(a) == np.isnan(b)
        assert same.all(), l
        m = ~np.isnan(a)
        assert m.any()
        assert np.array_equal(a[m], b[m]), (l, np.abs(a[m] - b[m]).max())
    ma, mb = lbm.lbm_mass_momentum(ctx), lbm.lbm_shard_mass_momentum(sh)
    assert np.abs(ma - mb).max() <= 1e-11 * max(1.0, np.abs(ma).max())
    cuts = [lbm.lbm_shard_part(sh, p)[1] for p in range(nparts)] + [nb[0]]
    halo = lbm.lbm_shard_halo_bytes(sh)
    lbm.lbm_destroy(ctx)
    lbm.lbm_shard_destroy(sh)
    return cuts, halo


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
@pytest.mark.parametrize("nparts", [2, 4])
def test_uniform_periodic_sharded_bitwise(monkeypatch, model, nparts):
    nb = (8, 2, 3)
    cuts, halo = run_both(monkeypatch, model, "f32", nb, nparts)
    assert cuts == {2: [0, 4, 8], 4: [0, 2, 4, 6, 8]}[nparts]
    # every cut (the periodic wrap included) moves one face layer each way:
    # 9 (D3Q27) or 5 (D3Q19) populations of 16 x 24 cells, 4 bytes each
    nq = 9 if model == "d3q27" else 5
    assert halo == nparts * 2 * nq * 16 * 24 * 4


def test_large_uniform_sharded_bitwise(monkeypatch):
    """128^3 in 4 parts whose steps overlap on their own streams: every
    exchange must wait for all parts' previous steps and every part's step
    for the exchange (many CTAs, ten coarse steps)."""
    nb = (16, 16, 16)
    cuts, _ = run_both(monkeypatch, "d3q27", "f32", nb, 4, steps=10)
    assert cuts == [0, 4, 8, 12, 16]


@pytest.mark.parametrize("storage", ["f64", "f16"])
def test_open_channel_with_inflow_sharded_bitwise(monkeypatch, storage):
    nb = (9, 2, 2)
    run_both(monkeypatch, "d3q27", storage, nb, 3, periodic_x=False, inflow=(8.0, 8.0, 8.0, 0.05, 0.01, 11))


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_two_level_sharded_bitwise(monkeypatch, model):
    """Refined blocks (a patch on the inflow face) in the first part only."""
    nb = (10, 3, 3)
    r = np.zeros((3, 3, 10), dtype=bool)
    r[1, 1, 0:2] = True
    cuts, _ = run_both(monkeypatch, model, "f32", nb, 3, periodic_x=False, refine=[r],
                       inflow=(12.0, 12.0, 8.0, 0.05, 0.01, 5))
    assert cuts[1] >= 4          # the first cut keeps clear of the refined columns


def test_three_level_sharded_bitwise(monkeypatch):
    nb = (12, 2, 2)
    r0 = np.zeros((2, 2, 12), dtype=bool)
    r0[:, :, 0:3] = True
    r1 = np.zeros((4, 4, 24), dtype=bool)
    r1[:, :, 1:4] = True
    run_both(monkeypatch, "d3q27", "f32", nb, 2, periodic_x=False, refine=[r0, r1],
             inflow=(8.0, 8.0, 8.0, 0.05, 0.01, 3))


def test_tank_with_walls_and_outlet_sharded_bitwise(monkeypatch):
    """No-slip side walls and bottom, free-slip top, no-slip upstream wall and
    the pressure outlet on the last part; a refined patch in the first part."""
    nb = (10, 4, 4)
    r = np.zeros((4, 4, 10), dtype=bool)
    r[1:3, 1:3, 1:3] = True
    run_both(monkeypatch, "d3q27", "f32", nb, 2, periodic_x=False, refine=[r], walls=15 | 16, slip=8, outlet=1)


@pytest.mark.parametrize("kw", [dict(walls=15, slip=8), dict(outlet=1), dict(walls=15 | 16, slip=8)])
def test_single_level_tank_faces_sharded_bitwise(monkeypatch, kw):
    nb = (10, 4, 4)
    run_both(monkeypatch, "d3q27", "f32", nb, 2, periodic_x=False, inflow=(16.0, 16.0, 8.0, 0.05, 0.01, 9), **kw)


def test_nozzle_alone_sharded_bitwise(monkeypatch):
    nb = (12, 4, 4)
    run_both(monkeypatch, "d3q27", "f32", nb, 2, periodic_x=False, nozzle=(16.0, 16.0, 4.0, 16.0, 32.0),
             inflow=(16.0, 16.0, 8.0, 0.05, 0.01, 9))


def test_nozzle_sharded_bitwise(monkeypatch):
    nb = (12, 4, 4)
    run_both(monkeypatch, "d3q27", "f32", nb, 2, periodic_x=False, walls=15, slip=8, outlet=1,
             nozzle=(16.0, 16.0, 4.0, 16.0, 32.0), inflow=(16.0, 16.0, 8.0, 0.05, 0.01, 9))


def test_shard_rejects_grids_without_admissible_cuts():
    from paper_1206_0389_gb300 import lbm
    flags, _ = synth.jet_two_level(8, 4, 4, radius=8.0)   # refined along the whole x extent
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_shard_create("d3q27", "f32", (8, 4, 4), False, flags, 1.7, 0.0, 2)
    assert e.value.status == lbm.LBM_ERR_ARG

"""GPU parity of the jet's radial profiles (Section 3.3 evaluates the mean
axial velocity, the spreading width, the Gaussian radial profile and the
turbulence intensity on cross-sections), computed on the device from the
accumulated statistics, against the oracle's ring averages of its own time
means (float64)."""
import math

import numpy as np
import pytest

from oracle.jetstats import jet_fit, radial_profile
from tests.helpers import gpu, init_both, make_pair
from tests.test_gpu_parity import jet_grid, nested_fields

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_radial_profiles_match_oracle(model):
    lbm = gpu()
    nb, ref = jet_grid(2)
    ctx, orc = make_pair(model, "f64", nb, False, ref, omega=1.7, cs=0.18)
    init_both(ctx, orc, nested_fields(orc))
    lbm.lbm_set_inflow(ctx, 8.0, 8.0, 8.0, 0.05, 0.01, 99)
    orc.set_inflow(8.0, 8.0, 8.0, 0.05, 0.01, 99)
    lbm.lbm_stats_reset(ctx)
    acc = [None, None]
    for _ in range(3):
        lbm.lbm_step(ctx, 1)
        orc.step(1)
        lbm.lbm_stats_accumulate(ctx)
        for l in range(2):
            _, uo = orc.macroscopic(l)
            ux = uo.numpy()[0]
            v = np.stack([ux, ux * ux])
            acc[l] = v if acc[l] is None else acc[l] + v
    y0 = z0 = 8.137
    for l, stations in ((0, [20.5, 27.0]), (1, [4.3, 11.9])):
        mo = acc[l][0] / 3
        vo = acc[l][1] / 3 - mo * mo
        pm, pv, pc = radial_profile(mo, vo, l, y0, z0, 0.9, 12, stations)
        gm, gv, gc = lbm.lbm_stats_radial(ctx, l, y0, z0, 0.9, 12, stations)
        assert np.array_equal(gc, pc)
        ok = pc > 0
        assert np.array_equal(np.isnan(gm), ~ok)
        assert np.abs(gm[ok] - pm[ok]).max() <= 1e-12
        assert np.abs(gv[ok] - pv[ok]).max() <= 1e-12
        for s in range(len(stations)):
            o = jet_fit(pm[s], pv[s], pc[s], 0.9)
            g = lbm.lbm_jet_fit(gm[s], gv[s], gc[s], 0.9)
            for a, b in zip(o, g):
                assert (math.isnan(a) and math.isnan(b)) or abs(a - b) <= 1e-9 * max(1.0, abs(a))
    # every level: unrefined cells weighted by their cross-section area
    from oracle.jetstats import radial_profile_levels
    parts = []
    for l in range(2):
        mo = acc[l][0] / 3
        vo = acc[l][1] / 3 - mo * mo
        parts.append((mo, vo, orc.real(l, orc.levels[l].active).numpy()))
    stations = [3.7, 9.2, 20.5]
    pm, pv, pc = radial_profile_levels(parts, y0, z0, 0.9, 12, stations)
    gm, gv, gc = lbm.lbm_stats_radial(ctx, -1, y0, z0, 0.9, 12, stations)
    assert np.array_equal(gc, pc)
    ok = pc > 0
    assert np.abs(gm[ok] - pm[ok]).max() <= 1e-12
    assert np.abs(gv[ok] - pv[ok]).max() <= 1e-12
    with pytest.raises(lbm.LbmError):
        lbm.lbm_stats_radial(ctx, 0, y0, z0, 0.9, 12, [40.0])      # outside the level
    lbm.lbm_destroy(ctx)

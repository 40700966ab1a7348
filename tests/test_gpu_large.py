"""GPU test of a level box whose buffers pass 2^31 elements: the periodic
wrap across z moves the pull by more than the int range, so the
stream-collide kernel must form its element offsets in 64 bits.  The field
depends on z only, so every (x, y) column of the large box must hold, bit
for bit, what the same column of a narrow box (8 x 8 cells across, same z
extent, small offsets) holds after the same steps."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,storage,nb", [("d3q19", "f16", (64, 64, 56)),
                                              ("d3q27", "f16", (48, 48, 72))])
def test_wrap_offsets_beyond_int32(model, storage, nb, monkeypatch):
    from paper_1206_0389_gb300 import lbm
    Q = 19 if model == "d3q19" else 27
    nblocks = nb[0] * nb[1] * nb[2]
    assert nblocks * Q * 512 >= 2 ** 31                           # buffer past the int range
    assert nb[0] * nb[1] * (nb[2] - 1) * Q * 512 >= 2 ** 31       # and so is the z wrap
    # one fixed launch shape on both sides (no autotuning: same instance)
    monkeypatch.setenv("LBM_AUTOTUNE", "0")
    NZ = 8 * nb[2]
    z = np.arange(NZ)
    uz_col = np.stack([0.04 * np.sin(2 * np.pi * z / NZ), 0.02 * np.cos(4 * np.pi * z / NZ),
                       0.01 * np.sin(6 * np.pi * z / NZ)])                     # [3][NZ]
    rho_col = 1.0 + 0.002 * np.cos(2 * np.pi * z / NZ)
    results = []
    for shape in (nb, (1, 1, nb[2])):
        NX, NY = 8 * shape[0], 8 * shape[1]
        ctx = lbm.lbm_create(model, storage, shape, True, [], 1.7, 0.1 if model == "d3q19" else 0.0)
        u = np.empty((3, NZ, NY, NX))
        u[...] = uz_col[:, :, None, None]
        rho = np.empty((NZ, NY, NX))
        rho[...] = rho_col[:, None, None]
        lbm.lbm_init_equilibrium(ctx, 0, rho, u)
        del u, rho
        lbm.lbm_step(ctx, 2)
        xs = [0, 1, NX // 2, NX - 1]
        ys = [0, NY - 1, NY // 3]
        zs = [0, 1, NZ // 2, NZ - 2, NZ - 1]
        cells = np.array([x + NX * (y + NY * zz) for zz in zs for y in ys for x in xs], dtype=np.int64)
        f = lbm.lbm_get_cells(ctx, 0, cells).reshape(len(zs), len(ys) * len(xs), Q)
        results.append(f)
        lbm.lbm_destroy(ctx)
    big, small = results
    assert np.isfinite(big).all()
    # every sampled column of the large box equals the narrow box's columns
    for k in range(big.shape[1]):
        assert np.array_equal(big[:, k], small[:, 0])
    assert np.array_equal(small[:, 0], small[:, -1])
    # and the state is not trivially uniform along z
    assert np.abs(big[0, 0] - big[2, 0]).max() > 1e-4

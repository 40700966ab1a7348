"""GPU test of lbm_mass_momentum_noalloc, the audit entry point for callers
that cannot let the library allocate device memory (stream capture, a
framework's own memory pool, allocation-free loops).  It must give the same
float64 sums as lbm_mass_momentum on the same distributions, on two calls in
a row that share its static scratch array.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def storage_layout(f_dense, model, storage):
    """Dense unshifted [Q][NZ][NY][NX] float64 -> the library's block storage
    [block][Q][512] of a single periodic level (block id bx + BX (by + BY bz))."""
    from oracle.lattice import weights
    Q, NZ, NY, NX = f_dense.shape
    w = weights(Q).numpy()
    g = f_dense - (w[:, None, None, None] if model == "d3q27" else 0.0)
    if storage == "f16":
        g = g / w[:, None, None, None]
    BZ, BY, BX = NZ // 8, NY // 8, NX // 8
    b = g.reshape(Q, BZ, 8, BY, 8, BX, 8).transpose(1, 3, 5, 0, 2, 4, 6)
    dt = {"f64": np.float64, "f32": np.float32, "f16": np.float16}[storage]
    return np.ascontiguousarray(b.reshape(-1)).astype(dt), BX * BY * BZ


@pytest.mark.parametrize("model,storage", [("d3q27", "f32"), ("d3q19", "f64"), ("d3q27", "f16")])
def test_noalloc_audit_matches_mass_momentum_twice(model, storage):
    """Two calls in a row: the second on a smaller grid (fewer blocks, new
    contents), so slots the first call filled beyond the second call's
    range stay stale in the shared array and must not leak into its sums."""
    from paper_1206_0389_gb300 import lbm
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call, (nb, steps) in enumerate((((4, 3, 2), 0), ((2, 2, 1), 3))):
        shape = tuple(8 * n for n in nb)
        ctx = lbm.lbm_create(model, storage, nb, True, [], 1.6, 0.1)
        rho, u = synth.taylor_green_3d(shape[0], 0.05, shape=shape)
        rho = rho + 0.01 * np.sin(np.arange(shape[2]))[:, None, None]
        lbm.lbm_init_equilibrium(ctx, 0, rho, u)
        lbm.lbm_step(ctx, steps)
        ref = lbm.lbm_mass_momentum(ctx)
        host, nblocks = storage_layout(lbm.lbm_get_state(ctx, 0), model, storage)
        assert nblocks == nb[0] * nb[1] * nb[2]
        dev = torch.from_numpy(host).cuda()
        out.fill_(float("nan"))
        lbm.lbm_mass_momentum_noalloc(model, storage, dev.data_ptr(), nblocks, out.data_ptr(),
                                      stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (call, got, ref)
        lbm.lbm_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    from paper_1206_0389_gb300 import lbm
    x = torch.zeros(27 * 512, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_mass_momentum_noalloc("d3q27", "f32", x.data_ptr(), lbm.NOALLOC_MAX_BLOCKS + 1,
                                      out.data_ptr())
    assert e.value.status == lbm.LBM_ERR_ARG
    st = lbm.load().lbm_mass_momentum_noalloc(1, 1, None, 1, None, None)
    assert st == lbm.LBM_ERR_ARG
    st = lbm.load().lbm_mass_momentum_noalloc(1, 1, x.data_ptr(), lbm.NOALLOC_MAX_BLOCKS + 1,
                                              out.data_ptr(), None)
    assert st == lbm.LBM_ERR_ARG

"""GPU adjoint of the forced D3Q27 FCLB update through the C ABI and the
torch.autograd.Function: against the FP64 oracle's autograd gradient (16^3)
and against central finite differences of the FP64 GPU forward (20 random
unit directions, h = 1e-4), including the 96^3, T = 256, checkpoint-16 case."""
import numpy as np
import pytest
import torch

import synth
from oracle.adjoint import kinetic_energy_loss, reference_gradient
from oracle.collision import feq_fclb

pytestmark = pytest.mark.gpu


def initial_state(N, seed):
    rho, u = synth.spectrum_field(N, seed=seed)
    return feq_fclb(torch.from_numpy(rho).reshape(-1),
                    torch.from_numpy(u).reshape(3, -1)).reshape(27, N, N, N).numpy()


def gpu_gradient(lbm, storage, f0, F, T, every, region, omega):
    from paper_1206_0389_gb300.autograd import forced_fclb
    N = f0.shape[-1]
    ctx = lbm.lbm_create("d3q27", storage, (N // 8,) * 3, True, [], omega, 0.0)
    Ft = torch.from_numpy(F).clone().requires_grad_(True)
    fT = forced_fclb(Ft, ctx, f0, T, every)
    L = kinetic_energy_loss(fT, Ft, region)
    L.backward()
    lbm.lbm_destroy(ctx)
    return float(L.detach()), Ft.grad.numpy()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 2e-4)])
def test_adjoint_matches_oracle_reference_gradient(storage, tol):
    """16^3, T = 10 with checkpoints every 4 (segments 4, 4, 2)."""
    from paper_1206_0389_gb300 import lbm
    N, T, every, omega = 16, 10, 4, 1.0 / 0.53
    f0 = initial_state(N, 4)
    F = synth.random_force((N, N, N), 4096, sigma=1e-4)
    region = (4, 12, 4, 12, 4, 12)
    Lg, gg = gpu_gradient(lbm, storage, f0, F, T, every, region, omega)
    Lo, go = reference_gradient(torch.from_numpy(f0), torch.from_numpy(F), (2, 2, 2), omega, T, region)
    go = go.numpy()
    err = np.abs(gg - go).max() / np.abs(go).max()
    print(storage, "max rel gradient error vs oracle:", err)
    assert abs(Lg - Lo) <= 1e-9 * abs(Lo) if storage == "f64" else abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert err <= tol


def fd_check(N, T, every, storage, ndir, tol):
    from paper_1206_0389_gb300 import lbm
    omega = 1.0 / (3 * 0.005 + 0.5)
    f0 = initial_state(N, 4096)
    F = synth.random_force((N, N, N), 4096, sigma=1e-6)
    c = N // 2
    region = (c - 8, c + 8, c - 8, c + 8, c - 8, c + 8)
    _, g = gpu_gradient(lbm, storage, f0, F, T, every, region, omega)
    ctx = lbm.lbm_create("d3q27", "f64", (N // 8,) * 3, True, [], omega, 0.0)

    def loss(Fv):
        lbm.lbm_set_state(ctx, 0, f0)
        lbm.lbm_set_force(ctx, Fv)
        lbm.lbm_step(ctx, T)
        fT = torch.from_numpy(lbm.lbm_get_state(ctx, 0))
        return float(kinetic_energy_loss(fT, torch.from_numpy(Fv), region))

    h = 1e-4
    dirs = synth.random_directions(ndir, (N, N, N), 20)
    fd, ad = [], []
    for d in dirs:
        fd.append((loss(F + h * d) - loss(F - h * d)) / (2 * h))
        ad.append(float((g * d).sum()))
    lbm.lbm_destroy(ctx)
    fd, ad = np.array(fd), np.array(ad)
    err = np.abs(fd - ad).max() / np.abs(fd).max()
    print("FD directional derivatives:", fd[:4], "adjoint:", ad[:4], "max rel err:", err)
    assert err <= tol


def test_adjoint_central_differences_small():
    fd_check(16, 32, 8, "f64", 20, 1e-6)


def test_adjoint_central_differences_96_cubed_t256():
    """96^3 periodic FCLB, FP32 forward and adjoint, T = 256, checkpoints every
    16; loss = kinetic energy of the central 16^3 at T; force N(0, 1e-6)."""
    fd_check(96, 256, 16, "f32", 20, 2e-3)


def test_adjoint_rejects_unsupported_contexts():
    from paper_1206_0389_gb300 import lbm
    ctx = lbm.lbm_create("d3q19", "f32", (1, 1, 1))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_forward(ctx, 4, 2)
    assert e.value.status == lbm.LBM_ERR_STATE
    lbm.lbm_destroy(ctx)
    ctx = lbm.lbm_create("d3q27", "f32", (1, 1, 1))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_backward(ctx, np.zeros((27, 8, 8, 8)))
    assert e.value.status == lbm.LBM_ERR_STATE
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_forward(ctx, 4, 5)
    assert e.value.status == lbm.LBM_ERR_ARG
    lbm.lbm_destroy(ctx)

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


def _backward_with(lbm, ctx, f0, F, T, every, lam):
    lbm.lbm_set_state(ctx, 0, f0)
    lbm.lbm_set_force(ctx, F)
    lbm.lbm_adjoint_forward(ctx, T, every)
    fT = lbm.lbm_get_state(ctx, 0)
    return fT, lbm.lbm_adjoint_backward(ctx, lam)


def test_store_every_state_equals_checkpointing_bit_for_bit():
    """checkpoint_every = 1 keeps every state (no recomputation), 0 lets the
    library choose, 3 checkpoints; the recomputed states are the same
    kernel's outputs, so final states and gradients agree bit for bit."""
    from paper_1206_0389_gb300 import lbm
    N, T = 16, 7
    f0 = initial_state(N, 11)
    F = synth.random_force((N, N, N), 11, sigma=1e-4)
    lam = np.random.default_rng(5).standard_normal((27, N, N, N)) * 1e-3
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.0 / 0.53, 0.0)
    fT1, g1 = _backward_with(lbm, ctx, f0, F, T, 1, lam)
    assert lbm.lbm_adjoint_generation(ctx)[1] == 1
    fT3, g3 = _backward_with(lbm, ctx, f0, F, T, 3, lam)
    fT0, g0 = _backward_with(lbm, ctx, f0, F, T, 0, lam)
    assert lbm.lbm_adjoint_generation(ctx)[1] == 1   # a 16^3 grid fits: every state kept
    assert np.array_equal(fT1, fT3) and np.array_equal(fT1, fT0)
    assert np.array_equal(g1, g3) and np.array_equal(g1, g0)
    # the plain stepping path reaches the same final state
    lbm.lbm_set_state(ctx, 0, f0)
    lbm.lbm_set_force(ctx, F)
    lbm.lbm_step(ctx, T)
    assert np.array_equal(lbm.lbm_get_state(ctx, 0), fT1)
    lbm.lbm_destroy(ctx)


def test_failed_adjoint_allocation_frees_everything_and_retry_works(monkeypatch):
    """A host-side injected allocation failure (the k-th adjoint buffer) makes
    the forward return LBM_ERR_OOM and discard the record; the retry
    allocates everything again and gives the gradient of a clean context."""
    from paper_1206_0389_gb300 import lbm
    N, T = 16, 6
    f0 = initial_state(N, 12)
    F = synth.random_force((N, N, N), 12, sigma=1e-4)
    lam = np.random.default_rng(6).standard_normal((27, N, N, N)) * 1e-3
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], 1.0 / 0.53, 0.0)
    _, gref = _backward_with(lbm, ctx, f0, F, T, 2, lam)
    # a longer horizon needs more checkpoints: the buffers are allocated anew
    for k in (1, 7, 9):          # a checkpoint, a segment buffer, a lambda buffer
        lbm.lbm_set_state(ctx, 0, f0)
        lbm.lbm_set_force(ctx, F)
        monkeypatch.setenv("LBM_INJECT_ADJOINT_OOM", str(k))
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_adjoint_forward(ctx, 2 * T, 2)
        assert e.value.status == lbm.LBM_ERR_OOM
        monkeypatch.delenv("LBM_INJECT_ADJOINT_OOM")
        assert lbm.lbm_adjoint_generation(ctx) == (0, 0)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_adjoint_backward(ctx, lam)
        assert e.value.status == lbm.LBM_ERR_STATE
        _, g = _backward_with(lbm, ctx, f0, F, T, 2, lam)
        assert np.array_equal(g, gref)
    lbm.lbm_destroy(ctx)


def test_second_forward_or_new_force_invalidates_the_first_graph_node():
    from paper_1206_0389_gb300 import lbm
    from paper_1206_0389_gb300.autograd import forced_fclb
    N, T, omega = 16, 4, 1.0 / 0.53
    f0 = initial_state(N, 13)
    F = synth.random_force((N, N, N), 13, sigma=1e-4)
    region = (4, 12, 4, 12, 4, 12)
    ctx = lbm.lbm_create("d3q27", "f32", (2, 2, 2), True, [], omega, 0.0)
    F1 = torch.from_numpy(F).clone().requires_grad_(True)
    F2 = torch.from_numpy(2 * F).clone().requires_grad_(True)
    L1 = kinetic_energy_loss(forced_fclb(F1, ctx, f0, T, 2), F1, region)
    L2 = kinetic_energy_loss(forced_fclb(F2, ctx, f0, T, 2), F2, region)
    with pytest.raises(RuntimeError, match="another adjoint forward"):
        L1.backward()
    L2.backward()                  # the latest forward's node still works
    g2 = F2.grad.numpy().copy()
    F3 = torch.from_numpy(2 * F).clone().requires_grad_(True)
    kinetic_energy_loss(forced_fclb(F3, ctx, f0, T, 2), F3, region).backward()
    assert np.array_equal(g2, F3.grad.numpy())
    # a new force after the forward discards the record in the library too
    lbm.lbm_set_state(ctx, 0, f0)
    lbm.lbm_set_force(ctx, F)
    lbm.lbm_adjoint_forward(ctx, T, 2)
    gen = lbm.lbm_adjoint_generation(ctx)[0]
    assert gen == 4
    lbm.lbm_set_force(ctx, 2 * F)
    assert lbm.lbm_adjoint_generation(ctx) == (0, 0)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint_backward(ctx, np.zeros((27, N, N, N)))
    assert e.value.status == lbm.LBM_ERR_STATE
    lbm.lbm_destroy(ctx)

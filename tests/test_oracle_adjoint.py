"""Pin of the oracle's reference gradient (autograd through the FP64 forced
FCLB forward) against central finite differences of the same forward."""
import torch

import synth
from oracle.adjoint import forward_final_state, kinetic_energy_loss, reference_gradient
from oracle.collision import feq_fclb


def test_reference_gradient_matches_central_differences():
    rho, u = synth.spectrum_field(8, seed=3)
    f0 = feq_fclb(torch.from_numpy(rho).reshape(-1), torch.from_numpy(u).reshape(3, -1)).reshape(27, 8, 8, 8)
    F = torch.from_numpy(synth.random_force((8, 8, 8), 4, sigma=1e-4))
    region = (2, 6, 2, 6, 2, 6)
    L, g = reference_gradient(f0, F, (1, 1, 1), 1.6, 6, region)
    dirs = torch.from_numpy(synth.random_directions(3, (8, 8, 8), 5))
    h = 1e-4
    for d in dirs:
        Lp = float(kinetic_energy_loss(forward_final_state(f0, F + h * d, (1, 1, 1), 1.6, 6), F + h * d, region))
        Lm = float(kinetic_energy_loss(forward_final_state(f0, F - h * d, (1, 1, 1), 1.6, 6), F - h * d, region))
        fd = (Lp - Lm) / (2 * h)
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-12, (fd, ad)

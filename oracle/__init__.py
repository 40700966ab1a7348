"""Plain FP64 CPU oracle of the nested-grid lattice Boltzmann update.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method of Geller, Uphoff & Krafczyk, "Turbulent jet
computations based on MRT and Cascaded Lattice Boltzmann models"
(Section 2 and Section 3.2), written from the paper in float64 with plain
PyTorch CPU ops.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never imports, links or calls it, and it shares no code,
table or constant with the CUDA path: the lattice tables below are typed
again from the paper's tables.

Modules
-------
lattice    velocity sets, weights and opposite map (Section 2 tables)
collision  D3Q19 MRT + Smagorinsky (Eqs. MRT, relaxationTau, eqSmago,
           eqTauTotFinal, EqnQ; Table 1) and D3Q27 factorized cascaded
           collision by the central-moment definition (Table 2)
grid       cell masks of the block-structured, 2:1 nested grid
solver     streaming, boundary ghosts (inflow, zero-gradient or pressure
           outlet), walls (no-slip / free-slip), coarse-to-fine /
           fine-to-coarse interface transfer and the time-nested schedule
nozzle     the nozzle cylinder: solid cells, Bouzidi interpolated no-slip
           links and the inflow on its cap (Section 3.2)
jetstats   ring profiles, centreline velocity, half width, turbulence
           intensity and Gaussian fit of time averages (Section 3.3)
rng        SplitMix64 counter hash used for the inflow perturbation
adjoint    reference gradient of a loss w.r.t. a body force (autograd of
           the forward oracle)

Parity status: every function here is pinned by ``tests/test_oracle_*.py``.
"""
import torch

DTYPE = torch.float64

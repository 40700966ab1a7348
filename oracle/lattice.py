"""Velocity sets of Section 2 (the D3Q19 and D3Q27 tables), typed from the paper.

The column order is the paper's: index i of each list is the velocity e_i of
the printed table.  Weights: D3Q19 w = 1/3, 1/18, 1/36 and D3Q27
w = 8/27, 2/27, 1/54, 1/216 by |e|^2 = 0, 1, 2, 3 (Section 2, text after the
incompressible equilibrium).  Lattice speed c = 1.
"""
import torch

from . import DTYPE

# D3Q19 table, i = 0..18 (Section 2)
_D3Q19 = (
    (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0),
    (0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1),
    (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1),
)
# D3Q27 table in two printed parts, i = 0..15 and i = 16..26 (Section 2)
_D3Q27_A = (
    (0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0),
    (0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1),
    (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1),
)
_D3Q27_B = (
    (0, 0, 0, 1, -1, 1, 1, -1, -1, 1, -1),
    (-1, 1, -1, 1, 1, -1, 1, -1, 1, -1, -1),
    (-1, -1, 1, 1, 1, 1, -1, 1, -1, -1, -1),
)

_W19 = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
_W27 = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}


def velocities(Q: int) -> torch.Tensor:
    """(Q, 3) integer tensor of the lattice velocities e_i in table order."""
    if Q == 19:
        cols = list(zip(*_D3Q19))
    elif Q == 27:
        cols = list(zip(*_D3Q27_A)) + list(zip(*_D3Q27_B))
    else:
        raise ValueError("Q must be 19 or 27")
    return torch.tensor(cols, dtype=torch.int64)


def weights(Q: int) -> torch.Tensor:
    """Lattice weights w_i, chosen by |e_i|^2 as the paper lists them."""
    e = velocities(Q)
    table = _W19 if Q == 19 else _W27
    return torch.tensor([table[int((v * v).sum())] for v in e], dtype=DTYPE)


def opposite(Q: int) -> list:
    """opp[i] = j with e_j = -e_i, found by search (never by index parity)."""
    e = velocities(Q).tolist()
    return [e.index([-a for a in v]) for v in e]

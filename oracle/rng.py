"""Counter-based random numbers for the inflow perturbation.

SplitMix64 (Steele, Lea & Flood 2014, "Fast splittable pseudorandom number
generators"; constants as published by Vigna): the state is advanced by the
golden gamma 0x9E3779B97F4A7C15 and passed through the variant-13 mixer.

The perturbation drawn for one boundary value is the chain
    h = sm(seed); h = sm(h ^ coarse_step); h = sm(h ^ (level << 32 | substep));
    h = sm(h ^ cell); h = sm(h ^ component)
and xi = 2 (h >> 11) 2^-53 - 1 in [-1, 1).  This chain is the library's
documented convention (the paper only says the inflow velocity is constant).
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """One SplitMix64 output for state x (numpy uint64 array, wraps mod 2^64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def inflow_xi(seed, coarse_step, level, substep, cell, component):
    """xi in [-1, 1) for each element of `cell` (int array); other args scalars."""
    h = splitmix64(np.uint64(seed))
    h = splitmix64(h ^ np.uint64(coarse_step))
    h = splitmix64(h ^ np.uint64((int(level) << 32) | int(substep)))
    h = splitmix64(h ^ np.asarray(cell, dtype=np.uint64))
    h = splitmix64(h ^ np.uint64(component))
    return 2.0 * (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 1.0

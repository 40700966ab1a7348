"""Pins of the oracle's lattice tables (Section 2) by exact isotropy sums."""
import itertools
from fractions import Fraction

import pytest

from oracle.lattice import opposite, velocities, weights

W19 = {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)}
W27 = {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)}


def _exact(Q):
    e = velocities(Q).tolist()
    table = W19 if Q == 19 else W27
    return e, [table[sum(c * c for c in v)] for v in e]


@pytest.mark.parametrize("Q", [19, 27])
def test_velocity_set_shape(Q):
    e = velocities(Q).tolist()
    assert len(e) == Q and len({tuple(v) for v in e}) == Q
    assert e[0] == [0, 0, 0]
    if Q == 27:
        assert sorted(map(tuple, e)) == sorted(itertools.product((-1, 0, 1), repeat=3))
    else:
        assert all(sum(c * c for c in v) <= 2 for v in e)
        assert velocities(27).tolist()[:19] == e


@pytest.mark.parametrize("Q", [19, 27])
def test_isotropy_exact(Q):
    """sum w = 1, sum w e_a e_b = delta/3, fourth moment (dd+dd+dd)/9, odd = 0."""
    e, w = _exact(Q)
    d = lambda a, b: 1 if a == b else 0
    assert sum(w) == 1
    for a in range(3):
        assert sum(wi * v[a] for wi, v in zip(w, e)) == 0
        for b in range(3):
            assert sum(wi * v[a] * v[b] for wi, v in zip(w, e)) == Fraction(d(a, b), 3)
            for c in range(3):
                assert sum(wi * v[a] * v[b] * v[c] for wi, v in zip(w, e)) == 0
                for g in range(3):
                    s = sum(wi * v[a] * v[b] * v[c] * v[g] for wi, v in zip(w, e))
                    assert s == Fraction(d(a, b) * d(c, g) + d(a, c) * d(b, g) + d(a, g) * d(b, c), 9)


@pytest.mark.parametrize("Q", [19, 27])
def test_weights_float_match_exact(Q):
    _, w = _exact(Q)
    assert weights(Q).tolist() == [float(x) for x in w]


def test_d3q27_weights_are_a_tensor_product():
    """w(e) = w1(e_x) w1(e_y) w1(e_z) with the D1Q3 weights 2/3, 1/6."""
    e, w = _exact(27)
    w1 = {0: Fraction(2, 3), 1: Fraction(1, 6), -1: Fraction(1, 6)}
    assert all(wi == w1[v[0]] * w1[v[1]] * w1[v[2]] for wi, v in zip(w, e))


@pytest.mark.parametrize("Q", [19, 27])
def test_opposite_map(Q):
    opp = opposite(Q)
    e = velocities(Q).tolist()
    for i, j in enumerate(opp):
        assert e[j] == [-c for c in e[i]] and opp[j] == i
    if Q == 27:
        assert opp == [0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17,
                       26, 25, 24, 23, 22, 21, 20, 19]

"""Pins of the oracle's lattice tables against the guide and exact lattice algebra.

D2Q9 is checked entry by entry against the listing "Definition of the D2Q9
descriptor" (section "Descriptor"); both lattices are checked against the exact
isotropy identities a second-order lattice must satisfy (sum w = 1, sum w c = 0,
sum w c c = cs2 I, third moments vanish, fourth moments = cs2^2 (dd + dd + dd)).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_d2q9():
    rows = []
    with open(os.path.join(GOLDEN, "d2q9_descriptor.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


def test_d2q9_matches_the_printed_listing(oracle):
    dim, q, c, opp, w, cs2 = oracle.descriptor(oracle.D2Q9)
    rows = _golden_d2q9()
    assert (dim, q) == (2, 9) and len(rows) == 9
    for i, cx, cy, o, num, den in rows:
        assert tuple(c[i]) == (cx, cy, 0)
        assert opp[i] == o
        assert w[i] == num / den
    assert cs2 == 1.0 / 3.0
    # The two examples printed above the listing.
    assert tuple(c[1][:2]) == (-1, 1) and w[0] == 4.0 / 9.0


def _exact(w):
    return [Fraction(x).limit_denominator(1000) for x in w]


@pytest.mark.parametrize("d", [0, 1])
def test_isotropy_identities_exact(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    W = _exact(w)
    assert all(abs(float(Wi) - wi) == 0.0 for Wi, wi in zip(W, w))
    cs = Fraction(1, 3)
    assert sum(W) == 1
    for a in range(3):
        assert sum(W[i] * c[i][a] for i in range(q)) == 0
    for a, b in itertools.product(range(dim), repeat=2):
        assert sum(W[i] * c[i][a] * c[i][b] for i in range(q)) == (cs if a == b else 0)
    for a, b, g in itertools.product(range(dim), repeat=3):
        assert sum(W[i] * c[i][a] * c[i][b] * c[i][g] for i in range(q)) == 0
    for a, b, g, e in itertools.product(range(dim), repeat=4):
        lhs = sum(W[i] * c[i][a] * c[i][b] * c[i][g] * c[i][e] for i in range(q))
        delta = lambda x, y: 1 if x == y else 0
        rhs = cs * cs * (delta(a, b) * delta(g, e) + delta(a, g) * delta(b, e)
                         + delta(a, e) * delta(b, g))
        assert lhs == rhs


@pytest.mark.parametrize("d", [0, 1])
def test_opposites_and_velocity_set(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    for i in range(q):
        assert tuple(c[opp[i]]) == tuple(-c[i])
        assert w[opp[i]] == w[i]
    assert len({tuple(v) for v in c}) == q  # no duplicates
    assert tuple(c[0]) == (0, 0, 0)


def test_d3q19_set_and_ordering_reading(oracle):
    dim, q, c, opp, w, cs2 = oracle.descriptor(oracle.D3Q19)
    assert (dim, q) == (3, 19)
    expected = {v for v in itertools.product((-1, 0, 1), repeat=3)
                if sum(abs(x) for x in v) in (0, 1, 2)}
    assert {tuple(v) for v in c} == expected
    norms = np.abs(c).sum(axis=1)
    assert np.all(w[norms == 0] == 1.0 / 3.0)
    assert np.all(w[norms == 1] == 1.0 / 18.0)
    assert np.all(w[norms == 2] == 1.0 / 36.0)
    # Ordering rule of the D2Q9 listing applied to D3Q19: indices 1..9 start with -1
    # as first non-zero component, index i+9 is the opposite of i.
    for i in range(1, 10):
        first = next(x for x in c[i] if x != 0)
        assert first == -1
        assert opp[i] == i + 9 and opp[i + 9] == i

"""Pins the oracle's exact orientation sign against rational arithmetic.

The walk of Algorithm 1 and the containment test of the oracle both rest on
the signs of the barycentric coordinates (Eq. 6); their numerators are
orientation determinants.  A sign that is wrong near a degeneracy would move a
foot into the wrong triangle, so the predicate is checked on inputs built to
defeat double-precision evaluation.
"""
import math
import random

import numpy as np
import pytest

import oracle
from exact import orient as exact_orient


def _cases(seed=1):
    rnd = random.Random(seed)
    out = []
    # random points in the unit square
    for _ in range(400):
        out.append(tuple(rnd.random() for _ in range(6)))
    # exactly collinear triples on dyadic lines
    for _ in range(200):
        ax, ay = rnd.randint(0, 2**20) / 2**20, rnd.randint(0, 2**20) / 2**20
        dx, dy = rnd.randint(-2**10, 2**10) / 2**12, rnd.randint(-2**10, 2**10) / 2**12
        s, r = rnd.randint(-8, 8) / 8, rnd.randint(-8, 8) / 8
        out.append((ax, ay, ax + s * dx, ay + s * dy, ax + r * dx, ay + r * dy))
    # a third point a few ulps off the line through two others (double
    # evaluation is unreliable here)
    for _ in range(400):
        ax, ay, bx, by = (rnd.random() for _ in range(4))
        s = rnd.random()
        cx = ax + s * (bx - ax)
        cy = ay + s * (by - ay)
        for _ in range(rnd.randint(0, 4)):
            cx = math.nextafter(cx, rnd.choice((-1.0, 2.0)))
            cy = math.nextafter(cy, rnd.choice((-1.0, 2.0)))
        out.append((ax, ay, bx, by, cx, cy))
    # points on long thin configurations and near-equal coordinates
    for _ in range(200):
        base = rnd.random()
        eps = [rnd.choice((0.0, 1.0, -1.0)) * rnd.randint(1, 5) * 2.0**-52 for _ in range(6)]
        out.append(tuple(base + e for e in eps))
    # tiny and huge magnitudes (exercise the exact path's scaling)
    for _ in range(100):
        sc = 2.0 ** rnd.randint(-700, 700)
        out.append(tuple(sc * rnd.random() for _ in range(6)))
    out.append((0.0, 0.0, 1.0, 0.0, 0.5, 0.0))                       # on the edge line
    out.append((0.0, 0.0, 0.0, 0.0, 0.3, 0.7))                       # repeated point
    out.append((5e-324, 0.0, 0.0, 5e-324, 1e-323, 1e-323))           # subnormals
    return out


@pytest.mark.parametrize("force_exact", [False, True])
def test_orient_sign_matches_rationals(force_exact):
    L = oracle.lib()
    L.orc_set_force_exact(1 if force_exact else 0)
    try:
        bad = []
        for c in _cases():
            got = L.orc_orient_sign(*c)
            want = exact_orient(c[0:2], c[2:4], c[4:6])
            if got != want:
                bad.append((c, got, want))
        assert not bad, bad[:5]
    finally:
        L.orc_set_force_exact(0)


def test_filter_is_exercised():
    """The near-degenerate cases must actually reach the exact path, and
    give a zero sign on exact collinearity."""
    L = oracle.lib()
    before = L.orc_exact_calls()
    assert L.orc_orient_sign(0.1, 0.1, 0.3, 0.3, 0.7, 0.7) == exact_orient((0.1, 0.1), (0.3, 0.3), (0.7, 0.7))
    assert L.orc_orient_sign(0.0, 0.0, 0.5, 0.5, 0.25, 0.25) == 0
    assert L.orc_exact_calls() > before


def test_orient_antisymmetry_and_cyclic():
    rnd = np.random.default_rng(3)
    for _ in range(300):
        a, b, c = rnd.random(2), rnd.random(2), rnd.random(2)
        s = oracle.orient_sign(a, b, c)
        assert oracle.orient_sign(b, c, a) == s
        assert oracle.orient_sign(b, a, c) == -s

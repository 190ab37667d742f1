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
from fractions import Fraction as F

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


def _exact_orient_pair(a, b, qh, ql):
    """orient(a, b, qh + ql) in rationals."""
    ax, ay, bx, by = (F(float(v)) for v in (a[0], a[1], b[0], b[1]))
    qx, qy = F(float(qh[0])) + F(float(ql[0])), F(float(qh[1])) + F(float(ql[1]))
    d = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax)
    return (d > 0) - (d < 0)


def _split(v):
    """A rational v as (hi, lo) doubles with hi + lo == v exactly."""
    hi = float(v)
    lo = float(v - F(hi))
    assert F(hi) + F(lo) == v, "test construction: remainder not representable"
    return hi, lo


def _pair_cases(seed=5):
    rnd = random.Random(seed)
    out = []
    # random points with a remainder below half an ulp of the high part
    for _ in range(300):
        a, b = (rnd.random(), rnd.random()), (rnd.random(), rnd.random())
        qh = (rnd.random(), rnd.random())
        ql = tuple(rnd.uniform(-1, 1) * 2.0 ** rnd.randint(-80, -54) for _ in range(2))
        out.append((a, b, qh, ql))
    # points exactly on the line a-b whose high part is not: a + s (b - a)
    # with s carrying 70 bits, so the coordinates need more than one double;
    # then the same point nudged by one ulp of its remainder either way
    for _ in range(300):
        a = (F(rnd.randint(0, 2**20), 2**20), F(rnd.randint(0, 2**20), 2**20))
        b = (F(rnd.randint(0, 2**20), 2**20), F(rnd.randint(0, 2**20), 2**20))
        s = F(rnd.randint(1, 2**70 - 1), 2**70)
        q = (a[0] + s * (b[0] - a[0]), a[1] + s * (b[1] - a[1]))
        (xh, xl), (yh, yl) = _split(q[0]), _split(q[1])
        af, bf = (float(a[0]), float(a[1])), (float(b[0]), float(b[1]))
        out.append((af, bf, (xh, yh), (xl, yl)))
        for d in (-1.0, 1.0):
            out.append((af, bf, (xh, yh), (math.nextafter(xl, d * math.inf) if xl else d * 2.0**-1074, yl)))
            out.append((af, bf, (xh, yh), (xl, math.nextafter(yl, d * math.inf) if yl else d * 2.0**-1074)))
    # a remainder that is subnormal, and one that cancels the high part's offset
    out.append(((0.0, 0.0), (1.0, 1.0), (0.5, 0.5), (5e-324, 0.0)))
    out.append(((0.0, 0.0), (1.0, 1.0), (0.5, 0.5), (0.0, -5e-324)))
    out.append(((0.0, 0.0), (1.0, 0.0), (0.3, 2.0**-60), (0.0, -2.0**-60)))
    return out


@pytest.mark.parametrize("force_exact", [False, True])
def test_orient_sign_of_pair_points_matches_rationals(force_exact):
    """The sign for a point given as an exact sum of two doubles per
    coordinate (a double-float foot), against rationals, with and without
    the double filter; zero exactly when the sum lies on the line."""
    bad = []
    zeros = 0
    for a, b, qh, ql in _pair_cases():
        got = oracle.orient_sign2(a, b, qh, ql, force_exact=force_exact)
        want = _exact_orient_pair(a, b, qh, ql)
        zeros += want == 0
        if got != want:
            bad.append((a, b, qh, ql, got, want))
    assert not bad, bad[:5]
    assert zeros >= 300


def test_orient_sign_of_pair_points_with_zero_remainder_is_the_plain_sign():
    rnd = np.random.default_rng(9)
    for _ in range(300):
        a, b, c = rnd.random(2), rnd.random(2), rnd.random(2)
        assert oracle.orient_sign2(a, b, c, (0.0, 0.0)) == oracle.orient_sign(a, b, c)

"""Pins the oracle's point location.

(1) Brute force: on tiny meshes every triangle is tested with rational
    arithmetic; the oracle must return the lowest-index containing triangle,
    flag degeneracy (a zero sign) and multiplicity exactly.
(2) The paper's direct location formula on the structured Courant grid
    (Sec. 4, comparison with a structured grid): for a point (xi, eta) of the
    grid with M cells per side, l = floor(xi / dx), m = floor(eta / dx), and
    the point lies in the upper triangle of cell (l, m) when
    xi - l dx < eta - m dx, else in the lower one.  With this repository's
    numbering (0-based, [0,1]^2) the upper triangle is 2 (M m + l) and the
    lower one 2 (M m + l) + 1, which is the paper's T_{2(Mm+l)+1} and
    T_{2(Mm+l+1)} shifted to 0-based indices.
"""
from fractions import Fraction as F
import math
import random

import numpy as np
import pytest

import oracle
import sl_inputs as si
from sl_inputs.meshes import shuffled
from exact import contains


def _queries(mesh, rnd, n_random=300):
    xy = mesh.xy
    q = [(rnd.random(), rnd.random()) for _ in range(n_random)]
    q += [tuple(p) for p in xy]                                   # every vertex
    for t in mesh.tri[: min(len(mesh.tri), 200)]:                 # edge midpoints (rounded)
        for k in range(3):
            a, b = xy[t[k]], xy[t[(k + 1) % 3]]
            q.append(((a[0] + b[0]) / 2, (a[1] + b[1]) / 2))
    q += [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (1.0, 1.0), (0.5, 0.0), (0.0, 0.5), (1.0, 0.37), (0.61, 1.0)]
    return np.array(q, dtype=np.float64)


def _brute(mesh, q):
    tri = mesh.tri
    best, count, degen = -1, 0, False
    for j in range(tri.shape[0]):
        s = contains(mesh.xy, tri[j], q)
        if min(s) >= 0:
            if count == 0:
                best, degen = j, (0 in s)
            count += 1
    return best, count, degen


@pytest.mark.parametrize("M,jitter,seed,shuffle", [(3, 0.25, 1, False), (4, 0.25, 7, True),
                                                    (6, 0.0, 0, False), (5, 0.2, 11, True)])
def test_locate_matches_brute_force(M, jitter, seed, shuffle):
    mesh = si.grid_mesh(M, jitter=jitter, seed=seed)
    if shuffle:
        mesh = shuffled(mesh, seed + 100)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    rnd = random.Random(seed)
    q = _queries(mesh, rnd)
    tri, flags = om.locate(q)
    for i in range(q.shape[0]):
        best, count, degen = _brute(mesh, q[i])
        assert best >= 0
        assert tri[i] == best, (i, q[i], tri[i], best)
        assert bool(flags[i] & oracle.FLAG_DEGENERATE) == degen
        assert bool(flags[i] & oracle.FLAG_MULTI) == (count > 1)


def _paper_direct_location(M, xi, eta):
    """The paper's structured-grid formula in exact rationals."""
    xi, eta = F(float(xi)), F(float(eta))
    dx = F(1, M)
    l = math.floor(xi / dx)
    m = math.floor(eta / dx)
    l, m = min(max(l, 0), M - 1), min(max(m, 0), M - 1)
    if xi - l * dx < eta - m * dx:
        return 2 * (M * m + l)
    return 2 * (M * m + l) + 1


@pytest.mark.parametrize("M", [4, 16, 64])
def test_locate_matches_paper_structured_formula(M):
    mesh = si.courant_grid(M)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    rnd = np.random.default_rng(M)
    q = rnd.random((4000, 2))
    tri, flags = om.locate(q)
    nondeg = (flags & oracle.FLAG_DEGENERATE) == 0
    assert nondeg.sum() > 3900
    for i in np.nonzero(nondeg)[0]:
        assert tri[i] == _paper_direct_location(M, q[i, 0], q[i, 1])


def test_degenerate_points_on_structured_grid():
    """On a grid line or diagonal the formula and the oracle may pick
    different (equally valid) triangles; the oracle's pick must contain the
    point and be the lowest-index container."""
    M = 8
    mesh = si.courant_grid(M)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    pts = np.array([[3 / 8, 0.3], [0.3, 5 / 8], [0.25 + 1 / 64, 0.25 + 1 / 64], [0.5, 0.5], [1.0, 0.125]])
    tri, flags = om.locate(pts)
    for i, p in enumerate(pts):
        assert flags[i] & oracle.FLAG_DEGENERATE
        assert min(contains(mesh.xy, mesh.tri[tri[i]], p)) >= 0
        assert tri[i] == min(j for j in range(mesh.n_tri) if min(contains(mesh.xy, mesh.tri[j], p)) >= 0)


def test_bin_count_rule():
    mesh = si.grid_mesh(10, 0.25, 3)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    assert om.bins == math.ceil(math.sqrt(mesh.n_tri / 2))


def _brute_pair(mesh, qh, ql):
    """Lowest containing triangle of qh + ql, its degeneracy and the number of
    containers, in rationals."""
    from exact import orient_pair
    best, count, degen = -1, 0, False
    for j in range(mesh.n_tri):
        p1, p2, p3 = (mesh.xy[v] for v in mesh.tri[j])
        s = (orient_pair(p2, p3, qh, ql), orient_pair(p3, p1, qh, ql), orient_pair(p1, p2, qh, ql))
        if min(s) >= 0:
            if count == 0:
                best, degen = j, (0 in s)
            count += 1
    return best, count, degen


@pytest.mark.parametrize("M,jitter,seed", [(3, 0.25, 2), (5, 0.0, 0), (4, 0.2, 13)])
def test_locate_pair_points_matches_brute_force(M, jitter, seed):
    """Location of points given as exact sums of two doubles per coordinate
    (the double-float kernel's feet): brute force over every triangle in
    rationals, including points that lie exactly on an edge only through
    their low parts, and points a remainder-ulp off an edge."""
    mesh = shuffled(si.grid_mesh(M, jitter=jitter, seed=seed), seed + 7)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    rnd = random.Random(seed)
    qh, ql = [], []
    for _ in range(150):
        qh.append((rnd.random(), rnd.random()))
        ql.append(tuple(rnd.uniform(-1, 1) * 2.0 ** rnd.randint(-80, -55) for _ in range(2)))
    for t in mesh.tri[: min(mesh.n_tri, 30)]:
        for k in range(3):
            a, b = (F(float(c)) for c in mesh.xy[t[k]]), (F(float(c)) for c in mesh.xy[t[(k + 1) % 3]])
            a, b = tuple(a), tuple(b)
            s = F(rnd.randint(1, 2**40 - 1), 2**40)
            q = (a[0] + s * (b[0] - a[0]), a[1] + s * (b[1] - a[1]))
            hx, hy = float(q[0]), float(q[1])
            lx, ly = float(q[0] - F(hx)), float(q[1] - F(hy))
            if F(hx) + F(lx) != q[0] or F(hy) + F(ly) != q[1]:
                continue
            qh.append((hx, hy))
            ql.append((lx, ly))                                   # exactly on the edge
            qh.append((hx, hy))
            ql.append((math.nextafter(lx, math.inf) if lx else 2.0**-1074, ly))   # just off it
    # a point nudged off a boundary edge leaves the square: keep covered points
    brute = [_brute_pair(mesh, h, l) for h, l in zip(qh, ql)]
    keep = [i for i, b in enumerate(brute) if b[0] >= 0]
    assert len(keep) >= len(brute) - 30
    qh, ql = np.array(qh)[keep], np.array(ql)[keep]
    brute = [brute[i] for i in keep]
    tri, flags = om.locate(qh, ql)
    on_edge = 0
    for i in range(qh.shape[0]):
        best, count, degen = brute[i]
        assert tri[i] == best, (i, qh[i], ql[i], tri[i], best)
        assert bool(flags[i] & oracle.FLAG_DEGENERATE) == degen
        assert bool(flags[i] & oracle.FLAG_MULTI) == (count > 1)
        on_edge += degen
    assert on_edge >= 20
    # the exact signs of the located triangle: all >= 0, a zero iff degenerate
    sg = om.signs(tri, qh, ql)
    assert np.all(sg >= 0)
    assert np.array_equal((sg == 0).any(axis=1), (flags & oracle.FLAG_DEGENERATE) != 0)
    # zero remainders: the plain location
    t0, f0 = om.locate(qh)
    t1, f1 = om.locate(qh, np.zeros_like(qh))
    assert np.array_equal(t0, t1) and np.array_equal(f0, f1)


def test_signs_match_rationals_and_flag_non_triangles():
    mesh = si.grid_mesh(4, 0.25, 21)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    rnd = np.random.default_rng(4)
    q = rnd.random((200, 2))
    tri = rnd.integers(0, mesh.n_tri, 200).astype(np.int32)
    tri[:3] = (-1, mesh.n_tri, -5)
    sg = om.signs(tri, q)
    assert np.all(sg[:3] == -2)
    for i in range(3, 200):
        assert tuple(sg[i]) == contains(mesh.xy, mesh.tri[tri[i]], q[i])

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

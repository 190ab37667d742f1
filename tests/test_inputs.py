"""Checks of the synthetic input generator (meshes, fields, configs)."""
import numpy as np
import pytest

import sl_inputs as si
from sl_inputs.meshes import shuffled
from exact import orient


@pytest.mark.parametrize("M,jitter,graded", [(4, 0.25, False), (9, 0.25, False), (8, 0.2, True), (6, 0.0, False)])
def test_small_meshes_are_valid(M, jitter, graded):
    m = si.grid_mesh(M, jitter=jitter, seed=5, graded=graded)
    assert m.n_nodes == (M + 1) ** 2 and m.n_tri == 2 * M * M
    for t in m.tri:                                    # CCW, exactly
        assert orient(m.xy[t[0]], m.xy[t[1]], m.xy[t[2]]) > 0
    x, y = m.xy[:, 0], m.xy[:, 1]
    assert x.min() == 0.0 and x.max() == 1.0 and y.min() == 0.0 and y.max() == 1.0
    # every node of the outer rows/columns lies exactly on the boundary
    g = m.xy.reshape(M + 1, M + 1, 2)
    assert np.all(g[:, 0, 0] == 0) and np.all(g[:, -1, 0] == 1)
    assert np.all(g[0, :, 1] == 0) and np.all(g[-1, :, 1] == 1)
    # total area is 1 and every edge is shared by at most two triangles
    p = m.xy[m.tri]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert abs(area.sum() - 1.0) < 1e-12
    edges = {}
    for t in m.tri:
        for k in range(3):
            e = (t[(k + 1) % 3], t[(k + 2) % 3])
            assert e not in edges                        # consistent orientation
            edges[e] = 1
    boundary = [e for e in edges if (e[1], e[0]) not in edges]
    assert len(boundary) == 4 * M


def test_jitter_bounds_and_reproducibility():
    a = si.grid_mesh(32, 0.25, 9)
    b = si.grid_mesh(32, 0.25, 9)
    c = si.grid_mesh(32, 0.25, 10)
    assert np.array_equal(a.xy, b.xy) and np.array_equal(a.tri, b.tri)
    assert not np.array_equal(a.xy, c.xy)
    base = si.courant_grid(32)
    assert np.abs(a.xy - base.xy).max() <= 0.25 / 32


def test_shuffled_mesh_is_same_triangulation():
    m = si.grid_mesh(5, 0.25, 2)
    s = shuffled(m, 3)
    A = {frozenset(map(tuple, m.xy[t])) for t in m.tri}
    B = {frozenset(map(tuple, s.xy[t])) for t in s.tri}
    assert A == B
    for t in s.tri:
        assert orient(s.xy[t[0]], s.xy[t[1]], s.xy[t[2]]) > 0


def test_large_mesh_ccw_float_check():
    m = si.grid_mesh(256, 0.2, 3, graded=True)
    p = m.xy[m.tri]
    d = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    assert d.min() > 0


def test_configs_shapes():
    c1 = si.config("C1")
    assert c1.mesh.n_nodes == 4225 and c1.mesh.n_tri == 8192 and c1.n_steps == 20
    assert c1.field.kind == si.FIELD_SWIRL and c1.dt == 0.05
    assert abs(c1.v0.max() - 1.0) < 1e-2
    b = si.batch_config(16)
    assert len(b) == 16
    for p in b:
        assert 2e3 * 0.8 <= p.mesh.n_nodes <= 2e5 * 1.2
        assert p.field.kind in (si.FIELD_ROTATION, si.FIELD_SWIRL, si.FIELD_FOURIER8)
        courant = p.dt * p.field.scale * p.mesh.M
        assert 4.99 <= courant <= 30.01

"""Pins the oracle's step (Euler foot, clip, P1 interpolation, time
argument) against closed forms, invariants and convergence.

Eq. 4 (Euler foot) and Algorithm 2 define the step; P1 interpolation
reproduces linear functions exactly (Remark 1: I[V] = sum theta_k v_k with
barycentric theta), which gives closed-form results for linear data under
any field, and for all steps under affine fields.
"""
import os

import numpy as np
import pytest

import oracle
import sl_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lin(xy, a=0.25, b=1.0, c=-0.5):
    return a + b * xy[..., 0] + c * xy[..., 1]


def test_field_golden_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fields.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for kind, params, x, y, t, fx, fy, tol in rows:
        p = np.zeros(48)
        vals = [float(v) for v in params.split(",")]
        p[: len(vals)] = vals
        gx, gy = oracle.field(int(kind), p, float(x), float(y), float(t))
        assert abs(gx - float(fx)) <= float(tol) and abs(gy - float(fy)) <= float(tol), (kind, x, y, t, gx, gy)


def test_paper_field_has_unit_norm():
    """Sec. 4: |f| = 1 everywhere, L_x = C0, L_t = C1."""
    p = si.paper_field(8 * np.pi, 2 * np.pi).packed()
    rnd = np.random.default_rng(0)
    for x, y, t in rnd.random((200, 3)):
        fx, fy = oracle.field(si.FIELD_PAPER, p, x, y, t)
        assert abs(np.hypot(fx, fy) - 1.0) < 1e-15


def test_fourier_field_is_a_stream_function_gradient():
    """f = (d psi/dy, -d psi/dx) with psi the 8-mode stream function:
    compare with central differences of psi written from its definition,
    and check divergence-freeness and tangency to the boundary."""
    fld = si.fourier8_field(42)
    p = fld.packed()
    k, l, a, phi = p[0:32:4], p[1:32:4], p[2:32:4], p[3:32:4]

    def psi(x, y, t):
        return np.sum(a * np.cos(2 * np.pi * t + phi) * np.sin(k * np.pi * x) * np.sin(l * np.pi * y))

    h = 1e-6
    rnd = np.random.default_rng(1)
    for x, y, t in rnd.random((50, 3)):
        fx, fy = oracle.field(si.FIELD_FOURIER8, p, x, y, t)
        dpy = (psi(x, y + h, t) - psi(x, y - h, t)) / (2 * h)
        dpx = (psi(x + h, y, t) - psi(x - h, y, t)) / (2 * h)
        assert abs(fx - dpy) < 1e-6 and abs(fy + dpx) < 1e-6
        div = ((oracle.field(si.FIELD_FOURIER8, p, x + h, y, t)[0] - oracle.field(si.FIELD_FOURIER8, p, x - h, y, t)[0])
               + (oracle.field(si.FIELD_FOURIER8, p, x, y + h, t)[1] - oracle.field(si.FIELD_FOURIER8, p, x, y - h, t)[1])) / (2 * h)
        assert abs(div) < 1e-5
    # psi vanishes on every side of the square, so f is tangent to the sides:
    # the normal component is exactly 0 there (sin(k pi) = 0 exactly for
    # integer k; a boundary node's foot then stays on its side, reading c2)
    for s in rnd.random(20):
        for side in (0.0, 1.0):
            assert oracle.field(si.FIELD_FOURIER8, p, side, s, 0.3)[0] == 0.0
            assert oracle.field(si.FIELD_FOURIER8, p, s, side, 0.3)[1] == 0.0


def test_trigonometric_fields_match_their_formulas():
    """The swirl and stream-function fields against their formulas written
    out in numpy (np.sin of the product with pi): within a few ulps of the
    field's size at interior points, so the exact argument reduction of the
    oracle's sine changes no value beyond rounding; exactly zero normal
    component on all four sides."""
    rnd = np.random.default_rng(7)
    sw = si.swirl_field()
    fo = si.fourier8_field(9)
    p = fo.packed()
    k, l, a, phi = p[0:32:4], p[1:32:4], p[2:32:4], p[3:32:4]
    for x, y, t in rnd.random((200, 3)):
        c = np.cos(np.pi * t / sw.packed()[0])
        fx = c * np.sin(np.pi * x) ** 2 * np.sin(2 * np.pi * y)
        fy = -c * np.sin(np.pi * y) ** 2 * np.sin(2 * np.pi * x)
        gx, gy = oracle.field(sw.kind, sw.packed(), x, y, t)
        assert abs(gx - fx) <= 1e-15 and abs(gy - fy) <= 1e-15
        am = a * np.cos(2 * np.pi * t + phi)
        fx = np.sum(am * np.sin(k * np.pi * x) * (l * np.pi) * np.cos(l * np.pi * y))
        fy = -np.sum(am * (k * np.pi) * np.cos(k * np.pi * x) * np.sin(l * np.pi * y))
        gx, gy = oracle.field(fo.kind, p, x, y, t)
        scale = np.sum(np.abs(a) * (k + l) * np.pi)
        assert abs(gx - fx) <= 1e-14 * scale and abs(gy - fy) <= 1e-14 * scale
    for s in rnd.random(20):
        for side in (0.0, 1.0):
            for fld in (sw, fo):
                assert oracle.field(fld.kind, fld.packed(), side, s, 0.3)[0] == 0.0
                assert oracle.field(fld.kind, fld.packed(), s, side, 0.3)[1] == 0.0


def _mesh(M=24, seed=4):
    m = si.grid_mesh(M, 0.25, seed)
    return m, oracle.OracleMesh(m.xy, m.tri)


def test_linear_data_reproduced_after_one_step_any_field():
    """P1 reproduces linears, so V^1_i = u0(X_i) for the oracle's own feet."""
    m, om = _mesh()
    v0 = _lin(m.xy)
    for fld, dt in [(si.swirl_field(), 0.05), (si.fourier8_field(3), 0.02), (si.paper_field(), 0.03),
                    (si.rotation_field(), 0.02)]:
        v1, tri, flags, ft = om.step(fld.kind, fld.packed(), dt, 0, v0)
        assert np.abs(v1 - _lin(ft)).max() <= 1e-14, fld.kind


def test_translation_closed_form_uses_t_n_plus_1():
    """Time-dependent translation f = (p0 + p3 t, p4 + p7 t): the foot is
    x - dt f(t_{n+1}) (Eq. 4).  With linear data the new value is the data at
    that point; using t_n instead would miss by dt^2 (p3 b + p7 c)."""
    m, om = _mesh()
    dt, n = 0.01, 3
    p = np.zeros(48)
    p[[0, 3, 4, 7]] = (0.3, 2.0, -0.2, -1.0)
    v0 = _lin(m.xy)
    v1, tri, flags, ft = om.step(si.FIELD_AFFINE, p, dt, n, v0)
    t1 = (n + 1) * dt
    X = m.xy[:, 0] - dt * (0.3 + 2.0 * t1)
    Y = m.xy[:, 1] - dt * (-0.2 - 1.0 * t1)
    inside = (X >= 0) & (X <= 1) & (Y >= 0) & (Y <= 1)
    assert inside.sum() > 0.8 * m.n_nodes
    assert np.all((flags[inside] & oracle.FLAG_CLIPPED) == 0)
    assert np.all((flags[~inside] & oracle.FLAG_CLIPPED) != 0)
    want = 0.25 + 1.0 * X - 0.5 * Y
    assert np.abs(v1[inside] - want[inside]).max() < 1e-14


def test_rotation_closed_form():
    m, om = _mesh()
    dt, w = 0.02, 2 * np.pi
    v0 = _lin(m.xy)
    v1, tri, flags, ft = om.step(si.FIELD_ROTATION, si.rotation_field(w).packed(), dt, 0, v0)
    X = m.xy[:, 0] + dt * w * (m.xy[:, 1] - 0.5)
    Y = m.xy[:, 1] - dt * w * (m.xy[:, 0] - 0.5)
    inside = (X >= 0) & (X <= 1) & (Y >= 0) & (Y <= 1)
    assert np.abs(v1[inside] - (0.25 + X[inside] - 0.5 * Y[inside])).max() < 1e-14


def test_contracting_affine_field_many_steps():
    """f = k (x - c): X = c + (1 - k dt)(x - c) stays inside; after n steps
    linear data equal u0(c + (1 - k dt)^n (x - c))."""
    m, om = _mesh(32, 8)
    k, cx, cy, dt, steps = 3.0, 0.4, 0.6, 0.05, 12
    p = np.zeros(48)
    p[:8] = (-k * cx, k, 0.0, 0.0, -k * cy, 0.0, k, 0.0)
    v0 = _lin(m.xy)
    v = om.run(si.FIELD_AFFINE, p, dt, 0, steps, v0)
    r = (1 - k * dt) ** steps
    want = _lin(np.stack([cx + r * (m.xy[:, 0] - cx), cy + r * (m.xy[:, 1] - cy)], 1))
    assert np.abs(v - want).max() < 1e-13


def test_zero_field_is_identity_and_degenerate():
    m, om = _mesh()
    v0 = si.gaussian(m.xy)
    v1, tri, flags, ft = om.step(si.FIELD_ZERO, np.zeros(48), 0.1, 0, v0)
    assert np.array_equal(v1, v0)
    assert np.all(flags & oracle.FLAG_DEGENERATE)
    assert np.array_equal(ft, m.xy)


def test_constant_data_and_maximum_principle():
    p = si.config("C1", M=48)
    om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
    c = si.constant(p.mesh.xy, 0.7)
    v = om.run(p.field.kind, p.field.packed(), p.dt, 0, 5, c)
    assert np.abs(v - 0.7).max() < 1e-15
    v = p.v0.copy()
    for n in range(p.n_steps):
        w, _, _, _ = om.step(p.field.kind, p.field.packed(), p.dt, n, v, want_feet=False)
        assert w.min() >= v.min() - 1e-15 and w.max() <= v.max() + 1e-15
        v = w


def test_swirl_pauses_at_half_period():
    """With f evaluated at t_{n+1}, the step that ends at t = 1/2 sees
    cos(pi/2) ~ 6e-17 and leaves the data unchanged to round-off."""
    p = si.config("C1", M=32)
    om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
    v = om.run(p.field.kind, p.field.packed(), p.dt, 0, 9, p.v0)
    w, _, _, _ = om.step(p.field.kind, p.field.packed(), p.dt, 9, v)
    assert np.abs(w - v).max() < 1e-14
    w2, _, _, _ = om.step(p.field.kind, p.field.packed(), p.dt, 8, v)
    assert np.abs(w2 - v).max() > 1e-3


def test_clipped_feet_lie_on_boundary_and_segment():
    """Clip reading: the segment x_i -> x_i - dt f stops at the boundary."""
    m, om = _mesh(20, 2)
    p = np.zeros(48)
    p[[0, 4]] = (-3.0, 1.7)              # strong translation: many feet leave
    dt = 0.1
    ft, clipped = oracle.feet(si.FIELD_AFFINE, p, dt, 0, m.xy)
    q = m.xy - dt * np.array([-3.0, 1.7])
    assert clipped.sum() > 0.3 * m.n_nodes
    for i in np.nonzero(clipped)[0]:
        X, x, qq = ft[i], m.xy[i], q[i]
        assert X[0] in (0.0, 1.0) or X[1] in (0.0, 1.0)
        assert 0.0 <= X[0] <= 1.0 and 0.0 <= X[1] <= 1.0
        d, e = qq - x, X - x
        assert abs(d[0] * e[1] - d[1] * e[0]) <= 1e-15 * np.hypot(*d)
        assert d @ e >= -1e-300 and np.hypot(*e) <= np.hypot(*d)
    for i in np.nonzero(clipped == 0)[0]:
        assert np.array_equal(ft[i], q[i])


def test_corner_clip_snaps_both_coordinates():
    ft, c = oracle.feet(si.FIELD_AFFINE, np.r_[-1.0, 0, 0, 0, -1.0, 0, 0, 0, np.zeros(40)], 0.5, 0,
                        np.array([[0.75, 0.75], [1.0, 1.0], [0.9, 0.8]]))
    assert c.all()
    assert tuple(ft[0]) == (1.0, 1.0) and tuple(ft[1]) == (1.0, 1.0)
    assert ft[2][0] == 1.0 and abs(ft[2][1] - 0.9) < 1e-15


@pytest.mark.slow
def test_swirl_converges_under_refinement():
    """Swirl returns to u0 at t = 1; with the Courant number fixed the
    error of this first-order scheme falls as the mesh is refined."""
    errs = []
    for M in (32, 64, 128):
        p = si.config("C1", M=M)
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        steps = int(round(20 * M / 64))
        dt = 1.0 / steps
        v = om.run(p.field.kind, p.field.packed(), dt, 0, steps, p.v0)
        errs.append(np.abs(v - p.v0).mean())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.6 * errs[0]


def test_exclusion_keeps_the_value_of_nodes_whose_foot_leaves():
    """Sec. 4 excludes the nodes whose Euler foot leaves the domain.  A
    translation by (+0.25, 0) (f = (-0.25, 0), dt = 1) sends exactly the
    nodes with x > 0.75 out: those keep V^n and are flagged, the others get
    the clip-mode result bitwise (their feet are inside, so nothing else
    changes)."""
    m, om = _mesh()
    p = np.zeros(48)
    p[0] = -0.25
    v0 = np.sin(3.0 * m.xy[:, 0]) + m.xy[:, 1] ** 2
    vx, tri_x, fl_x, ft_x = om.step(si.FIELD_AFFINE, p, 1.0, 0, v0, exclude=True)
    vc, tri_c, fl_c, _ = om.step(si.FIELD_AFFINE, p, 1.0, 0, v0)
    x = m.xy[:, 0]
    out = (fl_x & oracle.FLAG_EXCLUDED) != 0
    assert np.all(out[x > 0.75 + 1e-12]) and not np.any(out[x < 0.75 - 1e-12])
    assert 0.1 * m.n_nodes < out.sum() < 0.4 * m.n_nodes
    assert np.array_equal(vx[out], v0[out])
    assert np.all(tri_x[out] == -1)
    # excluded feet are reported unclipped: outside the square, on the translated node
    assert np.all(ft_x[out, 0] > 1.0) and np.allclose(ft_x[out, 0], x[out] + 0.25, atol=1e-15)
    keep = ~out
    assert np.array_equal(vx[keep], vc[keep]) and np.array_equal(tri_x[keep], tri_c[keep])
    assert np.all((fl_c[keep] & oracle.FLAG_CLIPPED) == 0)


def test_exclusion_of_the_paper_field_matches_the_unclipped_feet():
    """The paper's rotating field (Sec. 4) with a large step: a node is
    excluded exactly when its unclipped Euler foot (Eq. 4) lies outside the
    square, and the exclusion does not depend on V."""
    m, om = _mesh()
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    dt = 0.05
    v0 = np.cos(2.0 * m.xy[:, 0]) * m.xy[:, 1]
    _, _, flags, feet = om.step(f.kind, f.packed(), dt, 2, v0, exclude=True)
    t = 3 * dt
    r = np.hypot(m.xy[:, 0] - 0.5, m.xy[:, 1] - 0.5)
    qx = m.xy[:, 0] - dt * np.cos(2 * np.pi * r + 2 * np.pi * t)
    qy = m.xy[:, 1] - dt * np.sin(2 * np.pi * r + 2 * np.pi * t)
    margin = np.minimum(np.minimum(np.abs(qx), np.abs(qx - 1)), np.minimum(np.abs(qy), np.abs(qy - 1)))
    outside = ~((qx >= 0) & (qx <= 1) & (qy >= 0) & (qy <= 1))
    sure = margin > 1e-12
    out = (flags & oracle.FLAG_EXCLUDED) != 0
    assert out.sum() > 0
    assert np.array_equal(out[sure], outside[sure])
    _, _, flags2, _ = om.step(f.kind, f.packed(), dt, 2, 2.0 * v0 + 1.0, exclude=True)
    assert np.array_equal(flags, flags2)
